"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the 512-image mixed-size batch (one persistent launch per
pass, autotuned mapping, 8-iteration decode) on a sample of images checked
against the oracle, and one 4096x4096 request through the server."""
import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    fic.lib()
    return fic


def test_mixed_batch_512_images_sampled(fic, orc):
    import bench
    sides = synth.mixed_sides()
    imgs = bench.gen_images([("g", int(s), 1000 + i) for i, s in enumerate(sides)])
    p = fic.params("mns", 32, 4, 8.0)
    d = [torch.from_numpy(im).cuda() for im in imgs]
    plan = fic.EncodePlan(d, p)
    plan.autotune(reps=1)
    plan.run()
    dplan = fic.DecodePlan(plan.outs)
    dplan.autotune(8, reps=1)
    dplan.run(8)
    torch.cuda.synchronize()
    op = orc.make_params("mns", 32, 4, 8.0)
    # every side, first and last image of the batch
    pick = sorted({0, len(imgs) - 1} | {int(np.nonzero(sides == s)[0][0]) for s in (256, 512, 1024, 2048)})
    for i in pick:
        im = imgs[i]
        leaves, split, fits = orc.encode(im, op)
        got = plan.outs[i].to_host()
        assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8)), f"image {i}"
        assert np.array_equal(got["split"], split) and got["fits"] == fits
        want = orc.decode(leaves, im.shape[1], im.shape[0], op, 8)
        assert np.array_equal(dplan.outs[i].cpu().numpy(), want), f"image {i}"
    # every other image: the stream's record count and tile offsets are consistent
    for st in plan.outs:
        h = st.to_host()
        assert h["tile_offsets"][-1] == len(h["records"])


def test_largest_request_through_the_server(fic, orc):
    img = synth.gaussian_scene(4096, 10 ** 6 + 7)
    p = fic.params("mns", 32, 4, 8.0)
    srv = fic.Server(hbm_budget_bytes=2 << 30, streams=2)
    try:
        got = srv.wait(srv.submit_encode(img, p), 120000)
    finally:
        srv.close()
    leaves, split, fits = orc.encode(img, orc.make_params("mns", 32, 4, 8.0))
    assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
    assert np.array_equal(got["split"], split) and got["fits"] == fits


def test_empty_batch_rejected(fic):
    with pytest.raises(fic.FicError):
        fic.fic_encode_batch([], [])
