"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: the 512-image mixed-size batch (one persistent launch per
pass, autotuned mapping, 8-iteration decode), every image checked against
the oracle, and one 4096x4096 request through the server."""
import os

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


def _oracle_pool():
    from concurrent.futures import ThreadPoolExecutor
    # the oracle's C calls release the GIL (ctypes), so threads run in parallel
    return ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1))


def test_mixed_batch_512_images_all(fic, orc):
    """Every one of the 512 mixed-size images (Section 3 encoder, quadtree
    32->4, RMS 8): records, split masks, fit counts and the 8-iteration
    decode equal the oracle's, in the benchmark's autotuned launch."""
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

    def want(i):
        im = imgs[i]
        leaves, split, fits = orc.encode(im, op)
        return leaves, split, fits, orc.decode(leaves, im.shape[1], im.shape[0], op, 8)

    bad = []
    with _oracle_pool() as ex:
        for i, (leaves, split, fits, dec) in enumerate(ex.map(want, range(len(imgs)))):
            got = plan.outs[i].to_host()
            ok = (got["records"].shape == leaves.shape
                  and np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
                  and np.array_equal(got["split"], split) and got["fits"] == fits
                  and got["tile_offsets"][-1] == len(leaves)
                  and np.array_equal(dplan.outs[i].cpu().numpy(), dec))
            if not ok:
                bad.append(i)
    assert not bad, f"{len(bad)} of {len(imgs)} images differ from the oracle, first {bad[:8]}"


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
