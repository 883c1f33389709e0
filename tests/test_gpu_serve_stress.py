"""The request server under load: hundreds of encode and decode jobs of many
sizes submitted back to back on four streams (batches overlap, the device
arena is reused while earlier batches still run), every result compared
with the standalone library call on the same input, and a sample with the
oracle."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    fic.lib()
    return fic


def test_many_overlapping_jobs_equal_standalone(fic, orc):
    rng = np.random.default_rng(77)
    sides = [64, 96, 128, 160, 192, 256, 320, 384, 512, 768, 1024]
    pool = {s: synth.gaussian_scene(s, 3000 + s) for s in sides}
    p_enc = fic.params("mns", 32, 4, 8.0)
    # decode inputs and the reference results: standalone calls, one at a time
    ref_enc, ref_dec, streams = {}, {}, {}
    for s, im in pool.items():
        st = fic.fic_encode(torch.from_numpy(im).cuda(), p_enc)
        ref_enc[s] = st.to_host()
        streams[s] = ref_enc[s]["records"]
        for iters in (3, 8):
            ref_dec[(s, iters)] = fic.fic_decode(st, iters).cpu().numpy()
    torch.cuda.synchronize()
    jobs = []
    srv = fic.Server(hbm_budget_bytes=1 << 30, streams=4, max_batch=32, queue_capacity=1 << 12)
    try:
        for i in range(600):
            s = int(rng.choice(sides))
            if rng.random() < 0.7:
                jobs.append(("e", s, srv.submit_encode(pool[s], p_enc)))
            else:
                iters = 3 if rng.random() < 0.5 else 8
                jobs.append(("d", (s, iters), srv.submit_decode(streams[s], s, s, p_enc, iters)))
        for kind, key, t in jobs:
            got = srv.wait(t, 120000)
            if kind == "e":
                want = ref_enc[key]
                assert np.array_equal(got["records"].view(np.uint8), want["records"].view(np.uint8)), key
                assert np.array_equal(got["split"], want["split"]), key
                assert got["fits"] == want["fits"], key
            else:
                assert np.array_equal(got["image"], ref_dec[key]), key
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["rejected"] == 0
        assert st["mean_batch"] > 1.0  # the load did form batches
    finally:
        srv.close()
    # the standalone references themselves against the oracle, on a sample
    op = orc.make_params("mns", 32, 4, 8.0)
    for s in (96, 320):
        leaves, split, fits = orc.encode(pool[s], op)
        assert np.array_equal(ref_enc[s]["records"].view(np.uint8), leaves.view(np.uint8))
        assert np.array_equal(ref_dec[(s, 8)], orc.decode(leaves, s, s, op, 8))
