"""The request server (fic_submit & co): every job's result equals the oracle
and the standalone call whatever it was batched with, admission respects
the memory budget, and the documented error paths hold."""
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


# (mode, W, H, bmax, bmin, thr, extra params)
ENC_JOBS = [
    ("mns", 256, 256, 32, 4, 8.0, {}),
    ("mns", 128, 384, 16, 4, 6.0, {}),
    ("mns", 512, 128, 32, 4, 12.0, {}),
    ("nosearch", 192, 192, 32, 4, 8.0, {}),
    ("local", 128, 128, 32, 4, 8.0, {}),
    ("local", 96, 64, 16, 4, 6.0, {"local_radius": 8, "local_step": 2}),
    ("exhaustive", 64, 64, 8, 8, 8.0, {"engine": 0}),
    ("exhaustive", 80, 48, 8, 8, 8.0, {"engine": 1, "dom_step": 2, "isometries": 4}),
]


def _oracle_kw(kw):
    return {k: v for k, v in kw.items() if k != "engine"}


def _enc_job(fic, orc, i, job):
    mode, W, H, bmax, bmin, thr, kw = job
    img = synth.gaussian_scene(W, 900 + i, H=H)
    return img, fic.params(mode, bmax, bmin, thr, **kw), orc.make_params(mode, bmax, bmin, thr, **_oracle_kw(kw))


def test_mixed_jobs_match_oracle(fic, orc):
    srv = fic.Server(hbm_budget_bytes=512 << 20, streams=3, max_batch=16)
    try:
        enc, dec = [], []
        for rep in range(2):
            for i, job in enumerate(ENC_JOBS):
                img, p, op = _enc_job(fic, orc, i, job)
                enc.append((srv.submit_encode(img, p), img, op))
        # decode jobs: oracle streams, two iteration counts (two batch keys)
        for i, job in enumerate(ENC_JOBS):
            img, p, op = _enc_job(fic, orc, i, job)
            leaves, _, _ = orc.encode(img, op)
            for iters in (4, 9):
                rec = leaves.view(fic.RECORD_DTYPE)
                dec.append((srv.submit_decode(rec, img.shape[1], img.shape[0], p, iters), leaves, img.shape, op,
                            iters))
        for t, img, op in enc:
            got = srv.wait(t, 60000)
            leaves, split, fits = orc.encode(img, op)
            assert len(got["records"]) == len(leaves)
            assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
            assert np.array_equal(got["split"], split)
            assert got["fits"] == fits
        for t, leaves, (H, W), op, iters in dec:
            got = srv.wait(t, 60000)
            assert np.array_equal(got["image"], orc.decode(leaves, W, H, op, iters))
        st = srv.stats()
        n = len(enc) + len(dec)
        assert st["submitted"] == n and st["completed"] == n and st["rejected"] == 0
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["batches"] >= 1 and st["mean_batch"] >= 1.0
        assert 0 < st["peak_device_bytes"] <= 512 << 20
    finally:
        srv.close()


def test_result_independent_of_batch_mates(fic, orc):
    """One job alone, and the same job among 24 others of different sizes
    and thresholds: identical bytes, equal to the standalone fic_encode."""
    img = synth.gaussian_scene(256, 4242)
    p = fic.params("mns", 32, 4, 8.0)
    standalone = fic.fic_encode(torch.from_numpy(img).cuda(), p).to_host()
    srv = fic.Server(hbm_budget_bytes=256 << 20, streams=2, max_batch=32)
    try:
        alone = srv.wait(srv.submit_encode(img, p))
        mates = []
        for i in range(12):
            side = [64, 128, 192, 320][i % 4]
            mates.append(srv.submit_encode(synth.gaussian_scene(side, 50 + i), fic.params("mns", 32, 4, 4.0 + i)))
        mid = srv.submit_encode(img, p)
        for i in range(12):
            mates.append(srv.submit_encode(synth.voronoi(128, 70 + i), fic.params("mns", 32, 4, 10.0)))
        mixed = srv.wait(mid)
        for t in mates:
            srv.wait(t)
        for got in (alone, mixed):
            assert np.array_equal(got["records"].view(np.uint8), standalone["records"].view(np.uint8))
            assert np.array_equal(got["split"], standalone["split"])
    finally:
        srv.close()


def test_small_budget_admits_in_turn(fic, orc):
    """A budget that holds about two 512x512 jobs: every job still completes,
    bit-exact, and the device arena never exceeds the budget."""
    p = fic.params("mns", 32, 4, 8.0)
    op = orc.make_params("mns", 32, 4, 8.0)
    budget = 8 << 20
    srv = fic.Server(hbm_budget_bytes=budget, streams=2, max_batch=8)
    try:
        imgs = [synth.gaussian_scene(512, 300 + i) for i in range(8)]
        ts = [srv.submit_encode(im, p) for im in imgs]
        for t, im in zip(ts, imgs):
            got = srv.wait(t, 60000)
            leaves, split, _ = orc.encode(im, op)
            assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
        st = srv.stats()
        assert st["completed"] == 8 and st["peak_device_bytes"] <= budget
    finally:
        srv.close()


def test_budget_rejection(fic):
    srv = fic.Server(hbm_budget_bytes=4 << 20, streams=1)
    try:
        with pytest.raises(fic.FicError) as e:
            srv.submit_encode(np.zeros((2048, 2048), dtype=np.uint8), fic.params("mns", 32, 4, 8.0))
        assert e.value.code == -7
        assert srv.stats()["rejected"] == 1
    finally:
        srv.close()


def test_queue_capacity_and_poll(fic):
    srv = fic.Server(hbm_budget_bytes=64 << 20, streams=1, queue_capacity=2)
    try:
        p = fic.params("mns", 32, 4, 8.0)
        img = synth.gaussian_scene(128, 5)
        a = srv.submit_encode(img, p)
        b = srv.submit_encode(img, p)
        with pytest.raises(fic.FicError) as e:  # two tickets held, none released yet
            srv.submit_encode(img, p)
        assert e.value.code == -8
        got = srv.wait(a, 60000)
        assert len(got["records"]) > 0
        srv.wait(b, 60000)
        c = srv.submit_encode(img, p)  # room again
        while srv.poll(c) is None:
            pass
    finally:
        srv.close()


def test_decode_rejects_malformed_records(fic, orc):
    img = synth.gaussian_scene(128, 6)
    p = fic.params("mns", 32, 4, 8.0)
    leaves, _, _ = orc.encode(img, orc.make_params("mns", 32, 4, 8.0))
    rec = leaves.view(fic.RECORD_DTYPE).copy()
    srv = fic.Server(hbm_budget_bytes=64 << 20, streams=1)
    try:
        bad_order = rec[::-1].copy()
        missing = rec[:-1].copy()
        outside = rec.copy()
        outside["x"][0] = 4000
        bad_code = rec.copy()
        bad_code["q"][0] = 200  # 7-bit luminance codebook
        for bad in (bad_order, missing, outside, bad_code):
            with pytest.raises(fic.FicError) as e:
                srv.submit_decode(bad, 128, 128, p, 4)
            assert e.value.code == -2
        srv.wait(srv.submit_decode(rec, 128, 128, p, 4), 60000)
    finally:
        srv.close()


def test_destroy_finishes_pending_jobs(fic):
    srv = fic.Server(hbm_budget_bytes=64 << 20, streams=2)
    p = fic.params("mns", 32, 4, 8.0)
    for i in range(10):
        srv.submit_encode(synth.gaussian_scene(256, 600 + i), p)
    srv.close()  # returns once every accepted job has run
