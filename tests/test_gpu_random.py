"""Randomised parity: encoder and decoder against the oracle over a seeded
sweep of sizes, quadtree depths, codebooks, thresholds and modes (small
images, so the oracle keeps up)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cases(n=40, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        bmax = int(rng.choice([8, 16, 32]))
        bmin = int(rng.choice([b for b in (4, 8, 16, 32) if b <= bmax and bmax // b <= 8]))
        tw, th = int(rng.integers(2, 8)), int(rng.integers(2, 6))
        W, H = bmax * tw, bmax * th
        W += (-W) % 16
        H += (-H) % 16
        if W % bmax or H % bmax:
            W, H = 16 * bmax // np.gcd(16, bmax) * 2, 16 * bmax // np.gcd(16, bmax) * 2
        mode = str(rng.choice(["mns", "mns", "nosearch", "local"]))
        kw = {"s_bits": int(rng.integers(2, 8)), "o_bits": int(rng.integers(4, 9))}
        if mode == "mns":
            kw["phase2_domain"] = int(rng.integers(0, 2))
        if mode == "local":
            kw["local_radius"] = int(rng.choice([0, 4, 8, 16]))
            kw["local_step"] = int(rng.choice([2, 4]))
        thr = [float(v) for v in rng.uniform(1.0, 20.0, size=4)] if rng.uniform() < 0.5 else float(rng.uniform(0, 24))
        kind = int(rng.integers(0, 3))
        out.append((i, mode, bmax, bmin, W, H, thr, kw, kind, int(rng.integers(1, 9))))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"c{c[0]}-{c[1]}-{c[2]}-{c[3]}-{c[4]}x{c[5]}")
def test_random_configuration(orc, case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    i, mode, bmax, bmin, W, H, thr, kw, kind, iters = case
    if kind == 0:
        img = synth.gaussian_scene(W, 7000 + i, H=H)
    elif kind == 1:
        img = synth.voronoi(W, 7000 + i, H=H)
    else:
        img = np.random.default_rng(i).integers(0, 256, size=(H, W), dtype=np.uint8)
    p = fic.params(mode, bmax, bmin, thr, **kw)
    assert fic.validate(W, H, p) == 0, (W, H, bmax, bmin)
    op = orc.make_params(mode, bmax, bmin, thr, **kw)
    st = fic.fic_encode(torch.from_numpy(img).cuda(), p)
    got = st.to_host()
    leaves, split, fits = orc.encode(img, op)
    assert np.array_equal(got["records"].view(np.uint8), leaves.view(np.uint8))
    assert np.array_equal(got["split"], split) and got["fits"] == fits
    dec = fic.fic_decode(st, iters).cpu().numpy()
    assert np.array_equal(dec, orc.decode(leaves, W, H, op, iters))


@pytest.mark.parametrize("b", range(8))
def test_random_batches_equal_single_calls(b):
    """A batch of images of random sizes (one bmax and mode, thresholds per
    image) in one plan equals the images encoded and decoded one by one."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    rng = np.random.default_rng(500 + b)
    bmax = int(rng.choice([8, 16, 32]))
    mode = str(rng.choice(["mns", "nosearch"]))
    imgs, plist = [], []
    for k in range(int(rng.integers(2, 10))):
        W, H = bmax * int(rng.integers(2, 16)), bmax * int(rng.integers(2, 10))
        W += (-W) % 16
        H += (-H) % 16
        imgs.append(synth.gaussian_scene(W, 6000 + 50 * b + k, H=H))
        plist.append(fic.params(mode, bmax, 4, float(rng.uniform(2, 16))))
    plan = fic.EncodePlan([torch.from_numpy(im).cuda() for im in imgs], plist)
    plan.run()
    dplan = fic.DecodePlan(plan.outs)
    dplan.run(7)
    torch.cuda.synchronize()
    for im, p, st, out in zip(imgs, plist, plan.outs, dplan.outs):
        ref = fic.fic_encode(torch.from_numpy(im).cuda(), p)
        a, r = st.to_host(), ref.to_host()
        assert np.array_equal(a["records"].view(np.uint8), r["records"].view(np.uint8))
        assert np.array_equal(a["split"], r["split"]) and a["fits"] == r["fits"]
        assert np.array_equal(out.cpu().numpy(), fic.fic_decode(ref, 7).cpu().numpy())
