"""Exhaustive search (Section 1; flat 8x8 ranges, domains on a grid, eight
isometries) on the GPU: the tensor-core path (tcgen05) and the CUDA-core
path against the oracle and against each other, bit-exact."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ENGINES = {"tensor": 0, "cuda": 1}


@pytest.fixture(scope="module")
def fic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1501_02894_gb300 as fic
    fic.lib()
    return fic


def _encode(fic, img, engine, **kw):
    p = fic.params("exhaustive", 8, 8, 8.0, engine=ENGINES[engine], **kw)
    st = fic.fic_encode(torch.from_numpy(np.ascontiguousarray(img)).cuda(), p)
    return st, st.to_host()


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
@pytest.mark.parametrize("W,H,step,isos", [(64, 64, 4, 8), (128, 96, 4, 8), (96, 64, 2, 8), (64, 80, 4, 1),
                                            (64, 64, 6, 3)])
def test_exhaustive_small_vs_oracle(fic, orc, engine, W, H, step, isos):
    img = synth.gaussian_scene(W, 300 + W + H + step, H=H)
    st, got = _encode(fic, img, engine, dom_step=step, isometries=isos)
    op = orc.make_params("exhaustive", 8, 8, 8.0, dom_step=step, isometries=isos)
    leaves, split, fits = orc.encode(img, op)
    assert len(got["records"]) == len(leaves)
    gb, wb = got["records"].view(np.uint8).reshape(-1, 16), leaves.view(np.uint8).reshape(-1, 16)
    bad = np.nonzero(np.any(gb != wb, axis=1))[0]
    assert bad.size == 0, f"{bad.size} records differ, first {got['records'][bad[0]]} vs {leaves[bad[0]]}"
    assert np.array_equal(got["split"], split)
    assert got["fits"] == fits
    dec = fic.fic_decode(st, 6).cpu().numpy()
    assert np.array_equal(dec, orc.decode(leaves, W, H, op, 6))


@pytest.mark.parametrize("engine", ["tensor", "cuda"])
def test_exhaustive_finds_planted(fic, orc, engine):
    from tests.test_oracle_pins import _plant
    from fractions import Fraction as F
    rng = np.random.default_rng(7)
    img = np.clip(synth.gaussian_scene(64, 8).astype(int) + rng.integers(-40, 40, (64, 64)), 0, 255).astype(np.uint8)
    plants = [(48, 48, 8, 12, 3), (0, 56, 40, 0, 6), (32, 0, 0, 36, 1)]
    for (x, y, dx, dy, iso) in plants:
        _plant(img, x, y, 8, dx, dy, iso, F(3, 4) - F(1, 32), 120)
    _, got = _encode(fic, img, engine)
    rec = got["records"]
    for (x, y, dx, dy, iso) in plants:
        r = rec[(y // 8) * 8 + x // 8]
        assert (int(r["dx"]), int(r["dy"]), int(r["iso"])) == (dx, dy, iso)


@pytest.mark.parametrize("N,sample", [(512, 48), (1024, 16)])
def test_exhaustive_full_size_engines_agree_and_sampled_oracle(fic, orc, N, sample):
    img = synth.gaussian_scene(N, 1 if N == 512 else 9)
    _, a = _encode(fic, img, "tensor")
    _, b = _encode(fic, img, "cuda")
    assert np.array_equal(a["records"].view(np.uint8), b["records"].view(np.uint8))
    assert a["fits"] == b["fits"] == (N // 8) ** 2 * ((N - 16) // 4 + 1) ** 2 * 8
    rng = np.random.default_rng(N)
    idx = np.sort(rng.choice((N // 8) ** 2, size=sample, replace=False))
    xs, ys = (idx % (N // 8)) * 8, (idx // (N // 8)) * 8
    op = orc.make_params("exhaustive", 8, 8, 8.0)
    want = orc.search_ranges(img, op, xs, ys, np.full(sample, 8))
    rec = a["records"][idx]
    for i in range(sample):
        assert (int(rec[i]["k"]), int(rec[i]["q"]), int(rec[i]["dx"]), int(rec[i]["dy"]), int(rec[i]["iso"])) == (
            int(want["k"][i]), int(want["q"][i]), int(want["dx"][i]), int(want["dy"][i]), int(want["iso"][i])), i
