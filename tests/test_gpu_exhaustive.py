"""Exhaustive search (Section 1; flat 8x8 ranges, domains on a grid, eight
isometries) on the GPU: the tensor-core path (tcgen05) and the CUDA-core
path against the oracle and against each other, bit-exact."""
import os

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


def _search_threaded(orc, img, op, idx, N):
    """The oracle's phase-1 search (Section 1: every grid domain, every
    isometry) of the 8x8 ranges with raster indices `idx`, spread over host
    threads (ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    xs, ys = (idx % (N // 8)) * 8, (idx // (N // 8)) * 8
    nt = max(1, os.cpu_count() or 1)
    parts = np.array_split(np.arange(len(idx)), 8 * nt)

    def one(sl):
        return sl, orc.search_ranges(img, op, xs[sl], ys[sl], np.full(len(sl), 8))

    out = {k: np.zeros(len(idx), dtype=np.int64) for k in ("k", "q", "dx", "dy", "iso")}
    with ThreadPoolExecutor(max_workers=nt) as ex:
        for sl, w in ex.map(one, [q for q in parts if len(q)]):
            for k in out:
                out[k][sl] = w[k]
    return xs, ys, out


def _leaves(orc, xs, ys, w):
    """Oracle leaves of a flat 8x8 partition (one level, phase 1)."""
    lv = np.zeros(len(xs), dtype=orc.LEAF_DTYPE)
    lv["x"], lv["y"], lv["level"], lv["phase"] = xs, ys, 1, 1
    for k in ("k", "q", "dx", "dy", "iso"):
        lv[k] = w[k]
    return lv


def test_exhaustive_512_every_range_and_decode_vs_oracle(fic, orc):
    """512x512 scene, 8 isometries, domain step 4: every one of the 4096
    records of the tensor-core engine equals the oracle's search, the
    CUDA-core engine's stream is identical, and the 6-iteration decode of the
    stream equals the oracle's decode of its own leaves."""
    N = 512
    img = synth.gaussian_scene(N, 1)
    st, a = _encode(fic, img, "tensor")
    _, b = _encode(fic, img, "cuda")
    assert np.array_equal(a["records"].view(np.uint8), b["records"].view(np.uint8))
    assert a["fits"] == b["fits"] == (N // 8) ** 2 * ((N - 16) // 4 + 1) ** 2 * 8
    op = orc.make_params("exhaustive", 8, 8, 8.0)
    idx = np.arange((N // 8) ** 2)
    xs, ys, w = _search_threaded(orc, img, op, idx, N)
    want = _leaves(orc, xs, ys, w)
    gb, wb = a["records"].view(np.uint8).reshape(-1, 16), want.view(np.uint8).reshape(-1, 16)
    assert gb.shape == wb.shape
    bad = np.nonzero(np.any(gb != wb, axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {len(idx)} records differ, first {a['records'][bad[0]]} vs {want[bad[0]]}"
    assert np.array_equal(a["split"], np.zeros((N // 8) ** 2, dtype=np.uint32))
    dec = fic.fic_decode(st, 6).cpu().numpy()
    assert np.array_equal(dec, orc.decode(want, N, N, op, 6))


def test_exhaustive_1024_rows_and_random_ranges_vs_oracle(fic, orc):
    """1024x1024 scene: 1024 of the 16384 ranges against the oracle -- four
    whole range rows (top, bottom and two inner) and 512 random ranges --
    both engines identical everywhere, and the 6-iteration decode of the GPU
    stream equals the oracle's decode of the same records."""
    N = 1024
    img = synth.gaussian_scene(N, 9)
    st, a = _encode(fic, img, "tensor")
    _, b = _encode(fic, img, "cuda")
    assert np.array_equal(a["records"].view(np.uint8), b["records"].view(np.uint8))
    assert a["fits"] == b["fits"] == (N // 8) ** 2 * ((N - 16) // 4 + 1) ** 2 * 8
    per = N // 8
    rows = np.concatenate([np.arange(r * per, (r + 1) * per) for r in (0, 41, 86, per - 1)])
    rng = np.random.default_rng(N)
    rest = np.setdiff1d(np.arange(per * per), rows)
    idx = np.sort(np.concatenate([rows, rng.choice(rest, size=512, replace=False)]))
    op = orc.make_params("exhaustive", 8, 8, 8.0)
    xs, ys, w = _search_threaded(orc, img, op, idx, N)
    want = _leaves(orc, xs, ys, w)
    got = a["records"][idx]
    gb, wb = got.view(np.uint8).reshape(-1, 16), want.view(np.uint8).reshape(-1, 16)
    bad = np.nonzero(np.any(gb != wb, axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {len(idx)} records differ, first {got[bad[0]]} vs {want[bad[0]]}"
    dec = fic.fic_decode(st, 6).cpu().numpy()
    assert np.array_equal(dec, orc.decode(a["records"], N, N, op, 6))
