"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test states the passage of the paper (or the mathematical fact) that
fixes the expected value.  The helpers here recompute quantities directly from
pixel values with exact rational arithmetic; they never reuse the oracle's
moment formula, so a dropped term, a wrong sign or a transposed index in the
oracle makes one of them fail.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------------------
# Definitions restated directly (not through the oracle)

def s_values(s_bits):
    """Contrast codebook: midpoints of 2^b uniform cells covering [-1, 1)."""
    K = 2 ** s_bits
    return [F(-1) + F(2 * k + 1, K) for k in range(K)]


def round_half_up(f):
    return math.floor(f + F(1, 2))


def lum_values(o_bits):
    """Luminance codebook: 2^b levels spread evenly over 0..255, rounded."""
    Ko = 2 ** o_bits
    return [round_half_up(F(255 * q, Ko - 1)) for q in range(Ko)]


def decimate(img, dx, dy, B):
    """Mean of each 2x2 group of the 2B x 2B domain (Section 3), as Fractions."""
    blk = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64)
    s = blk[0::2, 0::2] + blk[1::2, 0::2] + blk[0::2, 1::2] + blk[1::2, 1::2]
    return [[F(int(s[v, u]), 4) for u in range(B)] for v in range(B)]


ISO_NUMPY = {
    0: lambda D: D,
    1: lambda D: np.rot90(D, -1),        # clockwise quarter turn
    2: lambda D: np.rot90(D, 2),
    3: lambda D: np.rot90(D, 1),
    4: lambda D: np.fliplr(D),
    5: lambda D: np.flipud(D),
    6: lambda D: D.T,
    7: lambda D: np.rot90(D, 2).T,
}


def direct_sse(r, d, s, O):
    """SSE of rhat = O + s (d - mean d) against r, exact (Fractions)."""
    n = len(r)
    dbar = sum(d) / n
    return sum((F(int(ri)) - (O + s * (di - dbar))) ** 2 for ri, di in zip(r, d))


def block_pairs(img, x, y, B, dx, dy, iso=0):
    D = np.array(decimate(img, dx, dy, B), dtype=object)
    D = ISO_NUMPY[iso](D)
    r = [int(v) for v in img[y:y + B, x:x + B].reshape(-1)]
    d = list(np.asarray(D).reshape(-1))
    return r, d


def brute_best(r, d, s_bits, o_bits):
    """Argmin of the SSE over every (s, O) code pair; ties: smaller |s|,
    then s > 0, then smaller luminance code."""
    best = None
    for k, s in enumerate(s_values(s_bits)):
        for q, O in enumerate(lum_values(o_bits)):
            e = direct_sse(r, d, s, O)
            key = (e, abs(s), 0 if s > 0 else 1, q)
            if best is None or key < best[0]:
                best = (key, k, q, e)
    return best[1], best[2], best[3]


def scaled_sse_int(img, x, y, B, dx, dy, c, O, iso=0):
    """Exact SSE * (512 n)^2 as a Python int, pixel by pixel, for contrast
    s = c/128 and luminance O: 512 n (r - rhat) is an integer."""
    n = B * B
    blk = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64)
    d4 = blk[0::2, 0::2] + blk[1::2, 0::2] + blk[0::2, 1::2] + blk[1::2, 1::2]
    d4 = np.asarray(ISO_NUMPY[iso](d4))
    r = img[y:y + B, x:x + B].astype(np.int64)
    res = 512 * n * r - 512 * n * O - c * (n * d4 - int(d4.sum()))
    return sum(int(v) * int(v) for v in res.reshape(-1))


# ---------------------------------------------------------------------------
# Section 1: range and domain counts

@pytest.mark.parametrize("N,n", [(256, 8), (64, 4), (96, 16), (512, 32), (40, 4)])
def test_counts_match_section1(orc, N, n):
    ranges = sum(1 for y in range(0, N - n + 1, n) for x in range(0, N - n + 1, n))
    domains = sum(1 for y in range(N) for x in range(N) if x + 2 * n <= N and y + 2 * n <= N)
    assert orc.count_ranges(N, N, n) == ranges == (N // n) ** 2
    assert orc.count_domains(N, N, n, 1) == domains == (N - 2 * n + 1) ** 2
    if (N, n) == (256, 8):
        assert (ranges, domains) == (1024, 58081)


def test_codebooks(orc):
    for b in (3, 5, 7):
        for k, s in enumerate(s_values(b)):
            assert F(orc.contrast(k, b), 128) == s
            assert abs(s) < 1            # contractive
    assert max(abs(orc.contrast(k, 5)) for k in range(32)) == 124   # |s| <= 31/32
    for b in (5, 7, 8):
        assert [orc.luminance(q, b) for q in range(2 ** b)] == lum_values(b)
    # Section 3.2 sets, rounded to the 1/128 grid
    want = {1: (F(2, 10), F(5, 10)), 2: (F(4, 10), F(65, 100)), 3: (F(5, 10), F(9, 10))}
    for lvl, (a, b) in want.items():
        assert orc.phase2_contrast(lvl, 0) == round_half_up(a * 128)
        assert orc.phase2_contrast(lvl, 1) == round_half_up(b * 128)


def test_isometries_match_numpy(orc):
    rng = np.random.default_rng(3)
    for B in (2, 4, 8):
        D = rng.integers(0, 1000, size=(B, B))
        for iso in range(8):
            T = np.empty_like(D)
            for v in range(B):
                for u in range(B):
                    su, sv = orc.iso_source(iso, B, u, v)
                    T[v, u] = D[sv, su]
            assert np.array_equal(T, ISO_NUMPY[iso](D)), (B, iso)


# ---------------------------------------------------------------------------
# Closed form of the code choice == brute force over the whole codebook

def _tiny_cases():
    rng = np.random.default_rng(11)
    cases = []
    for trial in range(14):
        img = rng.integers(0, 256, size=(8, 8), dtype=np.uint8)
        if trial == 0:
            img[:] = 77                       # flat range and domain
        if trial == 1:
            img[:, :] = rng.integers(0, 256, size=(8, 8))
            img[4:8, 0:4] = 200               # flat domain only
        if trial == 2:
            img = (np.arange(64).reshape(8, 8) * 4).astype(np.uint8)   # ramp
        if trial == 3:
            img = np.where(rng.uniform(size=(8, 8)) < 0.5, 0, 255).astype(np.uint8)
        cases.append((img, 0, 0, 2, 4, 4, trial % 8))
    return cases


@pytest.mark.parametrize("case", range(14))
def test_best_codes_equal_brute_force_B2(orc, case):
    img, x, y, B, dx, dy, iso = _tiny_cases()[case]
    r, d = block_pairs(img, x, y, B, dx, dy, iso)
    k, q, sse = brute_best(r, d, 5, 7)
    mom, ko, qo, eo = orc.fit_pair(img, x, y, B, dx, dy, iso, 5, 7)
    assert (ko, qo) == (k, q)
    assert eo == sse * B * B * 512 ** 2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_best_codes_equal_brute_force_B4(orc, seed):
    rng = np.random.default_rng(100 + seed)
    img = rng.integers(0, 256, size=(16, 16), dtype=np.uint8)
    if seed == 2:
        img = np.clip(rng.normal(120, 20, size=(16, 16)), 0, 255).astype(np.uint8)
    x, y, dx, dy = 12, 4, 0, 8
    iso = [0, 1, 6][seed]
    r, d = block_pairs(img, x, y, 4, dx, dy, iso)
    for sb, ob in ((5, 7), (3, 8)):
        k, q, sse = brute_best(r, d, sb, ob)
        _, ko, qo, eo = orc.fit_pair(img, x, y, 4, dx, dy, iso, sb, ob)
        assert (ko, qo) == (k, q), (sb, ob)
        assert eo == sse * 16 * 512 ** 2


def test_flat_domain_picks_smallest_positive_contrast(orc):
    img = np.full((16, 16), 90, dtype=np.uint8)
    img[0:4, 0:4] = np.arange(16).reshape(4, 4) * 9
    _, k, q, _ = orc.fit_pair(img, 0, 0, 4, 8, 8, 0, 5, 7)
    assert orc.contrast(k, 5) == 4          # s = +1/32


def test_error_formula_against_pixels_large_blocks(orc):
    img = synth.gaussian_scene(128, 5)
    for (x, y, B) in [(32, 32, 32), (64, 16, 16), (8, 96, 8)]:
        dx, dy = orc.centred(x, B, 128), orc.centred(y, B, 128)
        _, k, q, e = orc.fit_pair(img, x, y, B, dx, dy, 0, 5, 7)
        n = B * B
        direct = scaled_sse_int(img, x, y, B, dx, dy, orc.contrast(k, 5), orc.luminance(q, 7))
        # E = n 512^2 SSE, direct = (512 n)^2 SSE
        assert direct == e * n


# ---------------------------------------------------------------------------
# Constant images: zero error, accepted at the first level, decoded exactly

@pytest.mark.parametrize("value", [0, 2, 129, 255, 253])
def test_constant_on_grid(orc, value):
    grid = lum_values(7)
    assert value in grid
    img = synth.constant(64, value)
    p = orc.make_params("mns", 32, 4, 8.0)
    leaves, split, _ = orc.encode(img, p)
    assert len(leaves) == 4 and np.all(leaves["level"] == 1) and np.all(leaves["phase"] == 1)
    assert np.all(split == 0)
    for lf in leaves:
        _, _, _, e = orc.fit_pair(img, int(lf["x"]), int(lf["y"]), 32, int(lf["dx"]), int(lf["dy"]))
        assert e == 0
    dec = orc.decode(leaves, 64, 64, p, 10)
    assert np.array_equal(dec, img)


@pytest.mark.parametrize("value", [1, 100, 128, 201])
def test_constant_off_grid_half_step(orc, value):
    img = synth.constant(64, value)
    p = orc.make_params("mns", 32, 4, 8.0)
    leaves, _, _ = orc.encode(img, p)
    dec = orc.decode(leaves, 64, 64, p, 10)
    assert np.all(leaves["level"] == 1)
    assert np.max(np.abs(dec.astype(int) - value)) <= F(255, 127) / 2


# ---------------------------------------------------------------------------
# Quadtree decisions re-derived from pixels (Section 3 and 3.1 - 3.3)

def _mean_delta(img, x, y, h, Oi):
    blk = img[y:y + h, x:x + h].astype(np.int64)
    return round_half_up(F(int(blk.sum()), h * h) - Oi)


def _sub_domain(orc, p, x, y, B, sb, W, H):
    """Phase-2 domain of sub-block sb: its own centred B x B domain, or (the
    alternative reading) quadrant sb of the parent's centred 2B x 2B domain."""
    h = B // 2
    if p.phase2_domain:
        return orc.centred(x, B, W) + (sb & 1) * B, orc.centred(y, B, H) + (sb >> 1) * B
    return orc.centred(x + (sb & 1) * h, h, W), orc.centred(y + (sb >> 1) * h, h, H)


def _check_encoding(orc, img, p):
    H, W = img.shape
    leaves, split, _ = orc.encode(img, p)
    L = orc.nlevels(p)
    thr = p.thr_rms[0]
    T2 = F(round(thr * thr * 256), 256)
    covered = np.zeros((H, W), dtype=np.int32)
    keys = []
    tw = W // p.bmax
    for lf in leaves:
        x, y, lvl = int(lf["x"]), int(lf["y"]), int(lf["level"])
        B = p.bmax >> (lvl - 1)
        n = B * B
        covered[y:y + B, x:x + B] += 1
        top = (y // p.bmax) * tw + (x // p.bmax)
        zx, zy = (x % p.bmax) // p.bmin, (y % p.bmax) // p.bmin
        z = sum((((zx >> b) & 1) << (2 * b)) | (((zy >> b) & 1) << (2 * b + 1)) for b in range(8))
        keys.append((top, z))
        dx, dy = orc.centred(x, B, W), orc.centred(y, B, H)
        assert (int(lf["dx"]), int(lf["dy"])) == (dx, dy)
        if lf["phase"] == 1:
            _, k, q, _ = orc.fit_pair(img, x, y, B, dx, dy, 0, p.s_bits, p.o_bits)
            assert (int(lf["k"]), int(lf["q"])) == (k, q)
            if lvl < L:
                sse = scaled_sse_int(img, x, y, B, dx, dy, orc.contrast(k, p.s_bits),
                                     orc.luminance(q, p.o_bits))
                assert sse < T2 * n * (512 * n) ** 2
        else:
            assert p.mode == 1 and lvl < L
            _, _, qi, _ = orc.fit_pair(img, x, y, B, dx, dy, 0, p.s_bits, p.o_bits)
            assert int(lf["q"]) == qi
            Oi = orc.luminance(qi, p.o_bits)
            h = B // 2
            dmax = 2 ** ((5 if lvl == 1 else 6) - 1) - 1
            deltas = [_mean_delta(img, x + (sb & 1) * h, y + (sb >> 1) * h, h, Oi) for sb in range(4)]
            assert all(abs(dl) <= dmax for dl in deltas)
            assert [int(v) for v in lf["d"]] == deltas[:3]
            Os = [Oi + deltas[0], Oi + deltas[1], Oi + deltas[2]]
            Os.append(4 * Oi - sum(Os))                        # eq. (1)
            assert F(sum(Os), 4) == Oi
            for sb in range(4):
                sx, sy = x + (sb & 1) * h, y + (sb >> 1) * h
                sdx, sdy = _sub_domain(orc, p, x, y, B, sb, W, H)
                e = [scaled_sse_int(img, sx, sy, h, sdx, sdy, orc.phase2_contrast(lvl, b), Os[sb])
                     for b in (0, 1)]
                bit = (int(lf["k"]) >> sb) & 1
                assert e[bit] <= e[1 - bit] and (bit == 0 or e[1] < e[0])
                assert e[bit] < T2 * h * h * (512 * h * h) ** 2
    assert np.all(covered == 1)                                 # leaves tile the image once
    assert keys == sorted(keys)                                 # canonical order
    # split nodes: phase 1 (and phase 2 where allowed) must really fail
    for t, mask in enumerate(split):
        X, Y = (t % tw) * p.bmax, (t // tw) * p.bmax
        for lvl in range(1, L):
            B = p.bmax >> (lvl - 1)
            per = p.bmax // B
            off = (4 ** (lvl - 1) - 1) // 3
            for z in range(per * per):
                if not (int(mask) >> (off + z)) & 1:
                    continue
                bx = sum(((z >> (2 * b)) & 1) << b for b in range(4))
                by = sum(((z >> (2 * b + 1)) & 1) << b for b in range(4))
                x, y, n = X + bx * B, Y + by * B, B * B
                dx, dy = orc.centred(x, B, W), orc.centred(y, B, H)
                _, k, q, _ = orc.fit_pair(img, x, y, B, dx, dy, 0, p.s_bits, p.o_bits)
                sse = scaled_sse_int(img, x, y, B, dx, dy, orc.contrast(k, p.s_bits),
                                     orc.luminance(q, p.o_bits))
                assert sse >= T2 * n * (512 * n) ** 2
                if p.mode == 1 and p.phase2:
                    Oi = orc.luminance(q, p.o_bits)
                    h = B // 2
                    dmax = 2 ** ((5 if lvl == 1 else 6) - 1) - 1
                    deltas = [_mean_delta(img, x + (sb & 1) * h, y + (sb >> 1) * h, h, Oi)
                              for sb in range(4)]
                    if all(abs(dl) <= dmax for dl in deltas):
                        Os = [Oi + deltas[0], Oi + deltas[1], Oi + deltas[2]]
                        Os.append(4 * Oi - sum(Os))
                        worst_ok = True
                        for sb in range(4):
                            sx, sy = x + (sb & 1) * h, y + (sb >> 1) * h
                            sdx, sdy = _sub_domain(orc, p, x, y, B, sb, W, H)
                            e = min(scaled_sse_int(img, sx, sy, h, sdx, sdy,
                                                   orc.phase2_contrast(lvl, b), Os[sb]) for b in (0, 1))
                            worst_ok &= e < T2 * h * h * (512 * h * h) ** 2
                        assert not worst_ok
                # the children of a split node are present (split or leaves)
    # a leaf's ancestors are all split, the leaf itself is not
    for lf in leaves:
        x, y, lvl = int(lf["x"]), int(lf["y"]), int(lf["level"])
        t = (y // p.bmax) * tw + (x // p.bmax)
        for a in range(1, L):
            B = p.bmax >> (a - 1)
            bx, by = (x % p.bmax) // B, (y % p.bmax) // B
            z = sum((((bx >> b) & 1) << (2 * b)) | (((by >> b) & 1) << (2 * b + 1)) for b in range(4))
            bit = (int(split[t]) >> ((4 ** (a - 1) - 1) // 3 + z)) & 1
            assert bit == (1 if a < lvl else 0)
    return leaves


@pytest.mark.parametrize("thr", [8.0, 4.0])
@pytest.mark.parametrize("p2d", [0, 1])
def test_decisions_rederived_scene256(orc, thr, p2d):
    img = synth.scene256_image()
    p = orc.make_params("mns", 16, 4, thr, phase2_domain=p2d)
    leaves = _check_encoding(orc, img, p)
    assert (leaves["phase"] == 2).any() or thr == 4.0


def test_decisions_rederived_512_levels4(orc):
    img = synth.gaussian_scene(512, 2)[128:384, 128:384].copy()
    p = orc.make_params("mns", 32, 4, 6.0)
    leaves = _check_encoding(orc, img, p)
    assert set(np.unique(leaves["level"])) == {1, 2, 3, 4}
    assert (leaves["phase"] == 2).any()


def test_decisions_rederived_voronoi(orc):
    img = synth.voronoi(128, 101)
    p = orc.make_params("mns", 32, 4, 8.0)
    _check_encoding(orc, img, p)


def test_nosearch_equals_mns_without_phase2(orc):
    img = synth.gaussian_scene(256, 3)
    a = orc.encode(img, orc.make_params("nosearch", 32, 4, 8.0))
    b = orc.encode(img, orc.make_params("mns", 32, 4, 8.0, phase2=False))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------------------
# Local and exhaustive search

def test_local_candidates_81(orc):
    img = synth.gaussian_scene(256, 4)
    p = orc.make_params("local", 8, 8, 8.0)
    assert orc.count_candidates(img, p, 128, 128, 8) == 81       # Section 2
    for (x, y) in [(0, 0), (248, 8), (16, 240)]:
        cx, cy = orc.centred(x, 8, 256), orc.centred(y, 8, 256)
        want = sum(1 for oy in range(-16, 17, 4) for ox in range(-16, 17, 4)
                   if 0 <= cx + ox <= 256 - 16 and 0 <= cy + oy <= 256 - 16)
        assert orc.count_candidates(img, p, x, y, 8) == want


def _plant(img, x, y, B, dx, dy, iso, s, O):
    """Overwrite range (x, y) with round(O + s (d - dbar)) of domain (dx, dy)."""
    D = np.array(decimate(img, dx, dy, B), dtype=object)
    D = ISO_NUMPY[iso](D)
    dbar = sum(D.reshape(-1)) / (B * B)
    for v in range(B):
        for u in range(B):
            img[y + v, x + u] = min(255, max(0, round_half_up(O + s * (D[v, u] - dbar))))


def test_exhaustive_finds_planted_isometry(orc):
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(64, 64), dtype=np.uint8)
    # smooth random field so that decimation keeps structure
    img = np.clip(synth.gaussian_scene(64, 8).astype(int) + rng.integers(-40, 40, (64, 64)), 0, 255).astype(np.uint8)
    p = orc.make_params("exhaustive", 8, 8, 8.0, dom_step=4, isometries=8)
    for (x, y, dx, dy, iso) in [(48, 48, 8, 12, 3), (0, 56, 40, 0, 6), (32, 0, 0, 36, 1)]:
        _plant(img, x, y, 8, dx, dy, iso, F(3, 4) - F(1, 32), 120)
        res = orc.search_ranges(img, p, [x], [y], [8])
        assert (res["dx"][0], res["dy"][0], res["iso"][0]) == (dx, dy, iso)
        assert res["e"][0] <= 64 * 512 ** 2 * 64 // 4          # rounding only: SSE <= n/4


def _brute_search(img, x, y, B, cands):
    """Phase-1 search of range (x, y) over the candidates (dx, dy, iso), in
    the order given, by definition: every (s, O) code pair of each candidate,
    the error summed pixel by pixel (512 n (r - rhat) is an integer).
    Returns (scaled SSE, dx, dy, iso, k, q) of the winner; a later candidate
    wins only if strictly better; codes tied on the error go to the smaller
    |s|, then s > 0, then the smaller luminance code."""
    n = B * B
    cs = np.array([int(s * 128) for s in s_values(5)], dtype=np.int64)
    Os = np.array(lum_values(7), dtype=np.int64)
    r = img[y:y + B, x:x + B].astype(np.int64).reshape(-1)
    best = None
    for dx, dy, iso in cands:
        blk = img[dy:dy + 2 * B, dx:dx + 2 * B].astype(np.int64)
        d4 = blk[0::2, 0::2] + blk[1::2, 0::2] + blk[0::2, 1::2] + blk[1::2, 1::2]
        d = np.asarray(ISO_NUMPY[iso](d4)).reshape(-1)
        res = (512 * n * r)[None, None, :] - (512 * n * Os)[None, :, None] \
            - cs[:, None, None] * (n * d - int(d.sum()))[None, None, :]
        sse = (res * res).sum(-1)  # [contrast code, luminance code]
        m = int(sse.min())
        if best is None or m < best[0]:
            ks, qs = np.nonzero(sse == m)
            k, q = min(zip(ks, qs), key=lambda kq: (abs(cs[kq[0]]), cs[kq[0]] < 0, kq[1]))
            best = (m, dx, dy, iso, int(k), int(q))
    return best


def _brute_exhaustive(img, x, y, B=8, step=4):
    """Section 1's exhaustive search: every 2B x 2B domain of the step grid
    in raster order, each under the eight isometries in order."""
    H, W = img.shape
    cands = [(dx, dy, iso) for dy in range(0, H - 2 * B + 1, step) for dx in range(0, W - 2 * B + 1, step)
             for iso in range(8)]
    return _brute_search(img, x, y, B, cands)


def test_exhaustive_search_equals_brute_force(orc):
    # a smooth field with noise, and one range planted from a rotated domain
    rng = np.random.default_rng(21)
    img = np.clip(synth.gaussian_scene(32, 4).astype(int) + rng.integers(-25, 25, (32, 32)), 0, 255).astype(np.uint8)
    _plant(img, 16, 8, 8, 4, 16, 5, F(1, 2) + F(1, 32), 140)
    p = orc.make_params("exhaustive", 8, 8, 8.0, dom_step=4, isometries=8)
    xs, ys = [0, 24, 16, 8, 24, 0], [0, 0, 8, 16, 24, 24]
    res = orc.search_ranges(img, p, xs, ys, [8] * len(xs))
    for i, (x, y) in enumerate(zip(xs, ys)):
        sse, dx, dy, iso, k, q = _brute_exhaustive(img, x, y)
        got = (int(res["dx"][i]), int(res["dy"][i]), int(res["iso"][i]), int(res["k"][i]), int(res["q"][i]))
        assert got == (dx, dy, iso, k, q), (x, y)
        assert sse == int(res["e"][i]) * 64  # E = n 512^2 SSE, the scaled sum = (512 n)^2 SSE


def test_local_search_equals_brute_force(orc):
    """Section 2's local search: the domains whose offsets from the centred
    one (x - B/2 clamped into the image) are multiples of 4 within +-16 in x
    and y, offsets in raster order, those that leave the image skipped, no
    isometries; ranges at the border lose candidates."""
    img = np.clip(synth.gaussian_scene(64, 6).astype(int) + np.random.default_rng(8).integers(-30, 30, (64, 64)),
                  0, 255).astype(np.uint8)
    p = orc.make_params("local", 8, 8, 8.0)
    xs, ys = [0, 56, 24, 32, 8], [0, 8, 24, 56, 40]
    res = orc.search_ranges(img, p, xs, ys, [8] * len(xs))
    for i, (x, y) in enumerate(zip(xs, ys)):
        cx, cy = min(max(x - 4, 0), 64 - 16), min(max(y - 4, 0), 64 - 16)
        cands = [(cx + ox, cy + oy, 0) for oy in range(-16, 17, 4) for ox in range(-16, 17, 4)
                 if 0 <= cx + ox <= 64 - 16 and 0 <= cy + oy <= 64 - 16]
        sse, dx, dy, iso, k, q = _brute_search(img, x, y, 8, cands)
        got = (int(res["dx"][i]), int(res["dy"][i]), int(res["iso"][i]), int(res["k"][i]), int(res["q"][i]))
        assert got == (dx, dy, iso, k, q), (x, y)
        assert sse == int(res["e"][i]) * 64


def test_local_finds_planted_offset(orc):
    img = synth.gaussian_scene(128, 12)
    rng = np.random.default_rng(5)
    img = np.clip(img.astype(int) + rng.integers(-30, 30, img.shape), 0, 255).astype(np.uint8)
    p = orc.make_params("local", 8, 8, 8.0)
    x, y = 64, 64
    cx, cy = orc.centred(x, 8, 128), orc.centred(y, 8, 128)
    dx, dy = cx + 12, cy - 16
    _plant(img, x, y, 8, dx, dy, 0, F(5, 8) + F(1, 32) * 3, 90)
    res = orc.search_ranges(img, p, [x], [y], [8])
    assert (res["dx"][0], res["dy"][0], res["iso"][0]) == (dx, dy, 0)


# ---------------------------------------------------------------------------
# Decoder

def test_decoder_first_iterate_is_luminance(orc):
    img = synth.scene256_image()
    p = orc.make_params("mns", 16, 4, 8.0)
    leaves, _, _ = orc.encode(img, p)
    x1 = orc.decode(leaves, 256, 256, p, 1)
    for lf in leaves:
        x, y, lvl = int(lf["x"]), int(lf["y"]), int(lf["level"])
        B = 16 >> (lvl - 1)
        Oi = orc.luminance(int(lf["q"]), 7)
        if lf["phase"] == 1:
            assert np.all(x1[y:y + B, x:x + B] == Oi)
        else:
            h = B // 2
            Os = [Oi + int(lf["d"][0]), Oi + int(lf["d"][1]), Oi + int(lf["d"][2])]
            Os.append(4 * Oi - sum(Os))
            for sb in range(4):
                sx, sy = x + (sb & 1) * h, y + (sb >> 1) * h
                assert np.all(x1[sy:sy + h, sx:sx + h] == min(255, max(0, Os[sb])))


@pytest.mark.parametrize("p2d", [0, 1])
def test_decoder_second_iterate_direct(orc, p2d):
    img = synth.scene256_image()
    p = orc.make_params("mns", 16, 4, 8.0, phase2_domain=p2d)
    leaves, _, _ = orc.encode(img, p)
    x1 = orc.decode(leaves, 256, 256, p, 1)
    x2 = orc.decode(leaves, 256, 256, p, 2)
    for lf in leaves[::7]:
        x, y, lvl = int(lf["x"]), int(lf["y"]), int(lf["level"])
        B = 16 >> (lvl - 1)
        Oi = orc.luminance(int(lf["q"]), 7)
        if lf["phase"] == 1:
            parts = [(x, y, B, F(orc.contrast(int(lf["k"]), 5), 128), Oi)]
        else:
            h = B // 2
            Os = [Oi + int(lf["d"][0]), Oi + int(lf["d"][1]), Oi + int(lf["d"][2])]
            Os.append(4 * Oi - sum(Os))
            parts = [(x + (sb & 1) * h, y + (sb >> 1) * h, h,
                      F(orc.phase2_contrast(lvl, (int(lf["k"]) >> sb) & 1), 128), Os[sb],
                      _sub_domain(orc, p, x, y, B, sb, 256, 256))
                     for sb in range(4)]
        if lf["phase"] == 1:
            parts = [parts[0] + ((orc.centred(x, B, 256), orc.centred(y, B, 256)),)]
        for (sx, sy, b, s, O, (dx, dy)) in parts:
            D = decimate(x1, dx, dy, b)
            dbar = sum(sum(row) for row in D) / (b * b)
            for v in range(b):
                for u in range(b):
                    want = min(255, max(0, round_half_up(O + s * (D[v][u] - dbar))))
                    assert x2[sy + v, sx + u] == want


def test_attractor_reencodes_to_rounding(orc):
    """Random transforms on a fixed flat partition: iterate to the fixed point
    (or to a 1-LSB limit cycle, which integer rounding can produce), then
    encode that image again: the encoder finds codes at least as good as the
    ones that generated it, i.e. each block fits within rounding (RMS ~ 0.5)."""
    rng = np.random.default_rng(21)
    W = 64
    B = 16
    p = orc.make_params("mns", B, B, 255.0)
    leaves = np.zeros((W // B) ** 2, dtype=orc.LEAF_DTYPE)
    i = 0
    for y in range(0, W, B):
        for x in range(0, W, B):
            leaves[i]["x"], leaves[i]["y"], leaves[i]["level"], leaves[i]["phase"] = x, y, 1, 1
            leaves[i]["k"] = rng.integers(10, 22)
            leaves[i]["q"] = rng.integers(40, 88)
            leaves[i]["dx"], leaves[i]["dy"] = orc.centred(x, B, W), orc.centred(y, B, W)
            i += 1
    seq = [orc.decode(leaves, W, W, p, it) for it in range(1, 65)]
    settled = None
    for it in range(2, 64):
        if np.array_equal(seq[it], seq[it - 2]):
            settled = it
            break
    assert settled is not None, "no fixed point or 2-cycle within 64 iterations"
    fixed = seq[settled]
    cyc = np.abs(seq[settled].astype(int) - seq[settled - 1].astype(int))
    assert cyc.max() <= 1
    assert fixed.min() > 0 and fixed.max() < 255            # no clipping involved
    re, _, _ = orc.encode(fixed, p)
    assert len(re) == len(leaves)
    n = B * B
    slack = F(n, 4) + 2 * int((cyc > 0).sum())               # cycling pixels: |err| <= 1.5
    for orig, got in zip(leaves, re):
        x, y = int(orig["x"]), int(orig["y"])
        dx, dy = orc.centred(x, B, W), orc.centred(y, B, W)
        e_orig = scaled_sse_int(fixed, x, y, B, dx, dy, orc.contrast(int(orig["k"]), 5),
                                orc.luminance(int(orig["q"]), 7))
        e_got = scaled_sse_int(fixed, x, y, B, dx, dy, orc.contrast(int(got["k"]), 5),
                               orc.luminance(int(got["q"]), 7))
        assert e_got <= e_orig <= slack * (512 * n) ** 2


def test_decoder_converges(orc):
    """Within 64 iterations the iterates settle into a band of at most 1 LSB
    (integer rounding leaves a few pixels flickering between neighbouring
    values), and the attractor is close to the image."""
    img = synth.scene256_image()
    p = orc.make_params("mns", 16, 4, 8.0)
    leaves, _, _ = orc.encode(img, p)
    seq = [orc.decode(leaves, 256, 256, p, it) for it in range(1, 65)]
    diffs = [int(np.max(np.abs(seq[i].astype(int) - seq[i - 1].astype(int)))) for i in range(1, 64)]
    assert diffs[0] > 1                      # it does move at first
    assert max(diffs[-32:]) <= 1
    moving = int(np.sum(seq[-1] != seq[-2]))
    assert moving < 0.01 * seq[-1].size
    assert orc.psnr(img, seq[-1]) > 25.0


# ---------------------------------------------------------------------------
# Bit accounting (Sections 3.3, 3.4)

def _group_leaves(orc, groups, W):
    """`groups` sibling groups of four last-level (4x4) leaves, phase 1."""
    lv = np.zeros(4 * groups, dtype=orc.LEAF_DTYPE)
    per_row = W // 8
    for g in range(groups):
        gx, gy = (g % per_row) * 8, (g // per_row) * 8
        for c in range(4):
            r = lv[4 * g + c]
            r["x"], r["y"] = gx + (c & 1) * 4, gy + (c >> 1) * 4
            r["level"], r["phase"] = 4, 1
    return lv


def test_technique2_lena_numbers(orc):
    # Section 3.4: 4000 blocks at level 4 need 8000 level bits, 2000 with Technique 2
    W = 1024
    p = orc.make_params("mns", 32, 4, 8.0)
    lv = _group_leaves(orc, 1000, W)
    without = orc.bits(lv, W, W, p, technique2=False)
    with_t2 = orc.bits(lv, W, W, p, technique2=True)
    assert without - with_t2 == 8000 - 2000
    assert without == 4000 * (5 + 7 + 2)          # last level: no phase bit


def test_technique2_baboon_numbers(orc):
    # Section 3.4: about 25000 level-4 blocks: 6.25 kB of level bits, about 1.5 kB with Technique 2
    W = 2048
    p = orc.make_params("mns", 32, 4, 8.0)
    lv = _group_leaves(orc, 6250, W)
    without = orc.bits(lv, W, W, p, technique2=False)
    with_t2 = orc.bits(lv, W, W, p, technique2=True)
    payload = 25000 * (5 + 7)
    assert (without - payload) / 8 == 6250          # 6.25 kB
    assert 1500 <= (with_t2 - payload) / 8 < 1600   # "1.5 kbytes"


def test_fourteen_bits_per_phase1_block(orc):
    # Section 3.3: one byte luminance + three bits contrast + two level bits + one phase bit
    p = orc.make_params("mns", 16, 2, 8.0, s_bits=3, o_bits=8)
    lv = np.zeros(1, dtype=orc.LEAF_DTYPE)
    lv[0]["level"], lv[0]["phase"] = 1, 1
    assert orc.bits(lv, 64, 64, p) == 14
    lv[0]["level"], lv[0]["phase"] = 2, 2
    # phase 2: O_i (8) + three 6-bit differences + four 1-bit contrasts + level + phase
    assert orc.bits(lv, 64, 64, p) == 8 + 3 * 6 + 4 + 2 + 1


def test_psnr_definition(orc):
    a = np.zeros((4, 4), dtype=np.uint8)
    b = a.copy()
    b[0, 0] = 4                                  # MSE = 1
    assert abs(orc.psnr(a, b) - 10 * math.log10(255 ** 2)) < 1e-12


def test_bad_sizes_rejected(orc):
    p = orc.make_params("mns", 32, 4, 8.0)
    assert orc.check(512, 512, p) == 0
    assert orc.check(500, 512, p) != 0
    assert orc.check(32, 64, p) != 0
    assert orc.check(64, 64, orc.make_params("mns", 64, 2, 8.0)) != 0   # more than 4 levels


def test_phase2_domain_readings_differ(orc):
    """The two readings of the phase-2 domain give different streams (both
    re-derived above); phase 1 and the split rule are shared."""
    img = synth.scene256_image()
    a, _, _ = orc.encode(img, orc.make_params("mns", 16, 4, 8.0, phase2_domain=0))
    b, _, _ = orc.encode(img, orc.make_params("mns", 16, 4, 8.0, phase2_domain=1))
    assert (a["phase"] == 2).any() and (b["phase"] == 2).any()
    assert len(a) != len(b) or not np.array_equal(a.view(np.uint8), b.view(np.uint8))
