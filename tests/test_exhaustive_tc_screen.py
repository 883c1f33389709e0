"""The tensor-core exhaustive search's screen never drops a candidate that could win.

The tensor path contracts mean-removed range rows a_k = r_k - Sr / 64 with each
domain's screen operand w_k = (64 d4_k - Sd) 1024 / sqrt(nCdd), both rounded to
fp16, in fp32 accumulators.  Exactly, sum_k a_k w_k = 1024 nCdr / sqrt(nCdd),
whose magnitude is 2 sqrt(L) with L = 512^2 nCdr^2 / nCdd (the largest gain any
real contrast could give, Section 1's collage error with the luminance term
split off).  The kernel's per-row bound on the error of the computed value Y is
E_row = 1.1 sqrt(nCrr) + 4 (nCrr = 64 Srr - Sr^2), independent of the domain;
its screen passes a candidate when |Y| >= 2 thr(g) - E_row, thr(g) the float
lower bound of sqrt(-g) that the CUDA-core screen also uses.

These tests rebuild the operands as the prep kernels do (float32 arithmetic,
then round-to-nearest fp16), take the exact sum of their products and the
accumulation allowance the bound assumes (256 units of 2^-23 of sum |a_k w_k|),
and check that the result always lies within E_row of 2 sqrt(L), on blocks
built to stress it: the largest sums, near-flat ranges and domains, perfectly
(anti)correlated pairs.  Two concrete fp32 summation orders are checked too.
A failure means the tensor path's screen could change the search's result."""
from fractions import Fraction
import math

import numpy as np

F32 = np.float32
F16 = np.float16


def screen_operands(d, r):
    """fp16 operands of one (range row, domain) pair, as the prep kernels form them."""
    d = np.asarray(d, dtype=np.int64)
    r = np.asarray(r, dtype=np.int64)
    sd, sr = int(d.sum()), int(r.sum())
    ncdd = 64 * int((d * d).sum()) - sd * sd
    s = F32(1024.0) / np.sqrt(F32(ncdd)) if ncdd > 0 else F32(0.0)
    w = (np.asarray(64 * d - sd, dtype=F32) * s).astype(F16)
    mean = F32(sr) * F32(0.015625)
    a = (np.asarray(r, dtype=F32) - mean).astype(F16)
    return a, w


def row_bound(r) -> float:
    r = [int(x) for x in r]
    sr, srr = sum(r), sum(x * x for x in r)
    ncrr = 64 * srr - sr * sr
    return float(F32(F32(1.1) * np.sqrt(F32(ncrr)) + F32(4.0)))


def exact_y(d, r) -> float:
    """1024 nCdr / sqrt(nCdd) (0 for a flat domain)."""
    d = [int(x) for x in d]
    r = [int(x) for x in r]
    sd, sr = sum(d), sum(r)
    ncdd = 64 * sum(x * x for x in d) - sd * sd
    ncdr = 64 * sum(x * y for x, y in zip(d, r)) - sd * sr
    return 1024.0 * ncdr / math.sqrt(ncdd) if ncdd > 0 else 0.0


def exact_dot(a, w) -> Fraction:
    return sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, w)), Fraction(0))


def tc_threshold(g: int, er: float) -> np.float32:
    t = F32(F32(-g) * (F32(1.0) - F32(1e-5))) - F32(1.0)
    if t <= 0:
        return F32(-1.0)
    thr = F32(np.sqrt(t) * (F32(1.0) - F32(1e-6)))
    return F32(F32(F32(2.0) * thr - F32(er)) * (F32(1.0) - F32(1e-6))) - F32(1.0)


def cases(rng):
    """(d, r) pairs: d are 2x2 sums (0..1020), r pixels (0..255), 64 each."""
    for _ in range(300):
        yield rng.integers(0, 1021, 64), rng.integers(0, 256, 64)
    for _ in range(100):  # extremes: binary blocks at the range ends
        yield rng.choice([0, 1020], 64), rng.choice([0, 255], 64)
    for _ in range(100):  # near-flat domains: one or two elements differ
        d = np.full(64, rng.integers(0, 1021))
        i = rng.integers(0, 64, rng.integers(1, 3))
        d[i] = np.clip(d[i] + rng.choice([-1, 1], len(i)), 0, 1020)
        yield d, rng.integers(0, 256, 64)
    for _ in range(100):  # near-flat ranges (small nCrr, tight bound)
        r = np.full(64, rng.integers(0, 256))
        i = rng.integers(0, 64, rng.integers(1, 4))
        r[i] = np.clip(r[i] + rng.choice([-1, 1], len(i)), 0, 255)
        yield rng.integers(0, 1021, 64), r
    for _ in range(100):  # r an affine image of d: |nCdr| = sqrt(nCdd nCrr), the largest |Y|
        d = rng.integers(0, 1021, 64)
        sign = rng.choice([-1, 1])
        r = np.clip(np.round(127.5 + sign * (d - 510) / 4), 0, 255).astype(int)
        yield d, r
    for _ in range(100):  # the largest sums
        yield rng.integers(1000, 1021, 64), rng.integers(250, 256, 64)


def test_operands_fit_fp16_and_the_bound_holds():
    rng = np.random.default_rng(20150113)
    worst = 0.0
    for d, r in cases(rng):
        a, w = screen_operands(d, r)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(w))
        assert np.abs(w.astype(np.float64)).max() <= 8192.0 * (1 + 2.0 ** -10)
        y = exact_y(d, r)
        dot = exact_dot(a, w)
        allowance = 256 * 2.0 ** -23 * float(sum(abs(Fraction(float(x)) * Fraction(float(v))) for x, v in zip(a, w)))
        er = row_bound(r)
        err = abs(float(dot) - y) + allowance
        assert err <= er, (err, er, y)
        worst = max(worst, err / er)
        # two concrete fp32 summation orders stay inside the bound as well
        p = a.astype(F32) * w.astype(F32)  # exact: 11-bit x 11-bit significands
        seq = F32(0.0)
        for x in p:
            seq = F32(seq + x)
        pair = p.reshape(4, 16).sum(axis=1, dtype=F32).sum(dtype=F32)
        for v in (seq, pair):
            assert abs(float(v) - y) <= er
    assert worst > 0.05  # the cases reach a sizeable share of the bound


def test_screen_passes_every_candidate_that_can_win():
    rng = np.random.default_rng(1502)
    checked = 0
    for d, r in cases(rng):
        a, w = screen_operands(d, r)
        d64 = [int(x) for x in d]
        sd = sum(d64)
        ncdd = 64 * sum(x * x for x in d64) - sd * sd
        y = exact_y(d, r)
        er = row_bound(r)
        # the smallest |Y| the accumulators could hold
        dot = float(exact_dot(a, w))
        allowance = 256 * 2.0 ** -23 * float(sum(abs(Fraction(float(x)) * Fraction(float(v))) for x, v in zip(a, w)))
        y_low = max(0.0, abs(dot) - allowance)
        if ncdd <= 0:
            # a flat domain scores 0 at every contrast: it can only tie or beat g >= 0
            assert y_low >= tc_threshold(0, er)
            continue
        L = Fraction(round(y * y * 2 ** 20), 2 ** 22)  # (y / 2)^2, to well below one unit
        tight = -math.floor(L) + 1  # the most negative g this candidate can still match, with a unit to spare
        for g in {tight, tight + 1, tight // 2, -1, 0, 5}:
            if Fraction(-g) <= L:
                assert y_low >= tc_threshold(g, er), (g, y_low, er)
                checked += 1
    assert checked > 2000


def test_screen_rejects_clear_losers():
    """The bound is tight enough to matter: candidates far worse than the row's best fail."""
    rng = np.random.default_rng(8)
    rejected = total = 0
    for _ in range(300):
        d, r = rng.integers(0, 1021, 64), rng.integers(0, 256, 64)
        a, w = screen_operands(d, r)
        y = exact_y(d, r)
        if y == 0.0:
            continue
        dot = float(exact_dot(a, w))
        er = row_bound(r)
        # a best needing 25 % more gain than this candidate has even with the whole error allowance
        g = -int(((abs(y) + er) / 2) ** 2 * 1.25) - 1000
        total += 1
        rejected += bool(abs(dot) < tc_threshold(g, er))
    assert total > 250 and rejected == total


def tile_order(ntiles: int):
    """The CTA's tile visiting order: i * step mod ntiles, step near ntiles / phi and coprime with it."""
    step = max(1, int(F32(0.618034) * F32(ntiles)))
    while math.gcd(step, ntiles) != 1:
        step += 1
    out, t = [], 0
    for _ in range(ntiles):
        out.append(t)
        t = t + step - ntiles if t + step >= ntiles else t + step
    return step, out


def test_tile_order_visits_every_tile_once():
    for n in range(1, 700):
        step, order = tile_order(n)
        assert 1 <= step <= max(1, n - 1)
        assert sorted(order) == list(range(n))
