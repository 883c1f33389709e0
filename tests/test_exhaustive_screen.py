"""The exhaustive search's float screen never drops a candidate that could win.

For a (range row, domain) pair the exact score is g(c) = c^2 nCdd - 1024 c nCdr
at the chosen contrast code c; over real c it is at least -L with
L = 512^2 nCdr^2 / nCdd, so a candidate can beat (or tie) the row's best g only
when L >= -g.  The kernels decide "evaluate exactly" in float32:

    cs = (-Sd / 64, 64 sw, 130 sw),  sw = sqrt(262144 / nCdd)
    a  = fma(cs.x, Sr, Sdr)                  (= nCdr / 64, one rounding)
    v  = fma(|a|, cs.y, cs.z)
    thr(g) = sqrt(-g (1 - 1e-5) - 1) (1 - 1e-6), or -1 when that is not positive

and, in the CUDA-core engine's per-candidate pass, also |a| >= thra(g) = -g (1 - 1e-5) / (65536 C) - 1
(or -1 while g >= 0), C = 128 - 128 / 2^s_bits the largest contrast code: at
|c| <= C the score is at least -1024 C |nCdr|.  A candidate can reach g only if
-g <= M, M the largest value of 1024 c nCdr - c^2 nCdd over real c in [-C, C]
(M <= L).  Evaluate when both hold.  This test replays that arithmetic bit for bit
(IEEE float32 round-to-nearest for every step, fused multiply-adds rounded once
from the exact value) on blocks built to stress it -- the largest sums,
near-flat domains, perfectly (anti)correlated pairs -- with g at the tightest
value that must still pass, -floor(L).  A failure means the screen can change
the search's result."""
from fractions import Fraction
import math

import numpy as np

F32 = np.float32


def round_f32(x: Fraction) -> np.float32:
    """Nearest float32 to the exact rational x (ties to even)."""
    if x == 0:
        return F32(0.0)
    s = -1 if x < 0 else 1
    x = abs(x)
    e = math.floor(math.log2(x.numerator) - math.log2(x.denominator))
    # settle e so that 2^23 <= x / 2^(e - 23) < 2^24
    while x >= Fraction(2) ** (e + 1):
        e += 1
    while x < Fraction(2) ** e:
        e -= 1
    scale = Fraction(2) ** (e - 23)
    q = x / scale
    m = q.numerator // q.denominator
    rem = q - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return F32(s * float(m * scale))


def fma_f32(a, b, c) -> np.float32:
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def screen_value(sdr: int, sd: int, sr: int, ncdd: int, with_a=False):
    sw = np.sqrt(F32(262144.0) / F32(ncdd)) if ncdd > 0 else F32(0.0)
    cx = F32(-F32(sd)) * F32(0.015625)
    cy = F32(64.0) * sw
    cz = F32(130.0) * sw
    a = abs(fma_f32(cx, F32(sr), F32(sdr)))
    v = fma_f32(a, cy, cz)
    return (v, a) if with_a else v


def threshold_a(g: int, s_bits: int) -> np.float32:
    if g >= 0:
        return F32(-1.0)
    c = F32(128 - (128 >> s_bits))
    k = (F32(1.0) - F32(1e-5)) / (F32(65536.0) * c)
    return F32(F32(-g) * k) - F32(1.0)


def largest_gain(ncdr: int, ncdd: int, s_bits: int) -> Fraction:
    """max over real c in [-C, C] of 1024 c nCdr - c^2 nCdd."""
    C = 128 - (128 >> s_bits)
    if ncdd > 0 and abs(Fraction(512 * ncdr, ncdd)) <= C:
        return Fraction(262144 * ncdr * ncdr, ncdd)
    return Fraction(1024 * C * abs(ncdr) - C * C * ncdd)


def threshold(g: int) -> np.float32:
    t = F32(F32(-g) * (F32(1.0) - F32(1e-5))) - F32(1.0)
    return F32(np.sqrt(t) * (F32(1.0) - F32(1e-6))) if t > 0 else F32(-1.0)


def block_stats(d, r):
    d = [int(x) for x in d]
    r = [int(x) for x in r]
    sd, sr = sum(d), sum(r)
    sdr = sum(x * y for x, y in zip(d, r))
    ncdd = 64 * sum(x * x for x in d) - sd * sd
    ncdr = 64 * sdr - sd * sr
    return sdr, sd, sr, ncdd, ncdr


def cases(rng):
    """(d, r) pairs: d are 2x2 sums (0..1020), r pixels (0..255), 64 each."""
    for _ in range(300):
        yield rng.integers(0, 1021, 64), rng.integers(0, 256, 64)
    for _ in range(150):  # extremes: binary blocks at the range ends
        yield rng.choice([0, 1020], 64), rng.choice([0, 255], 64)
    for _ in range(150):  # near-flat domains: one or two elements differ
        d = np.full(64, rng.integers(0, 1021))
        i = rng.integers(0, 64, rng.integers(1, 3))
        d[i] = np.clip(d[i] + rng.choice([-1, 1], len(i)), 0, 1020)
        yield d, rng.integers(0, 256, 64)
    for _ in range(150):  # r an affine image of d: nCdr^2 = nCdd nCrr, the largest L
        d = rng.integers(0, 1021, 64)
        sign = rng.choice([-1, 1])
        r = np.clip(np.round(127.5 + sign * (d - 510) / 4), 0, 255).astype(int)
        yield d, r
    for _ in range(100):  # the largest sums: Sdr close to its 2^24 bound
        yield rng.integers(1000, 1021, 64), rng.integers(250, 256, 64)


def test_screen_passes_every_candidate_that_can_win():
    rng = np.random.default_rng(20150112)
    checked = 0
    for d, r in cases(rng):
        sdr, sd, sr, ncdd, ncdr = block_stats(d, r)
        assert sdr < 1 << 24  # the accumulator sums stay exact in float32
        v = screen_value(sdr, sd, sr, ncdd)
        if ncdd <= 0:
            # a flat domain scores 0 at every contrast: it can only tie or beat g >= 0
            assert v >= threshold(0)
            continue
        L = Fraction(262144 * ncdr * ncdr, ncdd)
        tight = -math.floor(L)  # the most negative g that this candidate can still match
        for g in {tight, tight + 1, tight // 2, -1, 0, 5}:
            if Fraction(-g) <= L:
                assert v >= threshold(g), (sdr, sd, sr, ncdd, g)
                checked += 1
    assert checked > 2000


def test_both_screens_pass_every_candidate_that_can_win():
    rng = np.random.default_rng(1501)
    checked = 0
    for s_bits in (1, 3, 5, 7):
        for d, r in cases(rng):
            sdr, sd, sr, ncdd, ncdr = block_stats(d, r)
            v, a = screen_value(sdr, sd, sr, ncdd, with_a=True)
            M = largest_gain(ncdr, ncdd, s_bits)
            tight = -math.floor(M)
            for g in {tight, tight + 1, tight // 2, -1, 0, 5}:
                if Fraction(-g) <= M:
                    assert v >= threshold(g) and a >= threshold_a(g, s_bits), (s_bits, sdr, sd, sr, ncdd, g)
                    checked += 1
    assert checked > 8000


def test_contrast_range_test_rejects_domains_needing_large_contrast():
    """Near-flat domains that correlate with a busy range pass the square-root
    screen (L does not depend on the domain's spread) but need |c| > C."""
    rng = np.random.default_rng(11)
    caught = 0
    for _ in range(100):
        r = rng.integers(0, 256, 64)
        d = np.full(64, 500) + (r > 127)  # follows r, spread 1
        sdr, sd, sr, ncdd, ncdr = block_stats(d, r)
        L = Fraction(262144 * ncdr * ncdr, ncdd)
        M = largest_gain(ncdr, ncdd, 5)
        g = -math.floor((L + M) / 2)  # a best this domain cannot reach at |c| <= C
        v, a = screen_value(sdr, sd, sr, ncdd, with_a=True)
        caught += bool(v >= threshold(g) and a < threshold_a(g, 5))
    assert caught == 100


def test_screen_rejects_clear_losers():
    """The screen is not vacuous: candidates far worse than the row's best fail."""
    rng = np.random.default_rng(7)
    rejected = 0
    for _ in range(200):
        d, r = rng.integers(0, 1021, 64), rng.integers(0, 256, 64)
        sdr, sd, sr, ncdd, ncdr = block_stats(d, r)
        if ncdd <= 0:
            continue
        L = Fraction(262144 * ncdr * ncdr, ncdd)
        g = -2 * math.ceil(L) - 1000  # a best this candidate cannot reach
        rejected += bool(screen_value(sdr, sd, sr, ncdd) < threshold(g))
    assert rejected == 200


def test_round_f32_matches_numpy():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a = F32(rng.normal() * 10.0 ** int(rng.integers(-3, 8)))
        b = F32(rng.normal() * 10.0 ** int(rng.integers(-3, 8)))
        assert round_f32(Fraction(float(a)) * Fraction(float(b))) == a * b
        assert round_f32(Fraction(float(a)) + Fraction(float(b))) == a + b
