"""The encoders' contrast-code search settles on the nearest code from any start.

The contrast s is coded as c = 128 s on 2^s_bits cell midpoints of [-1, 1)
(Section 3.3): c_k = (2k - (K - 1)) 128 / K, K = 2^s_bits.  For a block with
nCdd > 0 the kernels pick the code nearest c* = 512 nCdr / nCdd -- ties to the
smaller |c|, then to c > 0 -- by a float estimate of k followed by integer
steps against the midpoints m = 256 (k + 1) / K - 128 between neighbouring
codes (step up while 512 nCdr > m nCdd, or equal with m <= 0; then step down
while the lower midpoint is not passed).  The estimate uses an approximate
division, so the result must not depend on it: this test starts the integer
steps from every k and compares with a search over all codes, including exact
ties (c* on a midpoint), where the tie rule decides."""
from fractions import Fraction

import numpy as np
import pytest


def code(k, s_bits):
    K = 1 << s_bits
    return (2 * k - (K - 1)) * (128 >> s_bits)


def nearest_by_definition(ncdr, ncdd, s_bits):
    K = 1 << s_bits
    cstar = Fraction(512 * ncdr, ncdd)
    return min(range(K), key=lambda k: (abs(cstar - code(k, s_bits)), abs(code(k, s_bits)), -code(k, s_bits)))


def settle(k, ncdr, ncdd, s_bits):
    """The kernels' integer steps from a start k (any value in [0, K - 1])."""
    K, step = 1 << s_bits, 256 >> s_bits
    a = 512 * ncdr
    for _ in range(K):
        if k >= K - 1:
            break
        m = step * (k + 1) - 128
        if a > m * ncdd or (a == m * ncdd and m <= 0):
            k += 1
        else:
            break
    for _ in range(K):
        if k <= 0:
            break
        m = step * k - 128
        if a > m * ncdd or (a == m * ncdd and m <= 0):
            break
        k -= 1
    return k


def blocks(rng, s_bits):
    K, step = 1 << s_bits, 256 >> s_bits
    for _ in range(150):  # general positions, c* inside and far outside [-128, 128)
        ncdd = int(rng.integers(1, 1 << 32))
        ncdr = int(rng.integers(-(1 << 30), 1 << 30)) * int(rng.choice([1, 1, 1, 64]))
        yield ncdr, ncdd
    for k in range(K - 1):  # c* exactly on every midpoint: the tie rule decides
        m = step * (k + 1) - 128
        t = int(rng.integers(1, 1 << 12))
        yield m * t, 512 * t
    for c in (-128, 0, 127, 128):  # the range ends and zero
        t = int(rng.integers(1, 1 << 12))
        yield c * t, 512 * t


@pytest.mark.parametrize("s_bits", range(1, 8))
def test_integer_steps_reach_the_nearest_code_from_every_start(s_bits):
    rng = np.random.default_rng(100 + s_bits)
    K = 1 << s_bits
    for ncdr, ncdd in blocks(rng, s_bits):
        want = nearest_by_definition(ncdr, ncdd, s_bits)
        starts = range(K) if K <= 32 else list(range(0, K, 7)) + [K - 1]
        for k0 in starts:
            assert settle(k0, ncdr, ncdd, s_bits) == want, (s_bits, ncdr, ncdd, k0)


def test_midpoint_ties_follow_the_rule():
    """On the midpoint between c = -4 and c = +4 (s_bits 5) the positive code
    wins; between 4 and 12 the smaller |c| wins; between -12 and -4 likewise."""
    s = 5
    assert code(settle(0, 0, 512, s), s) == 4
    assert code(settle(0, 8, 512, s), s) == 4
    assert code(settle(31, -8, 512, s), s) == -4


@pytest.mark.parametrize("s_bits", (1, 3, 5, 7))
def test_nearest_code_is_the_oracles_smallest_score(orc, s_bits):
    """The oracle scans every code for the smallest c^2 nCdd - 1024 c nCdr with
    the same tie rule; nearest-to-c* is the same choice (the score is
    nCdd (c - c*)^2 up to a constant), on the oracle's own codebook."""
    rng = np.random.default_rng(7 + s_bits)
    K = 1 << s_bits
    codes = [orc.contrast(k, s_bits) for k in range(K)]
    assert codes == [code(k, s_bits) for k in range(K)]
    for ncdr, ncdd in blocks(rng, s_bits):
        g = [c * c * ncdd - 1024 * c * ncdr for c in codes]
        best = min(range(K), key=lambda k: (g[k], abs(codes[k]), -codes[k]))
        assert best == nearest_by_definition(ncdr, ncdd, s_bits)


def screened(ncdr, ncdd, s_bits, ulps):
    """The kernels' float screen with its quotient moved by `ulps` units in
    the last place (the approximate division is within 2 ulp of the exact
    quotient of the rounded operands): the code it returns, or None when it
    hands the block to the integer steps."""
    K, step = 1 << s_bits, 256 >> s_bits
    num = np.float32(512.0) * np.float32(ncdr)
    q = np.float32(num / np.float32(ncdd))
    for _ in range(abs(ulps)):
        q = np.nextafter(q, np.float32(np.inf) if ulps > 0 else np.float32(-np.inf), dtype=np.float32)
    kf = np.float32(np.float32(q + np.float32(128.0)) / np.float32(step)) - np.float32(0.5)
    kf = np.float32(min(max(kf, np.float32(0.0)), np.float32(K - 1)))
    kr = np.float32(np.rint(kf))
    return int(kr) if abs(np.float32(kf - kr)) < np.float32(0.499) else None


@pytest.mark.parametrize("s_bits", range(1, 8))
def test_float_screen_never_returns_a_wrong_code(s_bits):
    """Whenever the screen returns a code without the integer steps, it is
    the nearest code, with the division off by up to 2 ulp either way; blocks
    on or next to a midpoint go to the integer steps."""
    rng = np.random.default_rng(200 + s_bits)
    K, step = 1 << s_bits, 256 >> s_bits
    cases = list(blocks(rng, s_bits))
    for k in range(K - 1):  # c* a hair either side of every midpoint
        m = step * (k + 1) - 128
        for eps in (-3, -1, 1, 3):
            t = int(rng.integers(1 << 20, 1 << 30))
            cases.append((m * t + eps, 512 * t))
    decided = 0
    for ncdr, ncdd in cases:
        want = nearest_by_definition(ncdr, ncdd, s_bits)
        for u in (-2, 0, 2):
            got = screened(ncdr, ncdd, s_bits, u)
            if got is not None:
                decided += 1
                assert got == want, (s_bits, ncdr, ncdd, u, got, want)
    assert decided > len(cases) // 2  # the screen decides most blocks by itself
