"""The encoders' luminance-code shortcut equals the definition, exhaustively.

The offset o of a block is coded as the level L(q) = floor((510 q + K) / (2 K))
(K = 2^o_bits - 1) nearest the block mean Sr / n, ties to the smaller code
(Section 3, the quantised offset).  The kernels estimate the code in float32,
q0 = round_half_even(float(Sr) * float(K / 255) * 2^-lg2n), clamp it to
[0, K], and compare q0 with its one neighbour on the side of the block mean
(q0 + 1 when Sr >= n L(q0), else q0 - 1) by the exact integer distance
|Sr - n L(q)|.  That is right only if the estimate is never two or more codes
from the answer and the levels increase strictly with q.  This test replays the float steps bit for bit (numpy float32
is IEEE round-to-nearest) for every Sr of every block size 2^lg2n (1 to 4096
pixels) and every code width, and compares code and distance with a search
over all codes."""
import numpy as np
import pytest

F32 = np.float32


def levels(o_bits):
    k = (1 << o_bits) - 1
    q = np.arange(k + 1, dtype=np.int64)
    return (510 * q + k) // (2 * k)


def nearest_by_definition(sr, lg2n, lev):
    """Code q minimising |sr - n L(q)|, ties to the smaller q (all codes searched)."""
    nl = lev << lg2n
    hi = np.clip(np.searchsorted(nl, sr, side="left"), 0, len(nl) - 1)
    lo = np.clip(hi - 1, 0, len(nl) - 1)
    dlo, dhi = np.abs(sr - nl[lo]), np.abs(sr - nl[hi])
    q = np.where(dlo <= dhi, lo, hi)
    return q, np.minimum(dlo, dhi)


def kernel_estimate(sr, lg2n, o_bits, lev):
    k = (1 << o_bits) - 1
    qscale = F32(k) / F32(255.0)
    x = (sr.astype(F32) * qscale) * F32(2.0 ** -lg2n)
    q0 = np.clip(np.rint(x).astype(np.int64), 0, k)
    d0 = sr - (lev[q0] << lg2n)
    up = d0 >= 0
    q1 = np.where(up, q0 + 1, q0 - 1)
    ok1 = np.where(up, q1 <= k, q1 >= 0)
    big = np.iinfo(np.int64).max
    d1 = np.where(ok1, np.abs(sr - (lev[np.clip(q1, 0, k)] << lg2n)), big)
    a0 = np.abs(d0)
    take1 = np.where(up, d1 < a0, d1 <= a0)
    return np.where(take1, q1, q0), np.where(take1, d1, a0)


def test_levels_are_increasing_and_span_the_range():
    for o_bits in range(1, 9):
        lev = levels(o_bits)
        assert lev[0] == 0 and lev[-1] == 255
        assert np.all(np.diff(lev) >= 1)


@pytest.mark.parametrize("o_bits", range(1, 9))
def test_estimate_window_finds_the_nearest_level(o_bits):
    lev = levels(o_bits)
    for lg2n in range(0, 13):
        sr = np.arange(0, 255 * (1 << lg2n) + 1, dtype=np.int64)
        q_ref, d_ref = nearest_by_definition(sr, lg2n, lev)
        q, d = kernel_estimate(sr, lg2n, o_bits, lev)
        bad = np.nonzero((q != q_ref) | (d != d_ref))[0]
        assert bad.size == 0, (o_bits, lg2n, sr[bad[:5]], q[bad[:5]], q_ref[bad[:5]])
