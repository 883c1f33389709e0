// encode_common.cuh -- device helpers shared by the encoder kernels: the
// exact phase-1 fit (Section 3), the phase-2 sub-block test (Sections
// 3.1-3.2), lane-group reductions of the strip/patch geometry, leaf records
// and the per-patch moment sums (dp2a on packed decimated pairs).
#pragma once

#include "fic_internal.cuh"

namespace fic {

// Result of the phase-1 fit of one block.
struct Fit {
    long long ncrr, ncdr, ncdd;  // n Srr - Sr^2, n Sdr - Sd Sr, n Sdd - Sd^2
    int sr;
    int k, q;
    bool pass;  // collage error below the level threshold
};

__device__ __forceinline__ int lum(int q, int ko1, uint32_t magic) {
    // floor((510 q + ko1) / (2 ko1)) by multiply-high; exact for these ranges
    return (int)__umulhi((uint32_t)(510 * q + ko1), magic);
}

// The contrast code minimising c^2 nCdd - 1024 c nCdr over the 2^s_bits
// grid: the grid point nearest to c* = 512 nCdr / nCdd, from a float estimate
// settled by exact int64 comparisons against the grid midpoints; ties go to
// the smaller |c|, then to c > 0.  A flat domain (nCdd = 0, hence nCdr = 0)
// gives the smallest positive code.
// FAST: the estimate's division by the fast intrinsic (measured faster in the
// quadtree encoders, slower in the CUDA-core exhaustive search, whose hot
// loop compiles differently around it); the result is exact either way.
template <bool FAST = false>
__device__ __forceinline__ int best_contrast(long long ncdr, long long ncdd, int s_bits) {
    const int K = 1 << s_bits, step = 256 >> s_bits;
    if (ncdd <= 0) return K >> 1;
    // an estimate only, settled exactly below
    float cs = FAST ? __fdividef(512.f * (float)ncdr, (float)ncdd) : 512.f * (float)ncdr / (float)ncdd;
    float kf = (cs + 128.f) / (float)step - 0.5f;
    kf = fminf(fmaxf(kf, 0.f), (float)(K - 1));
    const float kr = rintf(kf);
    int k = (int)kr;
    // Far from every grid midpoint (k +- 1/2) the estimate is the answer.  Its
    // error, for a c* within the grid (|c*| <= 128 + step / 2; beyond it the
    // clamp decides), is at most |c*| (2^-24 + 2^-24 + 2^-22) from the two
    // roundings to float and the approximate division, plus 2^-24 (|c*| + 128)
    // from the sum, divided by the step (>= 2): below 3e-5, far inside the
    // 1e-3 band around a midpoint that goes to the exact comparisons below.
    if (fabsf(kf - kr) < 0.499f) return k;
    const long long a = 512LL * ncdr;
#pragma unroll 1
    for (int it = 0; it < K && k < K - 1; ++it) {
        long long m = (long long)(step * (k + 1) - 128);
        long long b = m * ncdd;
        if (a > b || (a == b && m <= 0)) ++k;
        else break;
    }
#pragma unroll 1
    for (int it = 0; it < K && k > 0; ++it) {
        long long m = (long long)(step * k - 128);
        long long b = m * ncdd;
        if (a > b || (a == b && m <= 0)) break;
        --k;
    }
    return k;
}

// The luminance code whose level is nearest the block mean Sr / n (ties to
// the smaller code); *dist = |Sr - n L(q)|.  The float estimate q0 is within
// one code of the answer; the levels increase with q, so the answer is q0 or
// its neighbour on the side of the block mean, settled by the exact distance.
__device__ __forceinline__ int best_luminance(int sr, int lg2n, int ko1, uint32_t magic, float qscale, int &dist) {
    int q0 = __float2int_rn((float)sr * qscale * __int_as_float((127 - lg2n) << 23));
    q0 = clampi(q0, 0, ko1);
    const int d0 = sr - (lum(q0, ko1, magic) << lg2n);
    // the answer is q0 or its neighbour on the side of the block mean
    const bool up = d0 >= 0;
    const int q1 = up ? q0 + 1 : q0 - 1;
    const bool ok1 = up ? q1 <= ko1 : q1 >= 0;
    const int d1 = ok1 ? abs(sr - (lum(q1, ko1, magic) << lg2n)) : 0x7fffffff;
    const int a0 = abs(d0);
    // ties: the smaller code
    const bool take1 = up ? d1 < a0 : d1 <= a0;
    dist = take1 ? d1 : a0;
    return take1 ? q1 : q0;
}

// Phase-1 fit (Section 3: the best contrast factor for the one domain, the
// error, the threshold test).  Exact: the contrast code is the grid point
// nearest to c* = 512 nCdr / nCdd, found from a float estimate and settled by
// int64 comparisons against the grid midpoints; ties go to the smaller |c|,
// then to c > 0.  The luminance code is the level nearest the block mean.
__device__ __forceinline__ void fit_phase1(int sr, int srr, int sd, int sdd, int sdr, int lg2n,
                                           int s_bits, int ko1, uint32_t magic, float qscale,
                                           long long thr, Fit &f) {
    f.sr = sr;
    f.ncrr = ((long long)srr << lg2n) - (long long)sr * sr;
    f.ncdr = ((long long)sdr << lg2n) - (long long)sd * sr;
    f.ncdd = ((long long)sdd << lg2n) - (long long)sd * sd;
    const int k = best_contrast<true>(f.ncdr, f.ncdd, s_bits);
    int bd;
    const int bq = best_luminance(sr, lg2n, ko1, magic, qscale, bd);
    f.k = k;
    f.q = bq;
    const long long c = contrast_code(k, s_bits);
    const long long e = (long long)bd;
    const long long E = 262144LL * f.ncrr - 1024LL * c * f.ncdr + c * c * f.ncdd + 262144LL * e * e;
    f.pass = E < thr;
}

// Collage error of a phase-2 sub-block with a given luminance and the
// better of the level's two contrasts (Section 3.2); returns pass and bit.
__device__ __forceinline__ bool fit_phase2_sub(const Fit &f, int lg2n, int O, int c0, int c1,
                                               long long thr, int &bit) {
    // E(c1) < E(c0)  <=>  (c1 + c0) nCdd < 1024 nCdr   (c1 > c0)
    bit = ((long long)(c1 + c0) * f.ncdd < 1024LL * f.ncdr) ? 1 : 0;
    const long long c = bit ? c1 : c0;
    const long long e = (long long)f.sr - ((long long)O << lg2n);
    const long long E = 262144LL * f.ncrr - 1024LL * c * f.ncdr + c * c * f.ncdd + 262144LL * e * e;
    return E < thr;
}

// Bitmask of the lanes that form the lane's block when a block spans gx patch
// columns and gy patch rows.
template <int PC>
__device__ __forceinline__ uint32_t group_mask(int pc, int pr, int gx, int gy) {
    // gy rows of gx bits, PC apart: the row pattern times a comb of gy ones
    // spaced PC apart (gx <= PC, so the copies do not overlap)
    static_assert(PC == 4 || PC == 8 || PC == 16, "patch columns per strip");
    constexpr uint32_t COMB = PC == 4 ? 0x11111111u : (PC == 8 ? 0x01010101u : 0x00010001u);
    const int base = (pr & ~(gy - 1)) * PC + (pc & ~(gx - 1));  // gx, gy powers of two
    const uint32_t row = (1u << gx) - 1u;
    return (row * (COMB >> (32 - PC * gy))) << base;
}

template <int PC>
__device__ __forceinline__ int group_sum(int v, int gx, int gy) {
    // a block spanning the whole warp (warp-uniform): one reduction
    if (gx * gy == 32) return __reduce_add_sync(0xffffffffu, v);
    for (int m = 1; m < gx; m <<= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    for (int m = 1; m < gy; m <<= 1) v += __shfl_xor_sync(0xffffffffu, v, m * PC);
    return v;
}

template <int PC>
__device__ __forceinline__ uint32_t group_or(uint32_t v, int gx, int gy) {
    if (gx * gy == 32) return __reduce_or_sync(0xffffffffu, v);  // the whole warp (warp-uniform)
    for (int m = 1; m < gx; m <<= 1) v |= __shfl_xor_sync(0xffffffffu, v, m);
    for (int m = 1; m < gy; m <<= 1) v |= __shfl_xor_sync(0xffffffffu, v, m * PC);
    return v;
}

struct Leaf {
    uint32_t w0, w1, w2, w3;  // the 16-byte fic_record
    int pos;                  // canonical position in the strip, -1 = none
};

__device__ __forceinline__ void make_leaf(Leaf &L, int x, int y, int level, int phase, int k, int q,
                                          int d0, int d1, int d2, int dx, int dy, int pos) {
    L.w0 = (uint32_t)x | ((uint32_t)y << 16);
    L.w1 = (uint32_t)level | ((uint32_t)phase << 8) | ((uint32_t)k << 16) | ((uint32_t)q << 24);
    L.w2 = ((uint32_t)d0 & 0xffu) | (((uint32_t)d1 & 0xffu) << 8) | (((uint32_t)d2 & 0xffu) << 16);
    L.w3 = (uint32_t)dx | ((uint32_t)dy << 16);
    L.pos = pos;
}

// Moments of the lane's part of a block of side B >= 8: the patch's 4 rows x
// 8 pixels against the 4 x 8 decimated domain values at (c, rr) (c even).
template <int NP>
__device__ __forceinline__ void patch_moments(const uint32_t *d4e, int c, int rr, const uint2 *rw,
                                              int &sd, int &sdd, int &sdr) {
    unsigned a_dr = 0, pk = 0, ql = 0, qh = 0;
    const uint32_t *base = d4e + rr * NP + (c >> 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        // 32-bit loads: for 8x8 blocks the window starts at an odd word
        const uint2 lo = make_uint2(base[i * NP], base[i * NP + 1]);
        const uint2 hi = make_uint2(base[i * NP + 2], base[i * NP + 3]);
        a_dr = dp2a_lo(lo.x, rw[i].x, a_dr);
        a_dr = dp2a_hi(lo.y, rw[i].x, a_dr);
        a_dr = dp2a_lo(hi.x, rw[i].y, a_dr);
        a_dr = dp2a_hi(hi.y, rw[i].y, a_dr);
        pk += lo.x + lo.y + hi.x + hi.y;
        acc_sq(lo.x, ql, qh);
        acc_sq(lo.y, ql, qh);
        acc_sq(hi.x, ql, qh);
        acc_sq(hi.y, ql, qh);
    }
    sd = (int)((pk & 0xffffu) + (pk >> 16));
    sdd = (int)(ql + (qh << 8));
    sdr = (int)a_dr;
}

// Moments of one 4x4 block (one half of the patch): 4 rows x 4 pixels (word
// `h` of each row) against 4 x 4 decimated values starting at column c of
// either parity (an odd start is realigned from three even pairs).
template <int NP>
__device__ __forceinline__ void half_moments(const uint32_t *d4e, int c, int rr, const uint2 *rw, int h,
                                             int &sd, int &sdd, int &sdr) {
    unsigned a_dr = 0, pk = 0, ql = 0, qh = 0;
    const uint32_t *base = d4e + rr * NP + (c >> 1);
    const bool odd = c & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t e0 = base[i * NP], e1 = base[i * NP + 1];
        uint32_t p0 = e0, p1 = e1;
        if (odd) {
            const uint32_t e2 = base[i * NP + 2];
            p0 = __funnelshift_r(e0, e1, 16);
            p1 = __funnelshift_r(e1, e2, 16);
        }
        const uint32_t r = h ? rw[i].y : rw[i].x;
        a_dr = dp2a_lo(p0, r, a_dr);
        a_dr = dp2a_hi(p1, r, a_dr);
        pk += p0 + p1;
        acc_sq(p0, ql, qh);
        acc_sq(p1, ql, qh);
    }
    sd = (int)((pk & 0xffffu) + (pk >> 16));
    sdd = (int)(ql + (qh << 8));
    sdr = (int)a_dr;
}

// 2x2 sums of two rows of four pixels: (p0+p1+q0+q1) | (p2+p3+q2+q3) << 16.
__device__ __forceinline__ uint32_t pair2x2(uint32_t a, uint32_t b) {
    const uint32_t lo = __dp4a(a, 0x00000101u, __dp4a(b, 0x00000101u, 0u));
    const uint32_t hi = __dp4a(a, 0x01010000u, __dp4a(b, 0x01010000u, 0u));
    return __byte_perm(lo, hi, 0x5410);
}

// Phase-1 summary of a block that the level loop carries forward.
struct Code {
    int k, q;
    bool pass;
};

}  // namespace fic
