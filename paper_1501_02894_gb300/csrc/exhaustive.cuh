// exhaustive.cuh -- shared definitions of the exhaustive-search encoder
// (paper Section 1: every domain of the pool, every isometry).
#pragma once

#include <cuda_fp16.h>

#include "encode_common.cuh"

namespace fic {

constexpr int kExhB = 8;    // range side
constexpr int kExhK = 64;   // decimated values per block
constexpr int kExhNTile = 128;  // domains per tile (the tensor path's N)
constexpr int kExhMaxSeg = 8;   // domain segments (CTAs sharing one row tile) at most

// One image of an exhaustive-search launch; all arrays live in the workspace.
struct ExhDesc {
    const uint8_t *img;
    int32_t W, H;
    int32_t nrx, nry, nr;     // ranges per row, per column, total
    int32_t ndx, ndy, nd;     // domain grid (positions step apart), total
    int32_t nd_pad;           // nd rounded up to kExhNTile
    int32_t step, isos;
    int32_t s_bits, o_bits;
    int32_t nseg;             // domain segments whose per-row bests exh_finalize merges
    uint32_t *dpairs;         // [nd][32]   packed (d4, d4) pairs for dp2a
    __half *dsc;              // [nd_pad][64] screen operand of the tensor path, K-major, fp16:
                              //            (64 d4_k - Sd) 1024 / sqrt(nCdd) (0 for flat or padding domains)
    int4 *dstat;              // [nd_pad]   Sd, nCdd (u32), 512/nCdd (float bits), valid
    float4 *dscr;             // [nd_pad]   screening constants: -Sd/64, 64 sqrt(512^2/nCdd), 130 sqrt(512^2/nCdd), 0
                              //            (NaN: padding)
    __half *afp16;            // [nr * 8][64] range rows permuted per isometry, mean removed (r - Sr / 64), fp16
    uint8_t *rbytes;          // [nr * 8][64] the same rows as pixel bytes (exact sum r*d4 by dp2a)
    int4 *rstat;              // [nr]       Sr, Srr
    long long *row_g;         // [nseg][nr * 8] best s-part error of the (range, isometry) row
    int2 *row_dk;             // [nseg][nr * 8] its domain index and contrast code
    fic_record *rec;
    uint32_t *tile_off;
    uint32_t *split;
    uint32_t *info;
};

// Source element of isometry t for output (u, v) of a B x B block: column
// su, row sv of the decimated domain (0 identity, 1 quarter turn clockwise,
// 2 half turn, 3 quarter turn anticlockwise, 4 left-right mirror, 5 up-down
// mirror, 6 transpose, 7 anti-transpose).
__host__ __device__ inline void exh_iso_src(int t, int B, int u, int v, int &su, int &sv) {
    const int m = B - 1;
    switch (t) {
    case 0: su = u; sv = v; break;
    case 1: su = v; sv = m - u; break;
    case 2: su = m - u; sv = m - v; break;
    case 3: su = m - v; sv = u; break;
    case 4: su = m - u; sv = v; break;
    case 5: su = u; sv = m - v; break;
    case 6: su = v; sv = u; break;
    default: su = m - v; sv = m - u; break;
    }
}

// Screening of one candidate against the row's best so far.  Over real c,
// c^2 nCdd - 1024 c nCdr is smallest at c* = 512 nCdr / nCdd, where it is
// -L with L = 512^2 nCdr^2 / nCdd; the grid's best code can only do worse,
// so a candidate with L < -g (g the row's best exact error) cannot win.  The
// screen compares square roots: v = (64 |a| + 130) sqrt(512^2 / nCdd) with
// a = Sdr - (Sd / 64) Sr, nCdr / 64 formed by one fused multiply-add (Sd / 64
// and Sdr, below 2^24, are exact; |nCdr| < 2^31 bounds the single rounding
// by 1, so 64 a is nCdr within 64), so sqrt(L) <= v (1 + 3e-7); the row
// threshold sqrt(-g (1 - 1e-5) - 1) (1 - 1e-6) (or -1 while g >= 0) covers
// those relative errors, and a candidate is evaluated exactly (int64) only
// when v reaches it.  cs = (-Sd / 64, 64 sqrt(512^2 / nCdd), 130 sqrt(512^2 /
// nCdd)); padding domains carry NaN and never pass.
__device__ __forceinline__ float exh_screen(float sdr_f, float sr_f, float4 cs) {
    const float a = fmaf(cs.x, sr_f, sdr_f);
    return fmaf(fabsf(a), cs.y, cs.z);
}

// The magnitude |a| of the screen's a = nCdr / 64 as well: the CUDA-core
// engine's per-candidate pass uses both.
__device__ __forceinline__ float exh_screen_abs(float sdr_f, float sr_f, float4 cs, float &abs_a) {
    abs_a = fabsf(fmaf(cs.x, sr_f, sdr_f));
    return fmaf(abs_a, cs.y, cs.z);
}

// Second necessary condition, from the contrast range: at a code |c| <= C =
// 128 - 128 / 2^s_bits the score c^2 nCdd - 1024 c nCdr is at least
// -1024 C |nCdr|, so a candidate that can reach g has |nCdr| / 64 >=
// -g / (65536 C), and the screen's |a| (within 1 of |nCdr| / 64) is at least
// that minus 1.  It rejects domains that correlate well with the range but
// would need a contrast outside the codebook (the square-root screen ignores
// the range of c).  The threshold -g (1 - 1e-5) / (65536 C) - 1 covers the
// float roundings; -1 while g >= 0 (everything passes).
__device__ __forceinline__ float exh_threshold_a(long long g, int s_bits) {
    if (g >= 0) return -1.f;
    const float C = (float)(128 - (128 >> s_bits));
    return (float)(-g) * ((1.f - 1e-5f) / (65536.f * C)) - 1.f;
}

__device__ __forceinline__ float exh_threshold(long long g) {
    const float t = (float)(-g) * (1.f - 1e-5f) - 1.f;
    return t > 0.f ? sqrtf(t) * (1.f - 1e-6f) : -1.f;
}

// (g, d) lexicographic improvement: the smaller domain index wins ties.
__device__ __forceinline__ bool exh_better(long long g, int d, long long bg, int bd) {
    return g < bg || (g == bg && (unsigned)d < (unsigned)bd);
}

}  // namespace fic
