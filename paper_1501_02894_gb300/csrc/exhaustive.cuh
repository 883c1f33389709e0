// exhaustive.cuh -- shared definitions of the exhaustive-search encoder
// (paper Section 1: every domain of the pool, every isometry).
#pragma once

#include <cuda_fp16.h>

#include "encode_common.cuh"

namespace fic {

constexpr int kExhB = 8;    // range side
constexpr int kExhK = 64;   // decimated values per block
constexpr int kExhNTile = 128;  // domains per tile (the tensor path's N)

// One image of an exhaustive-search launch; all arrays live in the workspace.
struct ExhDesc {
    const uint8_t *img;
    int32_t W, H;
    int32_t nrx, nry, nr;     // ranges per row, per column, total
    int32_t ndx, ndy, nd;     // domain grid (positions step apart), total
    int32_t nd_pad;           // nd rounded up to kExhNTile
    int32_t step, isos;
    int32_t s_bits, o_bits;
    uint32_t *dpairs;         // [nd][32]   packed (d4, d4) pairs for dp2a
    __half *dfp16;            // [nd_pad][64] decimated domains, K-major, fp16
    int4 *dstat;              // [nd_pad]   Sd, nCdd (u32), 512/nCdd (float bits), valid
    float2 *dscr;             // [nd_pad]   screening constants: -Sd, 512^2/nCdd (NaN: padding)
    __half *afp16;            // [nr * 8][64] range rows permuted per isometry, fp16
    int4 *rstat;              // [nr]       Sr, Srr
    long long *row_g;         // [nr * 8]   best s-part error of the (range, isometry) row
    int2 *row_dk;             // [nr * 8]   its domain index and contrast code
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
// so a candidate with -L >= the row's best exact error g cannot win (ties
// keep the earlier domain).  The screen computes an upper bound of L in
// float: nCdr = 64 Sdr - Sd Sr is formed with at most 64 of absolute
// rounding error (|nCdr| < 2^31, Sdr exact below 2^24), widened by 130, and
// the product's relative error (< 1e-6) is covered by the row threshold
// thr(g) = -g (1 - 1e-5) - 1: a candidate is evaluated exactly (int64) only
// when its bound reaches thr.  Padding domains carry NaN and never pass.
__device__ __forceinline__ float exh_screen(float sdr_f, float sr_f, float2 cs) {
    const float u = fabsf(fmaf(sdr_f, 64.f, cs.x * sr_f)) + 130.f;
    return u * u * cs.y;
}

__device__ __forceinline__ float exh_threshold(long long g) { return (float)(-g) * (1.f - 1e-5f) - 1.f; }

}  // namespace fic
