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

// Screening of one candidate against the row's best so far.  g* (the
// minimum over the contrast grid of c^2 nCdd - 1024 c nCdr) is at least
// nCdd (dmin^2 - c*^2) with c* = 512 nCdr / nCdd the unconstrained optimum
// and dmin the distance from c* to the nearest grid code.  The bound is
// evaluated in float with a margin; a candidate is evaluated exactly (int64)
// only when the bound does not exclude it.
struct ExhCand {
    float cs;    // c* (clamped to the grid's range)
    float lb;    // lower bound of g*, minus the float margin
};

__device__ __forceinline__ float exh_lower_bound(float ncdr_f, float ncdd_f, float k512_over_ncdd, int s_bits) {
    // c* = 512 nCdr / nCdd ; g_cont = -c*^2 nCdd
    const int K = 1 << s_bits;
    const float step = (float)(256 >> s_bits);
    const float cmax = (float)((K - 1) * (128 >> s_bits));  // = 128 - step/2
    float cs = ncdr_f * k512_over_ncdd;
    const float csc = fminf(fmaxf(cs, -cmax), cmax);
    // nearest grid point to csc: c_k = step*k - 128 + step/2
    const float t = (csc + 128.f - 0.5f * step) / step;
    const float cnear = fmaf(rintf(t), step, 0.5f * step - 128.f);
    // a float slip near a grid midpoint may pick the second-nearest code:
    // shrink the distance by more than the possible error
    const float d = fmaxf(fabsf(cs - cnear) - 1e-3f, 0.f);
    // g(c) = nCdd (c - c*)^2 - nCdd c*^2
    const float g = ncdd_f * (d * d - cs * cs);
    const float mag = ncdd_f * (d * d + cs * cs);
    return g - (1e-5f * mag + 64.f);
}

}  // namespace fic
