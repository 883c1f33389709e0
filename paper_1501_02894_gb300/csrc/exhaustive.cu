// exhaustive.cu -- exhaustive domain search (paper Section 1): every range
// block (flat 8x8 partition) against every domain on a grid of step
// `dom_step`, under every isometry; the pair with the smallest collage error
// wins, ties to the smaller domain index, then the smaller isometry.
//
// Sum r*d4 of all (range, isometry) x domain pairs is a dense contraction
// over the 64 decimated values of a block, so it is computed either on the
// CUDA cores here (dp2a on packed operands), or replaced on the tensor cores
// (exhaustive_tc.cu: tcgen05, fp16 operands, fp32 accumulators) by a
// contraction that yields each candidate's screen value directly.  Either
// way a float bound of each candidate's best contrast error skips it unless
// it may beat the row's best, which is then settled in exact int64
// arithmetic.  The isometry is applied on the range side: row
// (range, t) holds the range pixel r(u, v) at the position of the domain
// element it meets under isometry t.
#include "exhaustive.cuh"

namespace fic {

// Decimated domains: packed pairs for dp2a, per-domain statistics (Sd,
// nCdd, 512 / nCdd), the CUDA-core engine's screening constants, and the
// tensor path's screen operand: x_k = 64 d4_k - Sd (sum x_k = 0, sum x_k^2 =
// 64 nCdd) scaled by 1024 / sqrt(nCdd), so that sum_k r_k w_k = 1024 nCdr /
// sqrt(nCdd) = 2 sqrt(L) in magnitude (L: exhaustive.cuh); |w_k| <= 8192.
// Eight threads per domain, one per row of its 8 x 8 decimated block; the
// grid covers nd_pad domains exactly.
__global__ void __launch_bounds__(256) exh_prep_domains(ExhDesc E) {
    const unsigned FULL = 0xffffffffu;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = gt >> 3, v = gt & 7;
    const bool real = d < E.nd;
    int vals[kExhB];
    int sd = 0, sdd = 0;  // sum d4^2 <= 64 * 1020^2 < 2^31
    if (real) {
        const int dy = (d / E.ndx) * E.step, dx = (d % E.ndx) * E.step;
        const uint8_t *p = E.img + (size_t)(dy + 2 * v) * E.W + dx;
#pragma unroll
        for (int u = 0; u < kExhB; ++u) {
            vals[u] = (int)p[2 * u] + p[2 * u + 1] + p[E.W + 2 * u] + p[E.W + 2 * u + 1];
            sd += vals[u];
            sdd += vals[u] * vals[u];
        }
    } else {
#pragma unroll
        for (int u = 0; u < kExhB; ++u) vals[u] = 0;
    }
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
        sd += __shfl_xor_sync(FULL, sd, m);
        sdd += __shfl_xor_sync(FULL, sdd, m);
    }
    if (d >= E.nd_pad) return;
    uint4 *wrow = reinterpret_cast<uint4 *>(E.dsc + (size_t)d * kExhK + v * kExhB);
    if (!real) {
        *wrow = make_uint4(0u, 0u, 0u, 0u);
        if (v == 0) {
            E.dstat[d] = make_int4(0, 0, 0, 0);
            E.dscr[d] = make_float4(0.f, __int_as_float(0x7fc00000), __int_as_float(0x7fc00000), 0.f);  // NaN
        }
        return;
    }
    *reinterpret_cast<uint4 *>(E.dpairs + (size_t)d * 32 + v * 4) =
        make_uint4((uint32_t)vals[0] | ((uint32_t)vals[1] << 16), (uint32_t)vals[2] | ((uint32_t)vals[3] << 16),
                   (uint32_t)vals[4] | ((uint32_t)vals[5] << 16), (uint32_t)vals[6] | ((uint32_t)vals[7] << 16));
    const long long ncdd = 64LL * sdd - (long long)sd * sd;  // <= 4.3e9: fits an unsigned word
    const float s = ncdd > 0 ? 1024.f / sqrtf((float)ncdd) : 0.f;
    uint32_t hw[4];
#pragma unroll
    for (int u = 0; u < kExhB; u += 2) {
        const uint32_t lo = __half_as_ushort(__float2half_rn((float)(64 * vals[u] - sd) * s));
        const uint32_t hi = __half_as_ushort(__float2half_rn((float)(64 * vals[u + 1] - sd) * s));
        hw[u / 2] = lo | (hi << 16);
    }
    *wrow = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    if (v == 0) {
        const float k512 = ncdd > 0 ? 512.f / (float)ncdd : 0.f;
        E.dstat[d] = make_int4(sd, (int)(uint32_t)ncdd, __float_as_int(k512), 1);
        const float sw = ncdd > 0 ? sqrtf(262144.f / (float)ncdd) : 0.f;
        E.dscr[d] = make_float4(-(float)sd * 0.015625f, 64.f * sw, 130.f * sw, 0.f);
    }
}

// Range rows, one per (range, isometry): A[sv * 8 + su] = r(u, v) where
// (su, sv) is the domain element that isometry t puts at (u, v), as bytes,
// and the tensor path's screen operand: the same row with the range's mean
// removed, r - Sr / 64, in fp16.  Eight threads per row, one per row sv of
// A: its element su holds the pixel at the inverse isometry's image of
// (su, sv) (the quarter turns 1 and 3 are each other's inverse, the other
// six are involutions).  The grid covers the nr * 8 rows exactly.
__global__ void __launch_bounds__(256) exh_prep_ranges(ExhDesc E) {
    const unsigned FULL = 0xffffffffu;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = gt >> 3, sv = gt & 7;
    const bool real = row < E.nr * 8;
    const int r = row >> 3, t = row & 7;
    int sr = 0, srr = 0;
    int px[kExhB];
    if (real) {
        const int x = (r % E.nrx) * kExhB, y = (r / E.nrx) * kExhB;
        const int ti = t == 1 ? 3 : (t == 3 ? 1 : t);
#pragma unroll
        for (int su = 0; su < kExhB; ++su) {
            int u, v;
            exh_iso_src(ti, kExhB, su, sv, u, v);
            px[su] = E.img[(size_t)(y + v) * E.W + x + u];
            sr += px[su];
            srr += px[su] * px[su];
        }
    } else {
#pragma unroll
        for (int su = 0; su < kExhB; ++su) px[su] = 0;
    }
#pragma unroll
    for (int m = 1; m < 8; m <<= 1) {
        sr += __shfl_xor_sync(FULL, sr, m);
        srr += __shfl_xor_sync(FULL, srr, m);
    }
    if (real) {
        uint32_t hw[4] = {0u, 0u, 0u, 0u}, bw[2] = {0u, 0u};
        const float mean = (float)sr * 0.015625f;  // exact (a multiple of 1/64 below 256)
#pragma unroll
        for (int su = 0; su < kExhB; ++su) {
            hw[su / 2] |= (uint32_t)__half_as_ushort(__float2half_rn((float)px[su] - mean)) << (16 * (su & 1));
            bw[su / 4] |= (uint32_t)px[su] << (8 * (su & 3));
        }
        *reinterpret_cast<uint4 *>(E.afp16 + (size_t)row * kExhK + sv * kExhB) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint2 *>(E.rbytes + (size_t)row * kExhK + sv * kExhB) = make_uint2(bw[0], bw[1]);
    }
    if (real && t == 0 && sv == 0) E.rstat[r] = make_int4(sr, srr, 0, 0);
}

// Row state of the screening epilogue.
struct ExhRow {
    long long g;  // best exact s-part error
    float thr;    // screening threshold of g (exh_threshold)
    float thra;   // threshold on |a| (exh_threshold_a)
    int d, k;
};

__device__ __forceinline__ void exh_row_init(ExhRow &b) {
    b.g = 0x7fffffffffffffffLL;
    b.thr = __int_as_float(0xff800000);  // -inf: everything passes
    b.thra = -1.f;
    b.d = -1;
    b.k = 0;
}

// Exact evaluation of candidate domain d (sum r*d4 = sdr) for the row.
// Domains are offered in increasing order, so a strict improvement test
// keeps the smallest domain index among equal errors.
__device__ __forceinline__ void exh_exact(ExhRow &b, int d, int sdr, int sr, int4 ds, int s_bits) {
    const int ncdr = 64 * sdr - ds.x * sr;
    const uint32_t ncdd = (uint32_t)ds.y;
    const int k = best_contrast((long long)ncdr, (long long)ncdd, s_bits);
    const long long c = contrast_code(k, s_bits);
    const long long g = c * c * (long long)ncdd - 1024LL * c * ncdr;
    if (exh_better(g, d, b.g, b.d)) {
        b.g = g;
        b.thr = exh_threshold(g);
        b.thra = exh_threshold_a(g, s_bits);
        b.d = d;
        b.k = k;
    }
}

// CUDA-core search: a warp holds 4 ranges x 8 isometries (one row per lane),
// domains are staged 64 at a time in shared memory and read by broadcast.
constexpr int kExhWarps = 4;
constexpr int kExhStage = 64;

__global__ void __launch_bounds__(kExhWarps * 32) exh_cuda_kernel(ExhDesc E) {
    __shared__ __align__(16) uint32_t s_dp[kExhStage][32];
    __shared__ int4 s_ds[kExhStage];
    __shared__ float4 s_cs[kExhStage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (blockIdx.x * kExhWarps + warp) * 4 + (lane >> 3);
    const int t = lane & 7;
    const bool live = r < E.nr && t < E.isos;
    // the row's permuted range pixels as 16 words of 4 bytes
    uint32_t aw[16];
    int sr = 0;
    {
        const int rr = live ? r : 0;
        const int x = (rr % E.nrx) * kExhB, y = (rr / E.nrx) * kExhB;
        uint8_t a[kExhK];
#pragma unroll
        for (int v = 0; v < kExhB; ++v) {
#pragma unroll
            for (int u = 0; u < kExhB; ++u) {
                int su, sv;
                exh_iso_src(t, kExhB, u, v, su, sv);
                const uint8_t px = E.img[(size_t)(y + v) * E.W + x + u];
                a[sv * kExhB + su] = px;
                sr += px;
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
            aw[i] = (uint32_t)a[4 * i] | ((uint32_t)a[4 * i + 1] << 8) | ((uint32_t)a[4 * i + 2] << 16) |
                    ((uint32_t)a[4 * i + 3] << 24);
    }
    ExhRow best;
    exh_row_init(best);
    for (int d0 = 0; d0 < E.nd; d0 += kExhStage) {
        __syncthreads();
        for (int i = threadIdx.x; i < kExhStage * 32; i += blockDim.x) {
            const int j = i >> 5, w = i & 31;
            s_dp[j][w] = (d0 + j < E.nd) ? E.dpairs[(size_t)(d0 + j) * 32 + w] : 0u;
        }
        for (int j = threadIdx.x; j < kExhStage; j += blockDim.x) {
            s_ds[j] = (d0 + j < E.nd) ? E.dstat[d0 + j] : make_int4(0, 0, 0, 0);
            s_cs[j] = (d0 + j < E.nd) ? E.dscr[d0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int nj = min(kExhStage, E.nd - d0);
        int j = 0;
        // four domains at a time: four independent dp2a chains, and one
        // branch on their largest screen value (the threshold only rises as
        // the row's best improves, so a largest value below it means nothing
        // to evaluate)
        for (; j + 4 <= nj; j += 4) {
            unsigned acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint4 p = reinterpret_cast<const uint4 *>(s_dp[j + u])[i];
                    acc[u] = dp2a_lo(p.x, aw[2 * i], acc[u]);
                    acc[u] = dp2a_hi(p.y, aw[2 * i], acc[u]);
                    acc[u] = dp2a_lo(p.z, aw[2 * i + 1], acc[u]);
                    acc[u] = dp2a_hi(p.w, aw[2 * i + 1], acc[u]);
                }
            }
            float m = -__int_as_float(0x7f800000);
#pragma unroll
            for (int u = 0; u < 4; ++u) m = fmaxf(m, exh_screen((float)acc[u], (float)sr, s_cs[j + u]));
            if (live && m >= best.thr) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float abs_a;
                    if (exh_screen_abs((float)acc[u], (float)sr, s_cs[j + u], abs_a) >= best.thr && abs_a >= best.thra)
                        exh_exact(best, d0 + j + u, (int)acc[u], sr, s_ds[j + u], E.s_bits);
                }
            }
        }
        for (; j < nj; ++j) {
            unsigned acc = 0;
            const uint4 *q = reinterpret_cast<const uint4 *>(s_dp[j]);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 p = q[i];
                acc = dp2a_lo(p.x, aw[2 * i], acc);
                acc = dp2a_hi(p.y, aw[2 * i], acc);
                acc = dp2a_lo(p.z, aw[2 * i + 1], acc);
                acc = dp2a_hi(p.w, aw[2 * i + 1], acc);
            }
            float abs_a;
            if (live && exh_screen_abs((float)acc, (float)sr, s_cs[j], abs_a) >= best.thr && abs_a >= best.thra)
                exh_exact(best, d0 + j, (int)acc, sr, s_ds[j], E.s_bits);
        }
    }
    if (live) {
        E.row_g[(size_t)r * 8 + t] = best.g;
        E.row_dk[(size_t)r * 8 + t] = make_int2(best.d, best.k);
    }
}

// Combine the isometry rows (and domain segments) of each range and write
// its record (the flat partition: one phase-1 leaf per range, in raster
// order).  Ties: smaller domain index, then smaller isometry.
__global__ void exh_finalize(ExhDesc E) {
    const int ko1 = (1 << E.o_bits) - 1;
    const uint32_t magic = c_lum_magic[E.o_bits];
    const float qscale = c_lum_qscale[E.o_bits];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < E.nr; r += gridDim.x * blockDim.x) {
        long long bg = 0x7fffffffffffffffLL;
        int bd = 0x7fffffff, bt = 0, bk = 0;
        for (int t = 0; t < E.isos; ++t) {
            for (int sg = 0; sg < E.nseg; ++sg) {
                const size_t i = (size_t)sg * E.nr * 8 + (size_t)r * 8 + t;
                const long long g = E.row_g[i];
                const int2 dk = E.row_dk[i];
                if (dk.x >= 0 && exh_better(g, dk.x, bg, bd)) {
                    bg = g;
                    bd = dk.x;
                    bt = t;
                    bk = dk.y;
                }
            }
        }
        const int sr = E.rstat[r].x;
        int dist;
        const int q = best_luminance(sr, 6, ko1, magic, qscale, dist);
        const int x = (r % E.nrx) * kExhB, y = (r / E.nrx) * kExhB;
        const int dx = (bd % E.ndx) * E.step, dy = (bd / E.ndx) * E.step;
        const uint4 w = make_uint4((uint32_t)x | ((uint32_t)y << 16),
                                   1u | (1u << 8) | ((uint32_t)bk << 16) | ((uint32_t)q << 24),
                                   (uint32_t)bt << 24, (uint32_t)dx | ((uint32_t)dy << 16));
        *reinterpret_cast<uint4 *>(E.rec + r) = w;
        E.tile_off[r] = (uint32_t)r;
        E.split[r] = 0u;
        if (r == 0) {
            const unsigned long long fits = (unsigned long long)E.nr * E.nd * E.isos;
            E.tile_off[E.nr] = (uint32_t)E.nr;
            E.info[FIC_INFO_RECORDS] = (uint32_t)E.nr;
            E.info[FIC_INFO_FITS_LO] = (uint32_t)fits;
            E.info[FIC_INFO_FITS_HI] = (uint32_t)(fits >> 32);
        }
    }
}

cudaError_t launch_exh_tc(const ExhDesc &E, uint32_t *err, int *nseg, cudaStream_t st);

// engine 0: tensor cores, 1: CUDA cores.  The stream's info block is
// cleared first; a device timeout of the tensor path leaves its error bit.
cudaError_t launch_exhaustive(const ExhDesc &E, int engine, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(E.info, 0, FIC_INFO_WORDS * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    exh_prep_domains<<<(E.nd_pad * 8 + 255) / 256, 256, 0, st>>>(E);
    stage_mark(st, "exh_prep_domains");
    exh_prep_ranges<<<(E.nr * 64 + 255) / 256, 256, 0, st>>>(E);
    stage_mark(st, "exh_prep_ranges");
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ExhDesc F = E;
    if (engine == 1) {
        const int ranges_per_cta = kExhWarps * 4;
        exh_cuda_kernel<<<(E.nr + ranges_per_cta - 1) / ranges_per_cta, kExhWarps * 32, 0, st>>>(E);
        stage_mark(st, "exh_cuda_kernel");
        e = cudaGetLastError();
        F.nseg = 1;
    } else {
        e = launch_exh_tc(E, E.info + FIC_INFO_ERROR, &F.nseg, st);
    }
    if (e != cudaSuccess) return e;
    exh_finalize<<<(E.nr + 255) / 256, 256, 0, st>>>(F);
    stage_mark(st, "exh_finalize");
    return cudaGetLastError();
}

}  // namespace fic
