// decode.cu -- iterated fixed-point decoder.
//
// The paper relies on the iterated-function-system property of the stored
// transforms (Section 1: decoding is fast because the attractor is reached
// by iterating the transforms from any start) but does not describe a
// decoder.  This one starts from mid-grey and applies every transform to the
// previous iterate (Jacobi):
//     x'(u,v) = clamp(floor((512 n O + c (n d4(u,v) - Sd4) + 256 n) / (512 n)), 0, 255)
// i.e. round-half-up of O + s (d - mean d) with c = 128 s and d4 the 2x2 sum
// of the domain.  512 n is a power of two, so the division is a shift.
//
// GPU design: the same strip / patch geometry as the encoder (one warp per
// 1024-pixel strip, lane = 8x4 patch).  Per launch (= one iteration) a warp
// stages its strip's records and the decimated window of the previous
// iterate in shared memory, finds the transform covering each 4x4 half-patch
// by binary search over the canonical keys, reduces Sd4 over the lanes of
// each transform with xor shuffles and writes 8 pixels per row with one
// 8-byte store.  Domains that do not lie in the staged window (local and
// exhaustive search, isometries) are read from global memory instead.
#include "fic_internal.cuh"

namespace fic {

template <int BMAX>
struct DGeom {
    static constexpr int SW = 1024 / BMAX;
    static constexpr int PC = SW / 8;
    static constexpr int PR = BMAX / 4;
    static constexpr int TOPS = SW / BMAX;
    static constexpr int NP = BMAX == 32 ? 16 : (BMAX == 16 ? 24 : 40);
    static constexpr int WORDS = BMAX * NP;
    static constexpr int PER_WARP = 2 * WORDS + 64 * 4 + 16;  // d4e, d4o, 64 records, 64 keys
};

constexpr int kDecWarps = 8;

__device__ __forceinline__ uint32_t dmorton3(uint32_t x, uint32_t y) {
    uint32_t z = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) z |= (((x >> b) & 1u) << (2 * b)) | (((y >> b) & 1u) << (2 * b + 1));
    return z;
}

// Source element of an isometry (column u, row v of a B x B block):
// 0 identity, 1 quarter turn clockwise, 2 half turn, 3 quarter turn
// anticlockwise, 4 left-right mirror, 5 up-down mirror, 6 transpose,
// 7 anti-transpose.
__device__ __forceinline__ void iso_src(int iso, int B, int u, int v, int &su, int &sv) {
    const int m = B - 1;
    switch (iso) {
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

template <int BMAX>
__global__ void __launch_bounds__(kDecWarps * 32)
    decode_iter_kernel(const DecDesc *__restrict__ descs, int count, int total_strips, int src_sel,
                       int first) {
    using G = DGeom<BMAX>;
    constexpr int PC = G::PC, NP = G::NP;
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *d4e = smem + warp * G::PER_WARP;
    uint32_t *d4o = d4e + G::WORDS;
    uint4 *recs = reinterpret_cast<uint4 *>(d4o + G::WORDS);
    uint8_t *keys = reinterpret_cast<uint8_t *>(recs + 64);
    const int pr = lane / PC, pc = lane % PC;
    const unsigned FULL = 0xffffffffu;
    const int gwarps = gridDim.x * kDecWarps;

    for (int g = blockIdx.x * kDecWarps + warp; g < total_strips; g += gwarps) {
        const int img = find_image(descs, count, g);
        const DecDesc &D = descs[img];
        const int W = D.W, H = D.H, tw = D.tw;
        const int s = g - D.strip_base;
        const int row = s / D.spr, sc = s % D.spr;
        const int sy0 = row * BMAX, sx0 = sc * G::SW;
        const int top0 = row * tw + sc * G::TOPS;
        const int nvalid = min(G::TOPS, tw - sc * G::TOPS);
        const int lane_top = (8 * pc) / BMAX;
        const bool valid = lane_top < nvalid;
        const int bmin = D.bmin;
        const int cpt_side = BMAX / bmin, cpt = cpt_side * cpt_side;
        const uint8_t *src = D.buf[src_sel];
        uint8_t *dst = D.buf[src_sel ^ 1];
        const bool centred = (D.mode == FIC_NOSEARCH || D.mode == FIC_MNS);
        const int ko1 = (1 << D.o_bits) - 1;

        // ---- records of the strip (at most 64) with their canonical keys
        const uint32_t rbeg = D.tile_off[top0], rend = D.tile_off[top0 + nvalid];
        const int nrec = (int)(rend - rbeg);
        __syncwarp();
        for (int i = lane; i < nrec && i < 64; i += 32) {
            const uint4 r = *reinterpret_cast<const uint4 *>(D.rec + rbeg + i);
            recs[i] = r;
            const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16);
            const int lt = x / BMAX - sc * G::TOPS;
            keys[i] = (uint8_t)(lt * cpt + (int)dmorton3((x % BMAX) / bmin, (y % BMAX) / bmin));
        }
        // ---- decimated window of the previous iterate
        int c_base = 0, r_base = 0;
        if (!first && centred) {
            const int rx0 = clampi(sx0 - BMAX / 2, 0, W - 2 * BMAX);
            const int xl = sx0 + (nvalid - 1) * BMAX;
            const int rx1 = clampi(xl - BMAX / 2, 0, W - 2 * BMAX) + 2 * BMAX;
            const int ax0 = rx0 & ~15, ax1 = (rx1 + 15) & ~15;
            const int ry0 = clampi(sy0 - BMAX / 2, 0, H - 2 * BMAX);
            c_base = ax0 >> 1;
            r_base = ry0 >> 1;
            const int upr = (ax1 - ax0) >> 4, npairs = upr * 4;
            for (int u = lane; u < BMAX * upr; u += 32) {
                const int r = u / upr, cu = u - r * upr;
                const uint8_t *p = src + (size_t)(ry0 + 2 * r) * W + ax0 + 16 * cu;
                const uint4 a = *reinterpret_cast<const uint4 *>(p);
                const uint4 b = *reinterpret_cast<const uint4 *>(p + W);
                uint4 o;
                o.x = d4_pair(a.x, b.x);
                o.y = d4_pair(a.y, b.y);
                o.z = d4_pair(a.z, b.z);
                o.w = d4_pair(a.w, b.w);
                *reinterpret_cast<uint4 *>(d4e + r * NP + 4 * cu) = o;
            }
            __syncwarp();
            for (int i = lane; i < BMAX * npairs; i += 32) {
                const int r = i / npairs, c = i - r * npairs;
                const uint32_t a = d4e[r * NP + c];
                const uint32_t b = (c + 1 < npairs) ? d4e[r * NP + c + 1] : 0u;
                d4o[r * NP + c] = __byte_perm(a, b, 0x5432);
            }
        }
        __syncwarp();

        // ---- transform of each half-patch
        int t_x[2], t_y[2], t_lg[2], t_dx[2], t_dy[2], t_c[2], t_O[2], t_iso[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            t_x[h] = t_y[h] = t_dx[h] = t_dy[h] = t_c[h] = t_O[h] = t_iso[h] = 0;
            t_lg[h] = 2;
            if (!valid || nrec <= 0) continue;
            const int px = 8 * pc + 4 * h, py = 4 * pr;  // in strip
            const int tx = px - lane_top * BMAX;
            const int key = lane_top * cpt + (int)dmorton3(tx / bmin, py / bmin);
            int lo = 0, hi = min(nrec, 64) - 1;
            while (lo < hi) {  // last record with keys[i] <= key
                const int mid = (lo + hi + 1) >> 1;
                if ((int)keys[mid] <= key) lo = mid;
                else hi = mid - 1;
            }
            const uint4 r = recs[lo];
            const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16);
            const int level = (int)(r.y & 0xffu), phase = (int)((r.y >> 8) & 0xffu);
            const int k = (int)((r.y >> 16) & 0xffu), q = (int)(r.y >> 24);
            const int B = BMAX >> (level - 1);
            const int Oi = (510 * q + ko1) / (2 * ko1);
            if (phase == 1) {
                t_x[h] = x;
                t_y[h] = y;
                t_lg[h] = 31 - __clz(B);
                t_dx[h] = (int)(r.w & 0xffffu);
                t_dy[h] = (int)(r.w >> 16);
                t_c[h] = contrast_code(k, D.s_bits);
                t_O[h] = Oi;
                t_iso[h] = (int)(r.z >> 24);
            } else {
                const int hb = B >> 1;
                const int ax = sx0 + px, ay = sy0 + py;
                const int sb = (ax - x >= hb ? 1 : 0) | (ay - y >= hb ? 2 : 0);
                const int d0 = (int)(int8_t)(r.z & 0xffu), d1 = (int)(int8_t)((r.z >> 8) & 0xffu),
                          d2 = (int)(int8_t)((r.z >> 16) & 0xffu);
                const int O0 = Oi + d0, O1 = Oi + d1, O2 = Oi + d2;
                const int O3 = 4 * Oi - (O0 + O1 + O2);  // eq. (1)
                const int Os = sb == 0 ? O0 : (sb == 1 ? O1 : (sb == 2 ? O2 : O3));
                t_x[h] = x + (sb & 1) * hb;
                t_y[h] = y + (sb >> 1) * hb;
                t_lg[h] = 31 - __clz(hb);
                t_dx[h] = centred_origin(t_x[h], hb, W);
                t_dy[h] = centred_origin(t_y[h], hb, H);
                t_c[h] = phase2_code(level, (k >> sb) & 1);
                t_O[h] = Os;
                t_iso[h] = 0;
            }
        }

        // ---- decimated domain values of the half-patches (16 each) and partial Sd4
        uint32_t dv[2][4][2];  // [half][row][pair]
        int part[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int i = 0; i < 4; ++i) dv[h][i][0] = dv[h][i][1] = 0x02000200u;  // 512, 512
            if (!valid || first) continue;
            const int ax = sx0 + 8 * pc + 4 * h, ay = sy0 + 4 * pr;
            const int u0 = ax - t_x[h], v0 = ay - t_y[h];
            if (centred && t_iso[h] == 0) {
                const int c = (t_dx[h] >> 1) + u0 - c_base, rr = (t_dy[h] >> 1) + v0 - r_base;
                const uint32_t *base = (c & 1) ? d4o + rr * NP + ((c - 1) >> 1) : d4e + rr * NP + (c >> 1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    dv[h][i][0] = base[i * NP];
                    dv[h][i][1] = base[i * NP + 1];
                }
            } else {
                const int B = 1 << t_lg[h];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint32_t vals[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        int su, sv;
                        iso_src(t_iso[h], B, u0 + e, v0 + i, su, sv);
                        const uint8_t *p = src + (size_t)(t_dy[h] + 2 * sv) * W + t_dx[h] + 2 * su;
                        vals[e] = (uint32_t)p[0] + p[1] + p[W] + p[W + 1];
                    }
                    dv[h][i][0] = vals[0] | (vals[1] << 16);
                    dv[h][i][1] = vals[2] | (vals[3] << 16);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t s2 = dv[h][i][0] + dv[h][i][1];
                part[h] += (int)((s2 & 0xffffu) + (s2 >> 16));
            }
        }
        // ---- Sd4 per transform: halves of one lane first (side >= 8), then the
        // lane group of the transform; every lane runs the same shuffles
        int sd4[2];
        {
            const bool big = t_lg[0] >= 3;  // a transform of side >= 8 covers both halves
            const int B = 1 << t_lg[0];
            const int gx = big ? B / 8 : 1, gy = big ? B / 4 : 1;
            int v = part[0] + part[1];
#pragma unroll
            for (int m = 1; m < 4; m <<= 1) {
                const int o = __shfl_xor_sync(FULL, v, m);
                if (m < gx) v += o;
            }
#pragma unroll
            for (int m = 1; m < 8; m <<= 1) {
                const int o = __shfl_xor_sync(FULL, v, (m * PC) & 31);
                if (m < gy && m * PC < 32) v += o;
            }
            sd4[0] = big ? v : part[0];
            sd4[1] = big ? v : part[1];
        }
        if (first) {
            sd4[0] = 512 << (2 * t_lg[0]);
            sd4[1] = 512 << (2 * t_lg[1]);
        }

        // ---- output pixels
        if (valid) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t wout[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int lg2n = 2 * t_lg[h];
                    const int n = 1 << lg2n;
                    const int base = t_O[h] * (1 << (9 + lg2n)) + (n << 8) - t_c[h] * sd4[h];
                    uint32_t w = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t pair = dv[h][i][e >> 1];
                        const int d = (int)((e & 1) ? (pair >> 16) : (pair & 0xffffu));
                        int p = (base + t_c[h] * (d << lg2n)) >> (9 + lg2n);
                        p = clampi(p, 0, 255);
                        w |= (uint32_t)p << (8 * e);
                    }
                    wout[h] = w;
                }
                *reinterpret_cast<uint2 *>(dst + (size_t)(sy0 + 4 * pr + i) * W + sx0 + 8 * pc) =
                    make_uint2(wout[0], wout[1]);
            }
        }
    }
}

size_t decode_smem_bytes(int bmax) {
    int words = bmax == 32 ? DGeom<32>::PER_WARP : (bmax == 16 ? DGeom<16>::PER_WARP : DGeom<8>::PER_WARP);
    return (size_t)kDecWarps * words * sizeof(uint32_t);
}

template <int BMAX>
static cudaError_t dlaunch_t(const DecDesc *descs, int count, int total_strips, int src_sel, int first,
                             cudaStream_t st) {
    static int grid_cache = 0;
    const size_t smem = decode_smem_bytes(BMAX);
    if (grid_cache == 0) {
        cudaError_t e = cudaFuncSetAttribute(decode_iter_kernel<BMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, decode_iter_kernel<BMAX>, kDecWarps * 32, smem);
        grid_cache = sms * (per > 0 ? per : 1);
    }
    const int need = (total_strips + kDecWarps - 1) / kDecWarps;
    const int grid = need < grid_cache ? need : grid_cache;
    decode_iter_kernel<BMAX><<<grid, kDecWarps * 32, smem, st>>>(descs, count, total_strips, src_sel, first);
    return cudaGetLastError();
}

cudaError_t launch_decode_iter(int bmax, const DecDesc *d_descs, int count, int total_strips, int src_sel,
                               int first, cudaStream_t st) {
    switch (bmax) {
    case 32: return dlaunch_t<32>(d_descs, count, total_strips, src_sel, first, st);
    case 16: return dlaunch_t<16>(d_descs, count, total_strips, src_sel, first, st);
    case 8: return dlaunch_t<8>(d_descs, count, total_strips, src_sel, first, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fic
