// encode_local.cu -- quadtree encoder with local domain search.
//
// Paper, Section 2: instead of the single centred domain, every range is
// compared with the domains around it -- here the centred domain shifted by
// (ox, oy), ox, oy in [-R, R] with step S (R = 16, S = 4 gives the 81
// candidates of Section 2), skipping candidates that leave the image, no
// isometries.  The best candidate is the one with the smallest collage
// error; ties go to the first candidate in (oy, ox) raster order.  The
// quadtree is the one of Section 3 (threshold per level, forced acceptance
// at the last level) without the MNS phase 2.
//
// GPU design: the strip/patch geometry of the MNS encoder, with the staged
// decimated window enlarged by R on every side.  At each level every lane
// scans all candidates of its block (or of its two 4x4 blocks): the moments
// of its patch by dp2a, group totals by xor shuffles, the exact s-part
// minimum in int64, a running best.  The range sums and the luminance code
// do not depend on the candidate and are computed once per block.  Leaves go
// to the strip's slot; pack_kernel compacts the stream.
#include "encode_common.cuh"

namespace fic {

constexpr int kLWarps = 8;
constexpr int kLSlot = 64;
constexpr int kLocalRmax = 16;

template <int BMAX>
struct LGeom {
    static constexpr int SW = 1024 / BMAX;
    static constexpr int PC = SW / 8;
    static constexpr int PR = BMAX / 4;
    static constexpr int TOPS = SW / BMAX;
    static constexpr int ROWS = BMAX + kLocalRmax;  // decimated rows of the window (max)
    static constexpr int UPR = BMAX == 32 ? 8 : 16;  // 16-pixel units per window row (max, power of two)
    static constexpr int NP = BMAX == 32 ? 32 : (BMAX == 16 ? 36 : 52);  // words per decimated row
    static constexpr int WORDS = ROWS * NP;
};

// Window staging for the local search: `rows` decimated rows, `upr` units.
template <int BMAX>
__device__ __forceinline__ void stage_local(const uint8_t *__restrict__ img, int W, int ry0, int ax0, int rows, int upr,
                                            uint32_t *d4e, int lane) {
    using G = LGeom<BMAX>;
    for (int u = lane; u < G::ROWS * G::UPR; u += 32) {
        const int r = u / G::UPR, cu = u % G::UPR;
        if (r < rows && cu < upr) {
            const uint8_t *p = img + (size_t)(ry0 + 2 * r) * W + ax0 + 16 * cu;
            const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
            const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p + W));
            uint4 o;
            o.x = d4_pair(a.x, b.x);
            o.y = d4_pair(a.y, b.y);
            o.z = d4_pair(a.z, b.z);
            o.w = d4_pair(a.w, b.w);
            *reinterpret_cast<uint4 *>(d4e + r * G::NP + 4 * cu) = o;
        }
    }
}

// Moments of `words` range words per row (1 or 2, starting at word w0 of
// the patch row) against the decimated values at column c (any parity) and
// row rr of the window.
template <int NP>
__device__ __forceinline__ void lmoments(const uint32_t *d4e, int c, int rr, const uint2 *rw, int w0, int words,
                                         int &sd, int &sdd, int &sdr) {
    unsigned a_dr = 0, pk = 0, ql = 0, qh = 0;
    const uint32_t *base = d4e + rr * NP + (c >> 1);
    const bool odd = c & 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            if (w >= words) break;
            const uint32_t *q = base + i * NP + 2 * w;
            uint32_t p0 = q[0], p1 = q[1];
            if (odd) {
                const uint32_t p2 = q[2];
                p0 = __funnelshift_r(p0, p1, 16);
                p1 = __funnelshift_r(p1, p2, 16);
            }
            const uint32_t r = (w0 + w) ? rw[i].y : rw[i].x;
            a_dr = dp2a_lo(p0, r, a_dr);
            a_dr = dp2a_hi(p1, r, a_dr);
            pk += p0 + p1;
            acc_sq(p0, ql, qh);
            acc_sq(p1, ql, qh);
        }
    }
    sd = (int)((pk & 0xffffu) + (pk >> 16));
    sdd = (int)(ql + (qh << 8));
    sdr = (int)a_dr;
}

// Best candidate of one block so far.
struct LBest {
    long long g;  // s-part of the error, c^2 nCdd - 1024 c nCdr
    int k, dx, dy;
    int tried;
};

template <int BMAX>
__global__ void __launch_bounds__(kLWarps * 32, 2)
    local_encode_kernel(const EncDesc *__restrict__ descs, int count, int total_strips,
                        uint32_t *__restrict__ pack_status, int total_chunks) {
    using G = LGeom<BMAX>;
    constexpr int PC = G::PC, NP = G::NP;
    extern __shared__ __align__(16) uint32_t lsmem[];
    __shared__ int s_base[kImgTable];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *d4e = lsmem + warp * G::WORDS;
    const int pr = lane / PC, pc = lane % PC;
    const unsigned FULL = 0xffffffffu;
    if (count <= kImgTable)
        for (int i = threadIdx.x; i < count; i += blockDim.x) s_base[i] = descs[i].strip_base;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total_chunks; i += gridDim.x * blockDim.x)
        pack_status[i] = 0u;
    __syncthreads();
    const int gstep = gridDim.x * kLWarps;
    for (int g = blockIdx.x * kLWarps + warp; g < total_strips; g += gstep) {
        const int img = find_image_s(s_base, descs, count, g);
        const EncDesc &D = descs[img];
        const int W = D.W, H = D.H, tw = D.tw;
        const int s = g - D.strip_base;
        const int row = s / D.spr, sc = s - row * D.spr;
        const int sy0 = row * BMAX, sx0 = sc * G::SW;
        const int top0 = row * tw + sc * G::TOPS;
        const int nvalid = min(G::TOPS, tw - sc * G::TOPS);
        const int lane_top = (8 * pc) / BMAX;
        const bool valid = lane_top < nvalid;
        const int L = D.L, bmin = D.bmin, s_bits = D.s_bits;
        const int ko1 = (1 << D.o_bits) - 1;
        const uint32_t magic = c_lum_magic[D.o_bits];
        const float qscale = c_lum_qscale[D.o_bits];
        const int R = D.local_radius, S = D.local_step;

        // ---- window: the level-1 domains of the strip, widened by R
        const int rx0 = clampi(sx0 - BMAX / 2, 0, W - 2 * BMAX);
        const int xl = sx0 + (nvalid - 1) * BMAX;
        const int rx1 = clampi(xl - BMAX / 2, 0, W - 2 * BMAX) + 2 * BMAX;
        const int ax0 = max(rx0 - R, 0) & ~15, ax1 = (min(rx1 + R, W) + 15) & ~15;
        const int ry1 = clampi(sy0 - BMAX / 2, 0, H - 2 * BMAX);
        const int ry0 = max(ry1 - R, 0) & ~1;
        const int ryend = min(ry1 + 2 * BMAX + R, H);
        const int c_base = ax0 >> 1, r_base = ry0 >> 1;
        __syncwarp();
        stage_local<BMAX>(D.img, W, ry0, ax0, (ryend - ry0) >> 1, (ax1 - ax0) >> 4, d4e, lane);
        uint2 rw[4];
        int sr_h[2] = {0, 0}, srr_h[2] = {0, 0};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            rw[i] = valid ? __ldg(reinterpret_cast<const uint2 *>(D.img + (size_t)(sy0 + 4 * pr + i) * W + sx0 + 8 * pc))
                          : make_uint2(0u, 0u);
            sr_h[0] += (int)__dp4a(rw[i].x, 0x01010101u, 0u);
            sr_h[1] += (int)__dp4a(rw[i].y, 0x01010101u, 0u);
            srr_h[0] += (int)__dp4a(rw[i].x, rw[i].x, 0u);
            srr_h[1] += (int)__dp4a(rw[i].y, rw[i].y, 0u);
        }
        __syncwarp();

        Leaf leaf[2];
        leaf[0].pos = -1;
        leaf[1].pos = -1;
        uint32_t splitbits = 0;
        unsigned fits = 0;
        // sides are powers of two: divisions by them are shifts
        const int lgbmin = 31 - __clz(bmin);
        const int cpt_side = BMAX >> lgbmin, cpt = cpt_side * cpt_side;
        bool act = valid;
        int B = BMAX, lgB = 31 - __clz(BMAX);
        for (int j = 1; j <= L; ++j, B >>= 1, --lgB) {
            if (!__any_sync(FULL, act)) break;
            const int lg2n = 2 * (31 - __clz(B));
            const long long thr = D.t2q[j - 1] << (2 * lg2n + 10);
            const int nh = (B >= 8) ? 1 : 2;  // blocks of the lane at this level
            const int gx = B >= 8 ? B / 8 : 1, gy = B >= 8 ? B / 4 : 1;
            int bxs[2], bys[2];
            LBest best[2];
            long long ncrr[2];
            int sr[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (B >= 8) {
                    bxs[h] = (8 * pc) >> lgB;
                } else {
                    bxs[h] = 2 * pc + h;
                }
                bys[h] = (4 * pr) >> lgB;
                best[h].g = 0x7fffffffffffffffLL;
                best[h].k = 0;
                best[h].dx = best[h].dy = 0;
                best[h].tried = 0;
                const int srl = B >= 8 ? sr_h[0] + sr_h[1] : sr_h[h];
                const int srrl = B >= 8 ? srr_h[0] + srr_h[1] : srr_h[h];
                sr[h] = group_sum<PC>(srl, gx, gy);
                const int srr = group_sum<PC>(srrl, gx, gy);
                ncrr[h] = ((long long)srr << lg2n) - (long long)sr[h] * sr[h];
            }
            // ---- scan the candidates
            for (int oy = -R; oy <= R; oy += S) {
                for (int ox = -R; ox <= R; ox += S) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h >= nh) break;
                        const int xa = sx0 + bxs[h] * B, ya = sy0 + bys[h] * B;
                        const int dx = centred_origin(xa, B, W) + ox, dy = centred_origin(ya, B, H) + oy;
                        const bool in = act && dx >= 0 && dy >= 0 && dx + 2 * B <= W && dy + 2 * B <= H;
                        const int u0 = B >= 8 ? 8 * pc - bxs[h] * B : 0;
                        const int v0 = 4 * pr - bys[h] * B;
                        int sd = 0, sdd = 0, sdr = 0;
                        if (in)
                            lmoments<NP>(d4e, (dx >> 1) + u0 - c_base, (dy >> 1) + v0 - r_base, rw, B >= 8 ? 0 : h,
                                         B >= 8 ? 2 : 1, sd, sdd, sdr);
                        sd = group_sum<PC>(sd, gx, gy);
                        sdd = group_sum<PC>(sdd, gx, gy);
                        sdr = group_sum<PC>(sdr, gx, gy);
                        if (in) {
                            const long long ncdr = ((long long)sdr << lg2n) - (long long)sd * sr[h];
                            const long long ncdd = ((long long)sdd << lg2n) - (long long)sd * sd;
                            const int k = best_contrast(ncdr, ncdd, s_bits);
                            const long long c = contrast_code(k, s_bits);
                            const long long gval = c * c * ncdd - 1024LL * c * ncdr;
                            if (gval < best[h].g) {
                                best[h].g = gval;
                                best[h].k = k;
                                best[h].dx = dx;
                                best[h].dy = dy;
                            }
                            best[h].tried += 1;
                        }
                    }
                }
            }
            // ---- decisions of the level
            bool split_any = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h >= nh) break;
                const int xa = sx0 + bxs[h] * B, ya = sy0 + bys[h] * B;
                const int u0 = B >= 8 ? 8 * pc - bxs[h] * B : 0;
                const int v0 = 4 * pr - bys[h] * B;
                const bool rep = act && u0 == 0 && v0 == 0;
                if (rep) fits += (unsigned)best[h].tried;
                // luminance code: the level nearest the block mean
                const int n = 1 << lg2n;
                int q0 = __float2int_rn((float)sr[h] * qscale / (float)n);
                q0 = clampi(q0, 0, ko1);
                int bq = q0, bd = 0x7fffffff;
#pragma unroll
                for (int dq = -1; dq <= 1; ++dq) {
                    const int q = q0 + dq;
                    if (q < 0 || q > ko1) continue;
                    const int d = abs(sr[h] - (lum(q, ko1, magic) << lg2n));
                    if (d < bd) {
                        bd = d;
                        bq = q;
                    }
                }
                const long long E = 262144LL * ncrr[h] + best[h].g + 262144LL * (long long)bd * bd;
                const bool pass = (j == L) || E < thr;
                const int tx = bxs[h] * B - lane_top * BMAX, ty = bys[h] * B;
                if (rep && pass) {
                    const int pos = lane_top * cpt + (int)morton3(tx >> lgbmin, ty >> lgbmin);
                    make_leaf(leaf[B >= 8 ? 0 : h], xa, ya, j, 1, best[h].k, bq, 0, 0, 0, best[h].dx, best[h].dy, pos);
                }
                const bool split = act && !pass;
                if (rep && split) {
                    const uint32_t z = morton3(tx >> lgB, ty >> lgB);
                    splitbits |= 1u << (((1u << (2 * (j - 1))) - 1) / 3 + z);
                }
                split_any = split_any || split;
            }
            act = split_any;  // the lane's block at the next level is a child of a split block
        }

        // ---- ranks and slot stores (compacted later by pack_kernel)
        unsigned long long mine = 0;
        if (leaf[0].pos >= 0) mine |= 1ull << leaf[0].pos;
        if (leaf[1].pos >= 0) mine |= 1ull << leaf[1].pos;
        const uint32_t mlo = __reduce_or_sync(FULL, (uint32_t)mine);
        const uint32_t mhi = __reduce_or_sync(FULL, (uint32_t)(mine >> 32));
        const unsigned long long mask = ((unsigned long long)mhi << 32) | mlo;
        const int cnt = __popcll(mask);
        fic_record *slot = D.slots + (size_t)s * kLSlot;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (leaf[h].pos < 0) continue;
            const int idx = __popcll(mask & ((1ull << leaf[h].pos) - 1ull));
            *reinterpret_cast<uint4 *>(slot + idx) = make_uint4(leaf[h].w0, leaf[h].w1, leaf[h].w2, leaf[h].w3);
        }
        const unsigned ftot = __reduce_add_sync(FULL, fits);
        splitbits = group_or<PC>(splitbits, BMAX / 8, BMAX / 4);
        if (valid && (8 * pc) % BMAX == 0 && pr == 0) {
            D.split[top0 + lane_top] = splitbits;
            D.tile_off[top0 + lane_top] = (uint32_t)__popcll(mask & ((1ull << (lane_top * cpt)) - 1ull));
        }
        if (lane == 0) D.stats[s] = make_uint2((uint32_t)cnt, ftot & 0x7fffffffu);
    }
}

size_t local_smem_bytes(int bmax) {
    const int words = bmax == 32 ? LGeom<32>::WORDS : (bmax == 16 ? LGeom<16>::WORDS : LGeom<8>::WORDS);
    return (size_t)kLWarps * words * sizeof(uint32_t);
}

template <int BMAX>
static cudaError_t llaunch_t(const EncDesc *descs, int count, int total_strips, uint32_t *pack_status,
                             int total_chunks, cudaStream_t st) {
    static KernelSlots ks;
    const size_t smem = local_smem_bytes(BMAX);
    int sms = 0, per = 0;
    cudaError_t e = kernel_slots(ks, (const void *)local_encode_kernel<BMAX>, kLWarps * 32, smem, sms, per);
    if (e != cudaSuccess) return e;
    const int need = (total_strips + kLWarps - 1) / kLWarps;
    const int grid = need < sms * per ? need : sms * per;
    local_encode_kernel<BMAX><<<grid, kLWarps * 32, smem, st>>>(descs, count, total_strips, pack_status, total_chunks);
    stage_mark(st, "local_encode_kernel");
    return cudaGetLastError();
}

cudaError_t launch_pack(const EncDesc *d_descs, int count, int total_chunks, uint32_t *pack_status,
                        uint32_t *ticket, cudaStream_t st);

cudaError_t launch_local_encode(int bmax, const EncDesc *d_descs, int count, int total_strips, int total_chunks,
                                uint32_t *pack_status, cudaStream_t st) {
    cudaError_t e;
    switch (bmax) {
    case 32: e = llaunch_t<32>(d_descs, count, total_strips, pack_status, total_chunks, st); break;
    case 16: e = llaunch_t<16>(d_descs, count, total_strips, pack_status, total_chunks, st); break;
    case 8: e = llaunch_t<8>(d_descs, count, total_strips, pack_status, total_chunks, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return launch_pack(d_descs, count, total_chunks, pack_status, nullptr, st);
}

}  // namespace fic
