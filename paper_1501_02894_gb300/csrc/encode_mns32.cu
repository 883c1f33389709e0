// encode_mns32.cu -- the no-search / MNS quadtree encoder for 32x32 top-level
// blocks (quadtree 32 -> 16 -> 8 -> 4 and its shorter prefixes).
//
// Paper: Section 3 (no-search fit of each range block to the one domain
// centred on it, per-level thresholds, forced acceptance at the last level),
// Sections 3.1-3.3 (MNS phase 2, "Technique 1": four sub-blocks coded with
// the block mean, three mean differences and one contrast bit each, O_4
// from eq. (1)).
//
// Output contract: identical to the slot variant of mns_encode_kernel
// (encode_mns.cu): each strip (here: one top-level block) writes its leaves
// in canonical order to its 64-record slot, its record and fit counts, its
// split mask and the offset of its block inside the strip; pack_kernel
// turns the slots into the stream.
//
// GPU design.  One warp per top-level block.  The block's level-1 domain is
// exactly the 64 x 64 window fetched by TMA, and more than half of the
// blocks of natural images are accepted at level 1, so the level-1 test is
// a path of its own: every lane decimates four 16-pixel units of the window
// (2x2 sums by dp4a), accumulates all five level-1 moments of them on the
// fly against the matching range pixels, and stores the decimated pairs for
// the deeper levels; one reduction per moment and one fit later the block is
// done or goes deeper.  Below level 1 the whole quadtree is evaluated level
// by level without a data-dependent loop: the block sizes are compile-time
// constants, each lane owns an 8 x 4 patch (a 16 x 16 block is 8 lanes, an
// 8 x 8 block 2 lanes, a 4 x 4 block half a lane), and each level computes
// the lanes' blocks' phase-1 fits together with their phase-2 sub-block
// fits against the parent (whose luminance code the same lanes already
// hold), so a parent's phase-2 outcome is one ballot.  The tree is then
// resolved from the pass bits, and leaves are ranked by a 64-bit warp mask.
#include "encode_common.cuh"
#include "pack.cuh"

namespace fic {

namespace m32 {
constexpr int kRawBytes = 64 * 64;  // the TMA window: the level-1 domain
constexpr int kNP = 16;             // words (2x2-sum pairs) per decimated row
constexpr int kWords = 32 * kNP;
constexpr int kPerWarp = kRawBytes + kWords * 4;
static_assert(kPerWarp % 128 == 0, "every warp's TMA window starts 128-byte aligned");
constexpr int kSlotRecs = 64;
}  // namespace m32

// Moments of a lane's 8 x 4 patch against the 8 x 4 decimated domain values
// at column c (even), row rr of the decimated window.  W64: c is a multiple
// of 4, so rows load as 64-bit words.
template <bool W64>
__device__ __forceinline__ void patch_mom(const uint32_t *d4e, int c, int rr, const uint2 (&rw)[4], int &sd,
                                          int &sdd, int &sdr) {
    unsigned a_dr = 0, pk = 0, ql = 0, qh = 0;
    const uint32_t *base = d4e + rr * m32::kNP + (c >> 1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t p0, p1, p2, p3;
        if (W64) {
            const uint2 lo = *reinterpret_cast<const uint2 *>(base + i * m32::kNP);
            const uint2 hi = *reinterpret_cast<const uint2 *>(base + i * m32::kNP + 2);
            p0 = lo.x, p1 = lo.y, p2 = hi.x, p3 = hi.y;
        } else {
            p0 = base[i * m32::kNP], p1 = base[i * m32::kNP + 1];
            p2 = base[i * m32::kNP + 2], p3 = base[i * m32::kNP + 3];
        }
        a_dr = dp2a_lo(p0, rw[i].x, a_dr);
        a_dr = dp2a_hi(p1, rw[i].x, a_dr);
        a_dr = dp2a_lo(p2, rw[i].y, a_dr);
        a_dr = dp2a_hi(p3, rw[i].y, a_dr);
        pk += p0 + p1 + p2 + p3;
        acc_sq(p0, ql, qh);
        acc_sq(p1, ql, qh);
        acc_sq(p2, ql, qh);
        acc_sq(p3, ql, qh);
    }
    sd = (int)((pk & 0xffffu) + (pk >> 16));
    sdd = (int)(ql + (qh << 8));
    sdr = (int)a_dr;
}

// Sum over the lanes xor-related by the given masks (a block's lanes).
template <int M0, int M1 = 0, int M2 = 0>
__device__ __forceinline__ int xsum(int v) {
    v += __shfl_xor_sync(0xffffffffu, v, M0);
    if (M1) v += __shfl_xor_sync(0xffffffffu, v, M1);
    if (M2) v += __shfl_xor_sync(0xffffffffu, v, M2);
    return v;
}

// Codes and pass bit of a phase-1 fit without the collage-error test (a
// last-level block is accepted whatever its error).
__device__ __forceinline__ void fit_codes(int sr, int sd, int sdd, int sdr, int lg2n, int s_bits, int ko1,
                                          uint32_t magic, float qscale, Fit &f) {
    f.sr = sr;
    f.ncdr = ((long long)sdr << lg2n) - (long long)sd * sr;
    f.ncdd = ((long long)sdd << lg2n) - (long long)sd * sd;
    f.k = best_contrast<true>(f.ncdr, f.ncdd, s_bits);
    int bd;
    f.q = best_luminance(sr, lg2n, ko1, magic, qscale, bd);
    f.pass = true;
}

// Round half up of (block mean - Oi) for a sub-block of n = 2^lg2n pixels.
__device__ __forceinline__ int mean_delta(int sr, int Oi, int lg2n) {
    return (2 * (sr - (Oi << lg2n)) + (1 << lg2n)) >> (lg2n + 1);
}

__device__ __forceinline__ uint4 leaf_words(int x, int y, int level, int phase, int k, int q, int d0, int d1, int d2,
                                            int dx, int dy) {
    return make_uint4((uint32_t)x | ((uint32_t)y << 16),
                      (uint32_t)level | ((uint32_t)phase << 8) | ((uint32_t)k << 16) | ((uint32_t)q << 24),
                      ((uint32_t)d0 & 0xffu) | (((uint32_t)d1 & 0xffu) << 8) | (((uint32_t)d2 & 0xffu) << 16),
                      (uint32_t)dx | ((uint32_t)dy << 16));
}

// Geometry of one strip (one top-level block), uniform across the warp.
struct Strip32 {
    int g;        // global strip index (>= total: none)
    int img;      // image of the launch
    int s;        // strip index inside the image
    int sx0, sy0; // top-left pixel of the block
    int rx0, ry0; // top-left pixel of its level-1 domain (= the TMA window)
};

__device__ __forceinline__ Strip32 strip32_of(const int *s_base, const EncDesc *descs, int count, int g,
                                              int total) {
    Strip32 t;
    t.g = g;
    t.img = t.s = t.sx0 = t.sy0 = t.rx0 = t.ry0 = 0;
    if (g >= total) return t;
    t.img = find_image_s(s_base, descs, count, g);
    const EncDesc &E = descs[t.img];
    t.s = g - E.strip_base;
    const int row = t.s / E.tw;  // one block per strip: strips per row = blocks per row
    t.sx0 = (t.s - row * E.tw) * 32;
    t.sy0 = row * 32;
    t.rx0 = clampi(t.sx0 - 16, 0, E.W - 64);
    t.ry0 = clampi(t.sy0 - 16, 0, E.H - 64);
    return t;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 3 : 5)
    mns_encode32_kernel(const EncDesc *__restrict__ descs, int count, int total_strips, uint32_t *__restrict__ status,
                 uint32_t *__restrict__ ticket, int total_chunks, int dyn, int fused) {
    using namespace m32;
    constexpr int PC = 4;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_base[kImgTable];
    __shared__ __align__(8) uint64_t s_bar[NW];
    __shared__ int s_take;  // dynamic schedule: the CTA's strips handed out so far
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    uint8_t *const smem_a = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    uint8_t *const raw = smem_a + warp * kPerWarp;
    if (threadIdx.x == 0) s_take = 0;
    uint32_t *const d4e = reinterpret_cast<uint32_t *>(raw + kRawBytes);
    uint64_t *const bar = &s_bar[warp];
    const int pr = lane >> 2, pc = lane & 3;
    // the pack kernel may start as this grid's CTAs retire (it waits for the
    // grid's completion before it reads anything written here)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (count <= kImgTable)
        for (int i = threadIdx.x; i < count; i += blockDim.x) s_base[i] = descs[i].strip_base;
    if (!fused)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total_chunks; i += gridDim.x * blockDim.x)
            status[i] = 0u;
    uint32_t *chunk_done = status + total_chunks + 1;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](const Strip32 &t) {
        if (lane == 0 && t.g < total_strips) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (uint32_t)kRawBytes);
            tma_load_2d(raw, descs[t.img].map, t.rx0, t.ry0, bar);
        }
    };
    // Schedule.  Static: warp w takes strips w, w + gstep, ...  With `dyn`
    // the CTA owns strips blockIdx.x, blockIdx.x + gridDim.x, ... (spread
    // over the batch) and its warps take them one by one from a shared-memory
    // counter, one strip ahead: a warp whose strips were accepted at level 1
    // takes more of them, and the CTA's warps finish together.  (A global
    // ticket counter was slower: thousands of warps contend for one word.)
    const int gstep = gridDim.x * NW;
    int g0, g_next, tk = 0;  // tk (lane 0): the CTA-local index of the strip after the next one
    if (dyn) {
        if (lane == 0) {
            g0 = blockIdx.x + gridDim.x * atomicAdd(&s_take, 1);
            tk = atomicAdd(&s_take, 1);
        }
        g0 = __shfl_sync(FULL, g0, 0);
    } else {
        g0 = blockIdx.x * NW + warp;
    }
    g_next = g0 + gstep;
    Strip32 cur = strip32_of(s_base, descs, count, g0, total_strips);
    issue(cur);
    uint32_t phase = 0;

    while (cur.g < total_strips) {
        if (dyn) {
            g_next = blockIdx.x + gridDim.x * __shfl_sync(FULL, tk, 0);
            if (lane == 0) tk = atomicAdd(&s_take, 1);
        }
        const EncDesc &D = descs[cur.img];
        const int W = D.W, H = D.H;
        const int sx0 = cur.sx0, sy0 = cur.sy0, rx0 = cur.rx0, ry0 = cur.ry0;
        const int s = cur.s;
        const int L = D.L, s_bits = D.s_bits;
        const int ko1 = (1 << D.o_bits) - 1;
        const uint32_t magic = c_lum_magic[D.o_bits];
        const float qscale = c_lum_qscale[D.o_bits];
        const bool ph2 = (D.mode == FIC_MNS) && D.phase2;
        const int top = (sy0 >> 5) * D.tw + (sx0 >> 5);
        const int ox = sx0 - rx0, oy = sy0 - ry0;  // range block inside the window
        // the strip after this one: its window is fetched once this one's is consumed
        const Strip32 nxt = strip32_of(s_base, descs, count, g_next, total_strips);
        const int g_after = g_next + gstep;  // static schedule

        const bool arrived = mbar_wait(bar, phase, kMbarLimit);
        phase ^= 1u;
        if (!__all_sync(FULL, arrived)) {
            if (lane == 0) D.stats[s] = make_uint2(0u, 0x80000000u);  // no records, error flag
            mbar_wait(bar, phase ^ 1u, kMbarLimit);                   // let a late copy land
            return;
        }

        // ---- level 1 (Section 3): the lane's four units of 8 decimated
        // values (rows r, columns 8cu..8cu+7) against the range pixels they
        // meet; the decimated pairs are kept for the deeper levels
        uint2 rw[4];  // the lane's 8 x 4 range patch (deeper levels)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            rw[i] = *reinterpret_cast<const uint2 *>(raw + (oy + 4 * pr + i) * 64 + ox + 8 * pc);
        unsigned a_dr = 0, pk = 0, ql = 0, qh = 0, s_r = 0, s_rr = 0;
        {
            const int cu = lane & 3;
            // lanes 4-7 of every eight read their row pair the other way round
            // (2x2 sums do not care), so one load touches all 32 banks
            const int swap = (lane >> 2) & 1;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int r = (lane >> 2) + 8 * t;
                const uint8_t *p = raw + (2 * r + swap) * 64 + 16 * cu;
                const uint4 A = *reinterpret_cast<const uint4 *>(p);
                const uint4 B = *reinterpret_cast<const uint4 *>(p + (swap ? -64 : 64));
                const uint2 R = *reinterpret_cast<const uint2 *>(raw + (oy + r) * 64 + ox + 8 * cu);
                uint4 P;
                P.x = pair2x2(A.x, B.x);
                P.y = pair2x2(A.y, B.y);
                P.z = pair2x2(A.z, B.z);
                P.w = pair2x2(A.w, B.w);
                *reinterpret_cast<uint4 *>(d4e + r * kNP + 4 * cu) = P;
                a_dr = dp2a_lo(P.x, R.x, a_dr);
                a_dr = dp2a_hi(P.y, R.x, a_dr);
                a_dr = dp2a_lo(P.z, R.y, a_dr);
                a_dr = dp2a_hi(P.w, R.y, a_dr);
                pk += P.x + P.y + P.z + P.w;
                acc_sq(P.x, ql, qh);
                acc_sq(P.y, ql, qh);
                acc_sq(P.z, ql, qh);
                acc_sq(P.w, ql, qh);
                s_r = __dp4a(R.x, 0x01010101u, __dp4a(R.y, 0x01010101u, s_r));
                s_rr = __dp4a(R.x, R.x, __dp4a(R.y, R.y, s_rr));
            }
        }
        __syncwarp();
        // the window has been read: fetch the next strip's
        issue(nxt);
        Fit f1;
        {
            const int sr = (int)__reduce_add_sync(FULL, s_r);
            const int srr = (int)__reduce_add_sync(FULL, s_rr);
            const int sd = (int)__reduce_add_sync(FULL, (pk & 0xffffu) + (pk >> 16));
            const int sdd = (int)__reduce_add_sync(FULL, ql + (qh << 8));
            const int sdr = (int)__reduce_add_sync(FULL, a_dr);
            fit_phase1(sr, srr, sd, sdd, sdr, 10, s_bits, ko1, magic, qscale, D.t2q[0] << 30, f1);
        }
        fic_record *slot = D.slots + (size_t)s * kSlotRecs;
        unsigned cnt, ftot;
        if (f1.pass || L == 1) {
            // accepted at level 1 (or the only level): one record
            if (lane == 0) {
                *reinterpret_cast<uint4 *>(slot) = leaf_words(sx0, sy0, 1, 1, f1.k, f1.q, 0, 0, 0, rx0, ry0);
                D.split[top] = 0u;
                D.tile_off[top] = 0u;
            }
            cnt = 1;
            ftot = 1;
        } else {
            const int bmin = D.bmin;
            const int lgbmin = 31 - __clz(bmin);
            int sr_h[2] = {0, 0}, srr_h[2] = {0, 0};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                sr_h[0] += (int)__dp4a(rw[i].x, 0x01010101u, 0u);
                sr_h[1] += (int)__dp4a(rw[i].y, 0x01010101u, 0u);
                srr_h[0] += (int)__dp4a(rw[i].x, rw[i].x, 0u);
                srr_h[1] += (int)__dp4a(rw[i].y, rw[i].y, 0u);
            }
            const int c_base = rx0 >> 1, r_base = ry0 >> 1;
            unsigned fits = lane == 0 ? (ph2 ? 5u : 1u) : 0u;  // the level-1 fit (+ its phase-2 attempt)
            uint32_t splitbits = 0;
            uint4 leafA = make_uint4(0u, 0u, 0u, 0u), leafB = leafA;
            int posA = -1, posB = -1;

            // ---- level 2: 16 x 16 blocks (8 lanes each), children of the level-1 block
            const int bx2 = pc >> 1, by2 = pr >> 2;
            const int x2 = sx0 + 16 * bx2, y2 = sy0 + 16 * by2;
            const int dx2 = centred_origin(x2, 16, W), dy2 = centred_origin(y2, 16, H);
            Fit f2;
            bool pass2 = false;
            int q2 = 0, k2 = 0;
            bool p2_1 = false;  // phase 2 of the level-1 block
            int sb1 = 0, dl1[3] = {0, 0, 0};
            {
                int sd, sdd, sdr;
                patch_mom<true>(d4e, (dx2 >> 1) - c_base + 8 * pc - 16 * bx2, (dy2 >> 1) - r_base + 4 * pr - 16 * by2,
                                rw, sd, sdd, sdr);
                const int sr = xsum<1, 4, 8>(sr_h[0] + sr_h[1]);
                const int srr = xsum<1, 4, 8>(srr_h[0] + srr_h[1]);
                sd = xsum<1, 4, 8>(sd);
                sdd = xsum<1, 4, 8>(sdd);
                sdr = xsum<1, 4, 8>(sdr);
                if (L == 2) fit_codes(sr, sd, sdd, sdr, 8, s_bits, ko1, magic, qscale, f2);
                else fit_phase1(sr, srr, sd, sdd, sdr, 8, s_bits, ko1, magic, qscale, D.t2q[1] << 26, f2);
                f2.ncrr = ((long long)srr << 8) - (long long)sr * sr;
                pass2 = f2.pass;
                q2 = f2.q;
                k2 = f2.k;
                if (ph2) {
                    // sub-block of the level-1 block (Sections 3.1-3.2)
                    const int Oi = lum(f1.q, ko1, magic);
                    const int dlt = mean_delta(sr, Oi, 8);
                    const int d_tl = __shfl_sync(FULL, dlt, 0), d_tr = __shfl_sync(FULL, dlt, 2);
                    const int d_bl = __shfl_sync(FULL, dlt, 16);
                    const int kk = bx2 | (by2 << 1);
                    const int O = kk == 3 ? Oi - (d_tl + d_tr + d_bl) : Oi + dlt;  // eq. (1)
                    int bit;
                    const bool ok = fit_phase2_sub(f2, 8, O, phase2_code(1, 0), phase2_code(1, 1),
                                                   D.t2q[0] << 26, bit);
                    const bool inr = dlt <= 15 && dlt >= -15;
                    p2_1 = __all_sync(FULL, ok && inr);
                    const uint32_t bb = __ballot_sync(FULL, bit);
                    sb1 = (int)((bb & 1u) | ((bb >> 1) & 2u) | ((bb >> 14) & 4u) | ((bb >> 15) & 8u));
                    dl1[0] = d_tl;
                    dl1[1] = d_tr;
                    dl1[2] = d_bl;
                }
            }
            // Below level 1 every lane takes part in every level that any block
            // of the strip reaches (warp-uniform conditions only: the levels'
            // shuffles and ballots involve the whole warp); each lane then
            // keeps what belongs to the blocks it represents.
            const bool leaf1 = p2_1;
            if (leaf1) {
                if (lane == 0) {
                    leafA = leaf_words(sx0, sy0, 1, 2, sb1, f1.q, dl1[0], dl1[1], dl1[2], rx0, ry0);
                    posA = 0;
                }
            } else {
                if (lane == 0) splitbits |= 1u;
                const bool rep2 = (pc & 1) == 0 && (pr & 3) == 0;
                const int z2 = bx2 | (by2 << 1);
                const int pos2 = (int)morton3((16 * bx2) >> lgbmin, (16 * by2) >> lgbmin);
                if (rep2) fits += (ph2 && L > 2 && !pass2) ? 5u : 1u;
                // ---- level 3: 8 x 8 blocks (2 lanes each), if a level-2 block failed phase 1
                bool pass3 = true, p2_2 = false;
                int q3 = 0, k3 = 0, sb2 = 0, dl2[3] = {0, 0, 0};
                const int by3 = pr >> 1;
                const int x3 = sx0 + 8 * pc, y3 = sy0 + 8 * by3;
                const int dx3 = centred_origin(x3, 8, W), dy3 = centred_origin(y3, 8, H);
                Fit f3;
                const bool lev3 = L > 2 && __any_sync(FULL, !pass2);
                if (lev3) {
                    int sd, sdd, sdr;
                    patch_mom<false>(d4e, (dx3 >> 1) - c_base, (dy3 >> 1) - r_base + 4 * pr - 8 * by3, rw, sd, sdd,
                                     sdr);
                    const int sr = xsum<4>(sr_h[0] + sr_h[1]);
                    const int srr = xsum<4>(srr_h[0] + srr_h[1]);
                    sd = xsum<4>(sd);
                    sdd = xsum<4>(sdd);
                    sdr = xsum<4>(sdr);
                    if (L == 3) fit_codes(sr, sd, sdd, sdr, 6, s_bits, ko1, magic, qscale, f3);
                    else fit_phase1(sr, srr, sd, sdd, sdr, 6, s_bits, ko1, magic, qscale, D.t2q[2] << 22, f3);
                    f3.ncrr = ((long long)srr << 6) - (long long)sr * sr;
                    pass3 = f3.pass;
                    q3 = f3.q;
                    k3 = f3.k;
                    if (ph2) {
                        // sub-block of its level-2 block
                        const int Oi = lum(q2, ko1, magic);
                        const int dlt = mean_delta(sr, Oi, 6);
                        const int base = lane & 0x12;  // the level-2 block's top-left lane
                        const int d_tl = __shfl_sync(FULL, dlt, base), d_tr = __shfl_sync(FULL, dlt, base + 1);
                        const int d_bl = __shfl_sync(FULL, dlt, base + 8);
                        const int kk = (pc & 1) | ((by3 & 1) << 1);
                        const int O = kk == 3 ? Oi - (d_tl + d_tr + d_bl) : Oi + dlt;  // eq. (1)
                        int bit;
                        const bool ok = fit_phase2_sub(f3, 6, O, phase2_code(2, 0), phase2_code(2, 1),
                                                       D.t2q[1] << 22, bit);
                        const bool inr = dlt <= 31 && dlt >= -31;
                        const uint32_t okb = __ballot_sync(FULL, ok && inr);
                        const uint32_t gm = 0x3333u << base;  // the level-2 block's eight lanes
                        p2_2 = !pass2 && (okb & gm) == gm;
                        const uint32_t bb = __ballot_sync(FULL, bit) >> base;
                        sb2 = (int)((bb & 3u) | ((bb >> 6) & 0xCu));
                        dl2[0] = d_tl;
                        dl2[1] = d_tr;
                        dl2[2] = d_bl;
                    }
                }
                const bool leaf2 = pass2 || p2_2 || L == 2;
                if (leaf2 && rep2) {
                    leafA = p2_2 ? leaf_words(x2, y2, 2, 2, sb2, q2, dl2[0], dl2[1], dl2[2], dx2, dy2)
                                 : leaf_words(x2, y2, 2, 1, k2, q2, 0, 0, 0, dx2, dy2);
                    posA = pos2;
                }
                if (!leaf2 && rep2) splitbits |= 1u << (1 + z2);
                const bool reach3 = !leaf2;
                const bool rep3 = reach3 && (pr & 1) == 0;
                const int z3 = (int)morton3(pc, by3);
                const int pos3 = (int)morton3((8 * pc) >> lgbmin, (8 * by3) >> lgbmin);
                if (rep3) fits += (ph2 && L > 3 && !pass3) ? 5u : 1u;
                // ---- level 4: 4 x 4 blocks (the lane's two halves; always the last
                // level), if a level-3 block that is reached failed phase 1
                bool p2_3 = false;
                int sb3 = 0, dl3[3] = {0, 0, 0};
                Fit f4[2];
                const bool lev4 = L > 3 && __any_sync(FULL, reach3 && !pass3);
                if (lev4) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int x4 = sx0 + 8 * pc + 4 * h, y4 = sy0 + 4 * pr;
                        int sd, sdd, sdr;
                        half_moments<m32::kNP>(d4e, (centred_origin(x4, 4, W) >> 1) - c_base,
                                               (centred_origin(y4, 4, H) >> 1) - r_base, rw, h, sd, sdd, sdr);
                        fit_codes(sr_h[h], sd, sdd, sdr, 4, s_bits, ko1, magic, qscale, f4[h]);
                        f4[h].ncrr = ((long long)srr_h[h] << 4) - (long long)sr_h[h] * sr_h[h];
                    }
                    if (ph2) {
                        // sub-blocks of the lane pair's 8 x 8 block: TL, TR in
                        // the top lane, BL, BR in the bottom lane
                        const int Oi = lum(q3, ko1, magic);
                        const int e0 = mean_delta(sr_h[0], Oi, 4), e1 = mean_delta(sr_h[1], Oi, 4);
                        const bool topl = (pr & 1) == 0;
                        const int o0 = __shfl_xor_sync(FULL, e0, PC), o1 = __shfl_xor_sync(FULL, e1, PC);
                        const int d_tl = topl ? e0 : o0, d_tr = topl ? e1 : o1, d_bl = topl ? o0 : e0;
                        const int c0 = phase2_code(3, 0), c1 = phase2_code(3, 1);
                        const long long thr = D.t2q[2] << 18;
                        int b0, b1;
                        const bool ok0 = fit_phase2_sub(f4[0], 4, Oi + e0, c0, c1, thr, b0);
                        const int O1 = topl ? Oi + e1 : Oi - (d_tl + d_tr + d_bl);  // eq. (1) for BR
                        const bool ok1 = fit_phase2_sub(f4[1], 4, O1, c0, c1, thr, b1);
                        const bool inr = e0 <= 31 && e0 >= -31 && e1 <= 31 && e1 >= -31;
                        const bool okl = ok0 && ok1 && inr;
                        const bool oko = __shfl_xor_sync(FULL, okl ? 1 : 0, PC) != 0;
                        p2_3 = !pass3 && okl && oko;
                        const int my = b0 | (b1 << 1);
                        const int other = __shfl_xor_sync(FULL, my, PC);
                        sb3 = topl ? (my | (other << 2)) : (other | (my << 2));
                        dl3[0] = d_tl;
                        dl3[1] = d_tr;
                        dl3[2] = d_bl;
                    }
                }
                const bool leaf3 = reach3 && (pass3 || p2_3 || L == 3);
                if (leaf3 && rep3) {
                    leafA = p2_3 ? leaf_words(x3, y3, 3, 2, sb3, q3, dl3[0], dl3[1], dl3[2], dx3, dy3)
                                 : leaf_words(x3, y3, 3, 1, k3, q3, 0, 0, 0, dx3, dy3);
                    posA = pos3;
                }
                if (rep3 && !leaf3) splitbits |= 1u << (5 + z3);
                if (reach3 && !leaf3) {
                    fits += 2u;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int x4 = sx0 + 8 * pc + 4 * h, y4 = sy0 + 4 * pr;
                        const uint4 w = leaf_words(x4, y4, 4, 1, f4[h].k, f4[h].q, 0, 0, 0, centred_origin(x4, 4, W),
                                                   centred_origin(y4, 4, H));
                        const int pos = (int)morton3((8 * pc + 4 * h) >> 2, pr);
                        if (h == 0) {
                            leafA = w;
                            posA = pos;
                        } else {
                            leafB = w;
                            posB = pos;
                        }
                    }
                }
            }
            // ---- canonical ranks and the strip's slot
            unsigned long long mine = 0;
            if (posA >= 0) mine |= 1ull << posA;
            if (posB >= 0) mine |= 1ull << posB;
            const uint32_t mlo = __reduce_or_sync(FULL, (uint32_t)mine);
            const uint32_t mhi = __reduce_or_sync(FULL, (uint32_t)(mine >> 32));
            const unsigned long long mask = ((unsigned long long)mhi << 32) | mlo;
            cnt = (unsigned)__popcll(mask);
            if (posA >= 0)
                *reinterpret_cast<uint4 *>(slot + __popcll(mask & ((1ull << posA) - 1ull))) = leafA;
            if (posB >= 0)
                *reinterpret_cast<uint4 *>(slot + __popcll(mask & ((1ull << posB) - 1ull))) = leafB;
            ftot = __reduce_add_sync(FULL, fits);
            splitbits = __reduce_or_sync(FULL, splitbits);
            if (lane == 0) {
                D.split[top] = splitbits;
                D.tile_off[top] = 0u;
            }
        }
        if (lane == 0) D.stats[s] = make_uint2(cnt, ftot & 0x7fffffffu);
        if (fused) {
            // the warp that finishes a chunk's last strip packs the chunk
            __syncwarp();
            __threadfence();
            const int cl = s >> 5;
            uint32_t done = 0;
            if (lane == 0) done = atomicAdd(chunk_done + D.chunk_base + cl, 1u) + 1u;
            done = __shfl_sync(FULL, done, 0);
            if ((int)done == min(32, D.nstrips - cl * 32)) {
                __threadfence();
                pack_chunk_warp(D, cl, status, lane);
            }
        }
        __syncwarp();
        cur = nxt;
        g_next = g_after;
    }
}

size_t mns32_smem_bytes(int nw) { return (size_t)nw * m32::kPerWarp + 128; }

template <int NW>
static cudaError_t launch_m32(const EncDesc *descs, int count, int total_strips, uint32_t *status, uint32_t *ticket,
                              int total_chunks, int ctas_per_sm, int dyn, int fused, cudaStream_t st) {
    static KernelSlots ks;
    int sms = 0, per = 0;
    const size_t smem = mns32_smem_bytes(NW);
    cudaError_t e = kernel_slots(ks, (const void *)mns_encode32_kernel<NW>, NW * 32, smem, sms, per);
    if (e != cudaSuccess) return e;
    const int k = ctas_per_sm > 0 && ctas_per_sm < per ? ctas_per_sm : per;
    const int need = (total_strips + NW - 1) / NW;
    const int grid = need < sms * k ? need : sms * k;
    mns_encode32_kernel<NW><<<grid, NW * 32, smem, st>>>(descs, count, total_strips, status, ticket, total_chunks, dyn,
                                                  fused);
    stage_mark(st, "mns_encode_kernel");
    return cudaGetLastError();
}

cudaError_t launch_mns32_slots(const EncDesc *d_descs, int count, int total_strips, int total_chunks,
                               uint32_t *pack_status, uint32_t *ticket, const EncTune &tune, cudaStream_t st) {
    const int dyn = tune.dynamic ? 1 : 0, fused = tune.fused_pack ? 1 : 0;
    return tune.warps == 4
               ? launch_m32<4>(d_descs, count, total_strips, pack_status, ticket, total_chunks, tune.ctas_per_sm, dyn,
                               fused, st)
               : launch_m32<8>(d_descs, count, total_strips, pack_status, ticket, total_chunks, tune.ctas_per_sm, dyn,
                               fused, st);
}

}  // namespace fic
