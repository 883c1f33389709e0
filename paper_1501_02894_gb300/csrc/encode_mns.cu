// encode_mns.cu -- fused quadtree encoder for the no-search and MNS modes.
//
// Paper: Salarian, Mohamadinia, Rasekhi, "A Modified No Search Algorithm for
// Fractal Image Compression".  Section 3 (no-search quadtree with per-level
// thresholds, forced acceptance at the last level), Sections 3.1-3.2 (MNS
// phase 2, "Technique 1"), Section 3.3 (stored parameters, eq. (1)).
//
// GPU design.  One warp owns a strip of 1024 pixels: bmax rows by 1024/bmax
// columns, i.e. 1, 4 or 16 consecutive top-level blocks of one block row
// (consecutive in the stream's raster order).  Everything the quadtree of
// those blocks can touch lies inside the union of their level-1 domains, so
// the warp decimates that window once into shared memory (2x2 sums packed as
// 16-bit pairs; windows that start at an odd column are realigned with funnel
// shifts) and then runs all levels out of registers and shared memory:
//   * lane l owns an 8x4-pixel patch of the strip; every quadtree block of
//     side >= 8 is a power-of-two group of lanes, a 4x4 block is half a patch;
//   * moments per level: sum r*d4 and sum d4^2 by dp2a on packed operands,
//     sums by packed adds, group totals by xor-shuffle butterflies;
//   * the phase-1 code choice, the collage error and the phase-2 test are
//     exact int64 integer arithmetic, evaluated redundantly by every lane of
//     a block (lock-step, no divergence between blocks);
//   * a level is skipped as soon as no block of the strip needs it;
//   * leaves are ranked in the canonical order by a 64-bit warp mask and
//     written with one 16-byte store each, into the strip's slot of the
//     workspace; pack_kernel (pack.cu) compacts the slots into the stream.
// The grid is persistent and strips are assigned statically; each warp's
// next window is fetched by TMA (cp.async.bulk.tensor + mbarrier) while the
// current strip is encoded.  A second variant (used by the allocation-free
// entry point) takes strips from an atomic ticket in stream order and packs
// the stream in place with a decoupled look-back over the strips (bounded
// spin), so its only scratch is one status word per strip.
#include "encode_common.cuh"
#include "pack.cuh"

namespace fic {

template <int BMAX>
struct Geom {
    static constexpr int SW = 1024 / BMAX;  // strip width, pixels
    static constexpr int PC = SW / 8;       // patches per patch row
    static constexpr int PR = BMAX / 4;     // patch rows
    static constexpr int TOPS = SW / BMAX;  // top-level blocks per strip
    // words per row of each packed decimated array (pairs of 2x2 sums)
    static constexpr int NP = BMAX == 32 ? 16 : (BMAX == 16 ? 24 : 40);
    static constexpr int WORDS = BMAX * NP;  // one packed decimated window per warp
};

constexpr int kWarps = 8;
constexpr int kSlotRecords = 64;  // records a 1024-pixel strip can hold (4x4 leaves)
constexpr uint32_t kAgg = 1u << 30, kIncl = 2u << 30, kValMask = (1u << 30) - 1;

// SLOTS = true: every strip writes its records to a fixed slot of the
//   workspace and pack_kernel then compacts the canonical stream, so warps
//   need no ordering: strips are assigned statically (grid stride) or, with
//   `dyn`, taken from an atomic ticket (pack_kernel resets it).
// SLOTS = false: strips come from an atomic ticket in stream order and the
//   stream is packed in place by a decoupled look-back (needs only one status
//   word per strip of scratch).
// NW warps per CTA: 8 (registers capped at 80 for 3 CTAs = 24 warps per SM)
// or 4 (up to 128 registers, no spills, 4 CTAs = 16 warps per SM).
// MIN2 (slot variant only): the quadtree goes down to 2 x 2 blocks (bmin 2);
//   their domains (4 x 4 pixels, odd origins inside the image) are read from
//   the raw window, which is then kept until the strip is done, and the up to
//   256 leaves of a strip are staged in shared memory by canonical position.
template <int BMAX, bool SLOTS, int NW, bool MIN2 = false>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 3 : 4)
    mns_encode_kernel(const EncDesc *__restrict__ descs, int count, int total_strips,
                      uint32_t *__restrict__ status, uint32_t *__restrict__ ticket, int total_chunks, int dyn,
                      int fused) {
    using G = Geom<BMAX>;
    constexpr int PC = G::PC, NP = G::NP;
    constexpr int UPR = BMAX == 32 ? 4 : (BMAX == 16 ? 8 : 16);
    using BX = WinBox<BMAX>;
    constexpr int RAWB = BX::W * BX::H;  // bytes of the staged window (a multiple of 128)
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_base[kImgTable];
    __shared__ __align__(8) uint64_t s_bar[NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // TMA destinations need 128-byte alignment in the shared window
    uint8_t *const smem_a = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    // staged leaves + their position mask (8 words, padded: every warp's
    // window must start 128-byte aligned for its TMA copies)
    constexpr int STAGE = MIN2 ? 256 * 16 + 128 : 0;
    static_assert((RAWB + G::WORDS * 4 + STAGE) % 128 == 0, "per-warp shared memory keeps TMA alignment");
    uint8_t *raw = smem_a + warp * (RAWB + G::WORDS * 4 + STAGE);
    uint32_t *d4e = reinterpret_cast<uint32_t *>(raw + RAWB);
    uint4 *lrec = reinterpret_cast<uint4 *>(raw + RAWB + G::WORDS * 4);
    uint32_t *lmask = reinterpret_cast<uint32_t *>(lrec + (MIN2 ? 256 : 0));
    uint64_t *bar = &s_bar[warp];
    const int pr = lane / PC, pc = lane % PC;
    const unsigned FULL = 0xffffffffu;
    // the pack kernel may be scheduled as this grid's CTAs retire (it waits
    // for this grid's completion before reading anything it wrote)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (count <= kImgTable)
        for (int i = threadIdx.x; i < count; i += blockDim.x) s_base[i] = descs[i].strip_base;
    if (SLOTS && !fused) {
        // clear the pack kernel's look-back words (it runs after this kernel;
        // fused packing needs them zero before the launch instead)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total_chunks; i += gridDim.x * blockDim.x)
            status[i] = 0u;
    }
    // fused packing: per-chunk count of finished strips, after the ticket
    uint32_t *chunk_done = status + total_chunks + 1;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Window of strip gi: one TMA box load into `raw`, signalled on `bar`.
    // Issued by lane 0 only; a strip's window is fetched while the previous
    // strip is being encoded.
    auto issue_window = [&](int gi) {
        const int im = find_image_s(s_base, descs, count, gi);
        const EncDesc &E = descs[im];
        const int si = gi - E.strip_base;
        const int rw_ = si / E.spr, sc_ = si - rw_ * E.spr;
        const int sy = rw_ * BMAX, sx = sc_ * G::SW;
        const int nv = min(G::TOPS, E.tw - sc_ * G::TOPS);
        const int x0 = clampi(sx - BMAX / 2, 0, E.W - 2 * BMAX) & ~15;
        const int y0 = clampi(sy - BMAX / 2, 0, E.H - 2 * BMAX);
        (void)nv;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (uint32_t)(E.boxw * BX::H));
        tma_load_2d(raw, E.map, x0, y0, bar);
    };

    uint32_t phase = 0;
    const int gstep = gridDim.x * NW;
    const bool ticketed = !SLOTS || dyn;
    int g = 0, g_next = 0;
    if (!ticketed) {
        g = blockIdx.x * NW + warp;
        g_next = g + gstep;
        if (lane == 0 && g < total_strips) issue_window(g);
    } else {
        if (lane == 0) {
            g = (int)atomicAdd(ticket, 1u);
            if (g < total_strips) issue_window(g);
            g_next = (int)atomicAdd(ticket, 1u);
        }
        g = __shfl_sync(FULL, g, 0);
    }
    for (;;) {
        if (g >= total_strips) break;
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
        const bool ph2 = (D.mode == FIC_MNS) && D.phase2;
        const int pitch = D.boxw;
        const int rx0 = clampi(sx0 - BMAX / 2, 0, W - 2 * BMAX);
        const int xl = sx0 + (nvalid - 1) * BMAX;
        const int rx1 = clampi(xl - BMAX / 2, 0, W - 2 * BMAX) + 2 * BMAX;
        const int ax0 = rx0 & ~15, ax1 = (rx1 + 15) & ~15;
        const int ry0 = clampi(sy0 - BMAX / 2, 0, H - 2 * BMAX);
        const int c_base = ax0 >> 1, r_base = ry0 >> 1;

        // ---- wait for the window (bounded), then the range pixels and the
        // decimated pairs, both read from the staged window
        const bool arrived = mbar_wait(bar, phase, kMbarLimit);
        phase ^= 1u;
        if (!__all_sync(FULL, arrived)) {
            if (lane == 0) {
                if (SLOTS) D.stats[s] = make_uint2(0u, 0x80000000u);  // no records, error flag
                else raise_error(D.info, FIC_DEVERR_TIMEOUT);
            }
            mbar_wait(bar, phase ^ 1u, kMbarLimit);  // let a late copy land before leaving
            return;
        }
        uint2 rw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            rw[i] = valid ? *reinterpret_cast<const uint2 *>(raw + (sy0 + 4 * pr + i - ry0) * pitch + sx0 + 8 * pc - ax0)
                          : make_uint2(0u, 0u);
        stage_window_smem<BMAX, UPR, NP>(raw, pitch, (ax1 - ax0) >> 4, d4e, lane);
        if (MIN2 && lane < 8) lmask[lane] = 0u;
        __syncwarp();
        // the window buffer is free (MIN2: once the 2 x 2 blocks are done):
        // fetch the next strip's window now
        if (!MIN2 && lane == 0) {
            if (g_next < total_strips) issue_window(g_next);
        }
        int g_after = g_next + gstep;
        if (ticketed && lane == 0) g_after = (int)atomicAdd(ticket, 1u);
        int sr_h[2] = {0, 0}, srr_h[2] = {0, 0};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            sr_h[0] += (int)__dp4a(rw[i].x, 0x01010101u, 0u);
            sr_h[1] += (int)__dp4a(rw[i].y, 0x01010101u, 0u);
            srr_h[0] += (int)__dp4a(rw[i].x, rw[i].x, 0u);
            srr_h[1] += (int)__dp4a(rw[i].y, rw[i].y, 0u);
        }

        // ---- quadtree, level by level
        Leaf leaf[2];
        leaf[0].pos = -1;
        leaf[1].pos = -1;
        uint32_t splitbits = 0;
        unsigned fits = 0;
        // sides are powers of two: divisions by them are shifts (a division by
        // a run-time value would cost a few dozen instructions)
        const int lgbmin = 31 - __clz(bmin);
        const int cpt_side = BMAX >> lgbmin;  // bmin cells per top side
        const int cpt = cpt_side * cpt_side;
        bool act = valid;
        Code cur;       // phase-1 codes of the lane's level-j block (side >= 8)
        Code cur4[2];   // the two 4x4 blocks of the last level
        Fit ch[2];      // children's fits (ch[0] for side >= 8, both for the 4x4 halves)
        int B = BMAX, lgB = 31 - __clz(BMAX);
        {
            const int gx = B / 8, gy = B / 4;
            const int bx = (8 * pc) >> lgB, by = (4 * pr) >> lgB;
            const int xa = sx0 + bx * B, ya = sy0 + by * B;
            const int dxa = centred_origin(xa, B, W), dya = centred_origin(ya, B, H);
            const int u0 = 8 * pc - bx * B, v0 = 4 * pr - by * B;
            int sd = 0, sdd = 0, sdr = 0;
            if (valid) patch_moments<NP>(d4e, (dxa >> 1) + u0 - c_base, (dya >> 1) + v0 - r_base, rw, sd, sdd, sdr);
            const int sr = group_sum<PC>(sr_h[0] + sr_h[1], gx, gy);
            const int srr = group_sum<PC>(srr_h[0] + srr_h[1], gx, gy);
            sd = group_sum<PC>(sd, gx, gy);
            sdd = group_sum<PC>(sdd, gx, gy);
            sdr = group_sum<PC>(sdr, gx, gy);
            const int lg2n = 2 * (31 - __clz(B));
            Fit f;
            fit_phase1(sr, srr, sd, sdd, sdr, lg2n, s_bits, ko1, magic, qscale, D.t2q[0] << (2 * lg2n + 10), f);
            cur.k = f.k;
            cur.q = f.q;
            cur.pass = f.pass;
        }
        for (int j = 1; j <= L; ++j, B >>= 1, --lgB) {
            if (B >= 8) {
                const int gx = B / 8, gy = B / 4;
                const int bx = (8 * pc) >> lgB, by = (4 * pr) >> lgB;
                const int xa = sx0 + bx * B, ya = sy0 + by * B;
                const int u0 = 8 * pc - bx * B, v0 = 4 * pr - by * B;
                const bool rep = act && u0 == 0 && v0 == 0;
                if (rep) fits += 1;
                const int tx = bx * B - lane_top * BMAX, ty = by * B;  // inside the top block
                const int pos = lane_top * cpt + (int)morton3(tx >> lgbmin, ty >> lgbmin);
                const int dxa = centred_origin(xa, B, W), dya = centred_origin(ya, B, H);
                if (j == L) {
                    if (rep) make_leaf(leaf[0], xa, ya, j, 1, cur.k, cur.q, 0, 0, 0, dxa, dya, pos);
                    break;
                }
                if (rep && cur.pass) make_leaf(leaf[0], xa, ya, j, 1, cur.k, cur.q, 0, 0, 0, dxa, dya, pos);
                const bool need = act && !cur.pass;
                if (!__any_sync(FULL, need)) break;
                // ---- level j+1: moments and phase 1 of the children
                const int Bc = B >> 1;
                const int lg2c = 2 * (31 - __clz(Bc));
                const long long thr_c = D.t2q[j] << (2 * lg2c + 10);     // children as level-(j+1) blocks
                const long long thr_p2 = D.t2q[j - 1] << (2 * lg2c + 10); // sub-blocks coded at level j
                if (Bc >= 8) {
                    const int cgx = Bc / 8, cgy = Bc / 4;
                    const int cbx = (8 * pc) >> (lgB - 1), cby = (4 * pr) >> (lgB - 1);
                    const int cxa = sx0 + cbx * Bc, cya = sy0 + cby * Bc;
                    const int cdx = centred_origin(cxa, Bc, W), cdy = centred_origin(cya, Bc, H);
                    const int cu0 = 8 * pc - cbx * Bc, cv0 = 4 * pr - cby * Bc;
                    int sd = 0, sdd = 0, sdr = 0;
                    if (valid)
                        patch_moments<NP>(d4e, (cdx >> 1) + cu0 - c_base, (cdy >> 1) + cv0 - r_base, rw, sd, sdd, sdr);
                    const int sr = group_sum<PC>(sr_h[0] + sr_h[1], cgx, cgy);
                    const int srr = group_sum<PC>(srr_h[0] + srr_h[1], cgx, cgy);
                    sd = group_sum<PC>(sd, cgx, cgy);
                    sdd = group_sum<PC>(sdd, cgx, cgy);
                    sdr = group_sum<PC>(sdr, cgx, cgy);
                    fit_phase1(sr, srr, sd, sdd, sdr, lg2c, s_bits, ko1, magic, qscale, thr_c, ch[0]);
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int cxa = sx0 + 8 * pc + 4 * h, cya = sy0 + 4 * pr;
                        const int cdx = centred_origin(cxa, 4, W), cdy = centred_origin(cya, 4, H);
                        int sd = 0, sdd = 0, sdr = 0;
                        if (valid) half_moments<NP>(d4e, (cdx >> 1) - c_base, (cdy >> 1) - r_base, rw, h, sd, sdd, sdr);
                        fit_phase1(sr_h[h], srr_h[h], sd, sdd, sdr, 4, s_bits, ko1, magic, qscale, thr_c, ch[h]);
                    }
                }
                // ---- phase 2 of the level-j blocks that failed phase 1 (Sections 3.1-3.3)
                bool p2 = false;
                int d[4] = {0, 0, 0, 0};
                int sbits = 0;
                if (ph2) {
                    if (rep && need) fits += 4;
                    const int lg2n4 = lg2c;
                    const int Oi = lum(cur.q, ko1, magic);
                    int csr[4];
                    if (Bc >= 8) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int cbx = 2 * bx + (k & 1), cby = 2 * by + (k >> 1);
                            const int src = (cby * Bc / 4) * PC + (cbx * Bc / 8);
                            csr[k] = __shfl_sync(FULL, ch[0].sr, src & 31);
                        }
                    } else {
                        // B == 8: the top patch holds TL, TR, the bottom patch BL, BR
                        const int o0 = __shfl_xor_sync(FULL, ch[0].sr, PC);
                        const int o1 = __shfl_xor_sync(FULL, ch[1].sr, PC);
                        const bool top = (pr & 1) == 0;
                        csr[0] = top ? ch[0].sr : o0;
                        csr[1] = top ? ch[1].sr : o1;
                        csr[2] = top ? o0 : ch[0].sr;
                        csr[3] = top ? o1 : ch[1].sr;
                    }
                    const int dmax = (j == 1) ? 15 : 31;
                    bool inrange = true;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        // round half up of (mean_k - O_i)
                        d[k] = (2 * (csr[k] - (Oi << lg2n4)) + (1 << lg2n4)) >> (lg2n4 + 1);
                        inrange = inrange && d[k] <= dmax && d[k] >= -dmax;
                    }
                    int O[4];
                    O[0] = Oi + d[0];
                    O[1] = Oi + d[1];
                    O[2] = Oi + d[2];
                    O[3] = 4 * Oi - (O[0] + O[1] + O[2]);  // eq. (1)
                    const int c0 = phase2_code(j, 0), c1 = phase2_code(j, 1);
                    // the sub-blocks' fits: against their own centred domains
                    // (the children's phase-1 moments) or, with the other
                    // reading, against the quadrants of this block's domain
                    // (the children's domain moments are replaced in place:
                    // only their codes and pass bits are used later)
                    Fit (&sub)[2] = ch;
                    if (D.phase2_domain) {
                        if (Bc >= 8) {
                            int sd = 0, sdd = 0, sdr = 0;
                            if (valid)
                                patch_moments<NP>(d4e, (dxa >> 1) + u0 - c_base, (dya >> 1) + v0 - r_base, rw, sd, sdd,
                                                  sdr);
                            const int cgx = Bc / 8, cgy = Bc / 4;
                            sd = group_sum<PC>(sd, cgx, cgy);
                            sdd = group_sum<PC>(sdd, cgx, cgy);
                            sdr = group_sum<PC>(sdr, cgx, cgy);
                            sub[0].ncdr = ((long long)sdr << lg2n4) - (long long)sd * sub[0].sr;
                            sub[0].ncdd = ((long long)sdd << lg2n4) - (long long)sd * sd;
                        } else {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                int sd = 0, sdd = 0, sdr = 0;
                                if (valid)
                                    half_moments<NP>(d4e, (dxa >> 1) + u0 + 4 * h - c_base, (dya >> 1) + v0 - r_base, rw,
                                                     h, sd, sdd, sdr);
                                sub[h].ncdr = ((long long)sdr << 4) - (long long)sd * sub[h].sr;
                                sub[h].ncdd = ((long long)sdd << 4) - (long long)sd * sd;
                            }
                        }
                    }
                    bool ok_lane;
                    if (Bc >= 8) {
                        const int cbx = (8 * pc) >> (lgB - 1), cby = (4 * pr) >> (lgB - 1);
                        const int kk = (cbx & 1) | ((cby & 1) << 1);
                        int bit;
                        // (selects: an indexed array would live in local memory)
                        const int Ok = kk == 0 ? O[0] : (kk == 1 ? O[1] : (kk == 2 ? O[2] : O[3]));
                        ok_lane = fit_phase2_sub(sub[0], lg2n4, Ok, c0, c1, thr_p2, bit);
                        const uint32_t bits = __ballot_sync(FULL, bit);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int cbx2 = 2 * bx + (k & 1), cby2 = 2 * by + (k >> 1);
                            const int src = (cby2 * Bc / 4) * PC + (cbx2 * Bc / 8);
                            sbits |= (int)((bits >> (src & 31)) & 1u) << k;
                        }
                    } else {
                        const bool top = (pr & 1) == 0;
                        int b0, b1;
                        const bool ok0 = fit_phase2_sub(sub[0], 4, top ? O[0] : O[2], c0, c1, thr_p2, b0);
                        const bool ok1 = fit_phase2_sub(sub[1], 4, top ? O[1] : O[3], c0, c1, thr_p2, b1);
                        ok_lane = ok0 && ok1;
                        const int my = b0 | (b1 << 1);
                        const int other = __shfl_xor_sync(FULL, my, PC);
                        sbits = top ? (my | (other << 2)) : (other | (my << 2));
                    }
                    const uint32_t okb = __ballot_sync(FULL, ok_lane);
                    const uint32_t gm = group_mask<PC>(pc, pr, gx, gy);
                    p2 = need && inrange && ((okb & gm) == gm);
                }
                if (rep && p2) make_leaf(leaf[0], xa, ya, j, 2, sbits, cur.q, d[0], d[1], d[2], dxa, dya, pos);
                const bool split = need && !p2;
                if (rep && split) {
                    const uint32_t z = morton3(tx >> lgB, ty >> lgB);
                    splitbits |= 1u << (((1u << (2 * (j - 1))) - 1) / 3 + z);
                }
                act = split;
                if (Bc >= 8) {
                    cur.k = ch[0].k;
                    cur.q = ch[0].q;
                    cur.pass = ch[0].pass;
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        cur4[h].k = ch[h].k;
                        cur4[h].q = ch[h].q;
                        cur4[h].pass = ch[h].pass;
                    }
                }
            } else if (MIN2 && j < L) {
                // B == 4 above the last level: each half is a 4 x 4 block of
                // level j with four 2 x 2 children at level j + 1 = L, fitted
                // against their own centred domains (Section 3; phase 2 of the
                // 4 x 4 block, Sections 3.1-3.2, tests them as its sub-blocks)
                const long long thr_p2 = D.t2q[j - 1] << 14;  // n = 4: t2q n^2 1024
                const int dmax = (j == 1) ? 15 : 31;
                const int c0 = phase2_code(j, 0), c1 = phase2_code(j, 1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int xh = sx0 + 8 * pc + 4 * h, yh = sy0 + 4 * pr;
                    const int tx = 8 * pc + 4 * h - lane_top * BMAX, ty = 4 * pr;
                    const int posh = lane_top * cpt + (int)morton3(tx >> 1, ty >> 1);
                    const int dxh = centred_origin(xh, 4, W), dyh = centred_origin(yh, 4, H);
                    if (act) fits += 1;
                    if (act && cur4[h].pass)
                        make_leaf(leaf[h], xh, yh, j, 1, cur4[h].k, cur4[h].q, 0, 0, 0, dxh, dyh, posh);
                    const bool need_h = act && !cur4[h].pass;
                    if (!__any_sync(FULL, need_h)) continue;
                    if (ph2 && need_h) fits += 4;
                    const int Oi = lum(cur4[h].q, ko1, magic);
                    int csr[4], csrr[4], dl[4];
                    bool inr = true;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int bi = k & 1, bj = k >> 1;
                        const uint32_t t = h ? rw[2 * bj].y : rw[2 * bj].x;
                        const uint32_t u = h ? rw[2 * bj + 1].y : rw[2 * bj + 1].x;
                        const uint32_t m1 = bi ? 0x01010000u : 0x00000101u, mb = bi ? 0xffff0000u : 0x0000ffffu;
                        csr[k] = (int)__dp4a(t, m1, __dp4a(u, m1, 0u));
                        csrr[k] = (int)__dp4a(t, t & mb, __dp4a(u, u & mb, 0u));
                        // round half up of (mean_k - O_i), n = 4
                        dl[k] = (2 * (csr[k] - (Oi << 2)) + 4) >> 3;
                        inr = inr && dl[k] <= dmax && dl[k] >= -dmax;
                    }
                    const int O3 = Oi - (dl[0] + dl[1] + dl[2]);  // eq. (1)
                    bool allok = true;
                    int sb = 0;
                    uint4 cw[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int bi = k & 1, bj = k >> 1;
                        const int xc = xh + 2 * bi, yc = yh + 2 * bj;
                        const int dxc = centred_origin(xc, 2, W), dyc = centred_origin(yc, 2, H);
                        const uint32_t t = h ? rw[2 * bj].y : rw[2 * bj].x;
                        const uint32_t u = h ? rw[2 * bj + 1].y : rw[2 * bj + 1].x;
                        // moments of the child against a 4 x 4 domain read from
                        // the raw window (any column parity)
                        auto dom = [&](int ddx, int ddy, Fit &f) {
                            const int o = ddx - ax0;
                            const uint8_t *rp = raw + (ddy - ry0) * pitch + (o & ~3);
                            uint32_t rr[4];
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                const uint32_t w0 = *reinterpret_cast<const uint32_t *>(rp + r * pitch);
                                const uint32_t w1 = *reinterpret_cast<const uint32_t *>(rp + r * pitch + 4);
                                rr[r] = __funnelshift_r(w0, w1, 8 * (o & 3));
                            }
                            const uint32_t top = pair2x2(rr[0], rr[1]), bot = pair2x2(rr[2], rr[3]);
                            const int sdr = bi ? (int)dp2a_hi(top, t, dp2a_hi(bot, u, 0u))
                                               : (int)dp2a_lo(top, t, dp2a_lo(bot, u, 0u));
                            const uint32_t pk = top + bot;
                            const int sd = (int)((pk & 0xffffu) + (pk >> 16));
                            unsigned ql = 0, qh = 0;
                            acc_sq(top, ql, qh);
                            acc_sq(bot, ql, qh);
                            const int sdd = (int)(ql + (qh << 8));
                            f.sr = csr[k];
                            f.ncrr = ((long long)csrr[k] << 2) - (long long)csr[k] * csr[k];
                            f.ncdr = ((long long)sdr << 2) - (long long)sd * csr[k];
                            f.ncdd = ((long long)sdd << 2) - (long long)sd * sd;
                        };
                        Fit f;
                        dom(dxc, dyc, f);
                        const int kc = best_contrast<true>(f.ncdr, f.ncdd, s_bits);
                        int bd;
                        const int qc = best_luminance(csr[k], 2, ko1, magic, qscale, bd);
                        // the phase-2 sub-block fit: against its own centred domain
                        // or, with the other reading, quadrant k of the parent's
                        if (D.phase2_domain) dom(dxh + 4 * bi, dyh + 4 * bj, f);
                        int bit;
                        const bool ok = fit_phase2_sub(f, 2, k == 3 ? O3 : Oi + dl[k], c0, c1, thr_p2, bit);
                        allok = allok && ok;
                        sb |= bit << k;
                        cw[k] = make_uint4((uint32_t)xc | ((uint32_t)yc << 16),
                                           (uint32_t)(j + 1) | (1u << 8) | ((uint32_t)kc << 16) | ((uint32_t)qc << 24),
                                           0u, (uint32_t)dxc | ((uint32_t)dyc << 16));
                    }
                    const bool p2 = ph2 && need_h && inr && allok;
                    if (p2) make_leaf(leaf[h], xh, yh, j, 2, sb, cur4[h].q, dl[0], dl[1], dl[2], dxh, dyh, posh);
                    if (need_h && !p2) {
                        splitbits |= 1u << (((1u << (2 * (j - 1))) - 1) / 3 + morton3(tx >> 2, ty >> 2));
                        fits += 4;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int pos = lane_top * cpt + (int)morton3((tx >> 1) + (k & 1), (ty >> 1) + (k >> 1));
                            lrec[pos] = cw[k];
                            atomicOr(lmask + (pos >> 5), 1u << (pos & 31));
                        }
                    }
                }
                break;
            } else {
                // B == 4: last level, forced acceptance (two leaves per lane)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!act) continue;
                    fits += 1;
                    const int xa = sx0 + 8 * pc + 4 * h, ya = sy0 + 4 * pr;
                    const int tx = 8 * pc + 4 * h - lane_top * BMAX, ty = 4 * pr;
                    const int pos = lane_top * cpt + (int)morton3(tx >> lgbmin, ty >> lgbmin);
                    make_leaf(leaf[h], xa, ya, j, 1, cur4[h].k, cur4[h].q, 0, 0, 0, centred_origin(xa, 4, W),
                              centred_origin(ya, 4, H), pos);
                }
                break;
            }
        }

        if (MIN2 && SLOTS) {
            // the raw window is free now: fetch the next strip's
            __syncwarp();
            if (lane == 0 && g_next < total_strips) issue_window(g_next);
            // the lanes' own leaves join the staged ones; then each lane
            // stores the leaves at positions lane, lane + 32, ... at their
            // canonical ranks
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (leaf[h].pos < 0) continue;
                lrec[leaf[h].pos] = make_uint4(leaf[h].w0, leaf[h].w1, leaf[h].w2, leaf[h].w3);
                atomicOr(lmask + (leaf[h].pos >> 5), 1u << (leaf[h].pos & 31));
            }
            __syncwarp();
            uint32_t mw[8], before[8];
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                mw[w] = lmask[w];
                before[w] = run;
                run += (uint32_t)__popc(mw[w]);
            }
            fic_record *slot = D.slots + (size_t)s * D.slot_recs;
            const uint32_t below = (1u << lane) - 1u;
#pragma unroll
            for (int w = 0; w < 8; ++w)
                if ((mw[w] >> lane) & 1u)
                    *reinterpret_cast<uint4 *>(slot + before[w] + (uint32_t)__popc(mw[w] & below)) = lrec[32 * w + lane];
            const unsigned ftot = __reduce_add_sync(FULL, fits);
            splitbits = group_or<PC>(splitbits, BMAX / 8, BMAX / 4);
            if (valid && (8 * pc) % BMAX == 0 && pr == 0) {
                const int p0 = lane_top * cpt;  // first position of the lane's top-level block
                uint32_t first = 0;
#pragma unroll
                for (int w = 0; w < 8; ++w)
                    first += (32 * w + 32 <= p0) ? (uint32_t)__popc(mw[w])
                           : (32 * w < p0 ? (uint32_t)__popc(mw[w] & ((1u << (p0 & 31)) - 1u)) : 0u);
                D.split[top0 + lane_top] = splitbits;
                D.tile_off[top0 + lane_top] = first;
            }
            if (lane == 0) D.stats[s] = make_uint2(run, ftot & 0x7fffffffu);
            __syncwarp();
            g = ticketed ? __shfl_sync(FULL, g_next, 0) : g_next;
            g_next = g_after;
            continue;
        }
        // ---- canonical ranks, look-back, stores
        unsigned long long mine = 0;
        if (leaf[0].pos >= 0) mine |= 1ull << leaf[0].pos;
        if (leaf[1].pos >= 0) mine |= 1ull << leaf[1].pos;
        const uint32_t mlo = __reduce_or_sync(FULL, (uint32_t)mine);
        const uint32_t mhi = __reduce_or_sync(FULL, (uint32_t)(mine >> 32));
        const unsigned long long mask = ((unsigned long long)mhi << 32) | mlo;
        const int cnt = __popcll(mask);
        if (SLOTS) {
            // records to the strip's slot; counts, fits and per-top offsets
            // inside the strip for pack_kernel
            fic_record *slot = D.slots + (size_t)s * kSlotRecords;
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
            g = ticketed ? __shfl_sync(FULL, g_next, 0) : g_next;
            g_next = g_after;
            continue;
        }
        // decoupled look-back, 32 predecessors per round (one per lane)
        uint32_t prefix = 0;
        int ok = 1;
        if (s == 0) {
            if (lane == 0) st_volatile(status + g, kIncl | (uint32_t)cnt);
        } else {
            if (lane == 0) st_volatile(status + g, kAgg | (uint32_t)cnt);
            int p = g - 1;
            for (;;) {
                const int idx = p - lane;
                const bool in = idx >= D.strip_base;
                uint32_t v = in ? ld_volatile(status + idx) : kIncl;
                unsigned it = 0;
                while (!__all_sync(FULL, v != 0u) && ++it < kSpinLimit) {
                    __nanosleep(32);
                    if (v == 0u) v = ld_volatile(status + idx);
                }
                if (!__all_sync(FULL, v != 0u)) {
                    ok = 0;
                    break;
                }
                const uint32_t incl = __ballot_sync(FULL, (v & ~kValMask) == kIncl);
                const int first = incl ? __ffs(incl) - 1 : 32;
                uint32_t val = (lane <= first) ? (v & kValMask) : 0u;
                val = __reduce_add_sync(FULL, val);
                prefix += val;
                if (incl) break;
                p -= 32;
            }
            if (lane == 0) {
                if (ok) st_volatile(status + g, kIncl | (prefix + (uint32_t)cnt));
                else raise_error(D.info, FIC_DEVERR_TIMEOUT);
            }
        }
        const unsigned ftot = __reduce_add_sync(FULL, fits);
        if (lane == 0 && ftot)
            atomicAdd(reinterpret_cast<unsigned long long *>(D.info + FIC_INFO_FITS_LO), (unsigned long long)ftot);
        if (!ok) {
            g = __shfl_sync(FULL, g_next, 0);
            g_next = g_after;
            continue;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (leaf[h].pos < 0) continue;
            const uint32_t idx = prefix + (uint32_t)__popcll(mask & ((1ull << leaf[h].pos) - 1ull));
            if (idx < (uint32_t)D.capacity) {
                *reinterpret_cast<uint4 *>(D.rec + idx) = make_uint4(leaf[h].w0, leaf[h].w1, leaf[h].w2, leaf[h].w3);
            } else {
                raise_error(D.info, FIC_DEVERR_CAPACITY);
            }
        }
        // split masks: OR over the lanes of each top-level block
        splitbits = group_or<PC>(splitbits, BMAX / 8, BMAX / 4);
        if (valid && (8 * pc) % BMAX == 0 && pr == 0) {
            D.split[top0 + lane_top] = splitbits;
            D.tile_off[top0 + lane_top] = prefix + (uint32_t)__popcll(mask & ((1ull << (lane_top * cpt)) - 1ull));
        }
        if (lane == 0 && s == D.nstrips - 1) {
            D.tile_off[D.tw * D.th] = prefix + (uint32_t)cnt;
            D.info[FIC_INFO_RECORDS] = prefix + (uint32_t)cnt;
        }
        g = __shfl_sync(FULL, g_next, 0);
        g_next = g_after;
    }
}

// Zero the look-back (or pack) state, the ticket and every stream's info block.
__global__ void encode_init_kernel(const EncDesc *__restrict__ descs, int count, uint32_t *status,
                                   int total_strips, uint32_t *ticket) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int t = i; t < total_strips; t += stride) status[t] = 0u;
    for (int t = i; t < count * FIC_INFO_WORDS; t += stride) descs[t / FIC_INFO_WORDS].info[t % FIC_INFO_WORDS] = 0u;
    if (i == 0) *ticket = 0u;
}

size_t mns_smem_bytes(int bmax, int nw, bool min2) {
    const size_t per = (bmax == 32 ? WinBox<32>::W * WinBox<32>::H + Geom<32>::WORDS * 4
                        : bmax == 16 ? WinBox<16>::W * WinBox<16>::H + Geom<16>::WORDS * 4
                                     : WinBox<8>::W * WinBox<8>::H + Geom<8>::WORDS * 4) +
                       (min2 ? 256 * 16 + 128 : 0);
    return (size_t)nw * per + 128;  // + alignment slack
}

int mns_strip_width(int bmax) { return 1024 / bmax; }

// Resident CTAs per SM of one instantiation (its occupancy limit, per device).
template <int BMAX, bool SLOTS, int NW, bool MIN2>
static int mns_occupancy(int &sms) {
    static KernelSlots ks;
    int per = 0;
    if (kernel_slots(ks, (const void *)mns_encode_kernel<BMAX, SLOTS, NW, MIN2>, NW * 32,
                     mns_smem_bytes(BMAX, NW, MIN2), sms, per) != cudaSuccess)
        return 0;
    return per;
}

template <int BMAX, bool SLOTS, int NW, bool MIN2 = false>
static cudaError_t launch_t(const EncDesc *descs, int count, int total_strips, uint32_t *status,
                            uint32_t *ticket, int total_chunks, int ctas_per_sm, int dyn, int fused,
                            cudaStream_t st) {
    int sms = 0;
    const int per = mns_occupancy<BMAX, SLOTS, NW, MIN2>(sms);
    if (per == 0) return cudaErrorInvalidValue;
    const int k = ctas_per_sm > 0 && ctas_per_sm < per ? ctas_per_sm : per;
    const int need = (total_strips + NW - 1) / NW;
    const int grid = need < sms * k ? need : sms * k;
    mns_encode_kernel<BMAX, SLOTS, NW, MIN2><<<grid, NW * 32, mns_smem_bytes(BMAX, NW, MIN2), st>>>(
        descs, count, total_strips, status, ticket, total_chunks, dyn, fused);
    stage_mark(st, "mns_encode_kernel");
    return cudaGetLastError();
}

static cudaError_t launch_init(const EncDesc *d_descs, int count, int nstatus, uint32_t *status, uint32_t *ticket,
                               cudaStream_t st) {
    const int threads = 256;
    int blocks = (nstatus + threads - 1) / threads;
    int b2 = (count * FIC_INFO_WORDS + threads - 1) / threads;
    if (b2 > blocks) blocks = b2;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    encode_init_kernel<<<blocks, threads, 0, st>>>(d_descs, count, status, nstatus, ticket);
    return cudaGetLastError();
}

// Ticket + look-back variant: the stream is packed by the encoder itself.
cudaError_t launch_mns_encode(int bmax, const EncDesc *d_descs, int count, int total_strips,
                              uint32_t *status, uint32_t *ticket, cudaStream_t st) {
    cudaError_t e = launch_init(d_descs, count, total_strips, status, ticket, st);
    if (e != cudaSuccess) return e;
    switch (bmax) {
    case 32: return launch_t<32, false, kWarps>(d_descs, count, total_strips, status, ticket, 0, 0, 1, 0, st);
    case 16: return launch_t<16, false, kWarps>(d_descs, count, total_strips, status, ticket, 0, 0, 1, 0, st);
    case 8: return launch_t<8, false, kWarps>(d_descs, count, total_strips, status, ticket, 0, 0, 1, 0, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pack(const EncDesc *d_descs, int count, int total_chunks, uint32_t *pack_status,
                        uint32_t *ticket, cudaStream_t st);
cudaError_t launch_mns32_slots(const EncDesc *d_descs, int count, int total_strips, int total_chunks,
                               uint32_t *pack_status, uint32_t *ticket, const EncTune &tune, cudaStream_t st);

// Slot variant: encode into per-strip slots, then compact with pack_kernel.
// `tune` picks warps per CTA, CTAs per SM and the strip schedule; every
// choice writes the same stream.
cudaError_t launch_mns_encode_slots(int bmax, const EncDesc *d_descs, int count, int total_strips, int total_chunks,
                                    uint32_t *pack_status, uint32_t *ticket, const EncTune &tune, cudaStream_t st) {
    cudaError_t e;
    const int k = tune.ctas_per_sm, dyn = tune.dynamic ? 1 : 0;
    // fused packing copies at most 64 records per strip: not with 2 x 2 leaves
    const int fused = tune.fused_pack && !tune.min2 ? 1 : 0;
    uint32_t *tk = dyn ? ticket : nullptr;
    const bool w4 = tune.warps == 4;
    if (fused) {
        // look-back status, strip counter and chunk counters start at zero
        // (status, ticket and counters are contiguous in the workspace)
        e = cudaMemsetAsync(pack_status, 0, (2 * (size_t)total_chunks + 1) * sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
    }
    if (bmax == 32 && tune.kernel32) {
        e = launch_mns32_slots(d_descs, count, total_strips, total_chunks, pack_status, tk, tune, st);
        if (e != cudaSuccess || fused) return e;
        return launch_pack(d_descs, count, total_chunks, pack_status, tk, st);
    }
#define FIC_SLOTS_LAUNCH(B, M2)                                                                                    \
    e = w4 ? launch_t<B, true, 4, M2>(d_descs, count, total_strips, pack_status, tk, total_chunks, k, dyn, fused, st) \
           : launch_t<B, true, kWarps, M2>(d_descs, count, total_strips, pack_status, tk, total_chunks, k, dyn, fused, \
                                            st)
    if (tune.min2) {
        switch (bmax) {
        case 16: FIC_SLOTS_LAUNCH(16, true); break;
        case 8: FIC_SLOTS_LAUNCH(8, true); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (bmax) {
        case 32: FIC_SLOTS_LAUNCH(32, false); break;
        case 16: FIC_SLOTS_LAUNCH(16, false); break;
        case 8: FIC_SLOTS_LAUNCH(8, false); break;
        default: return cudaErrorInvalidValue;
        }
    }
#undef FIC_SLOTS_LAUNCH
    if (e != cudaSuccess || fused) return e;
    return launch_pack(d_descs, count, total_chunks, pack_status, tk, st);
}

}  // namespace fic

// ---------------------------------------------------------------------------
// Allocation-free encode entry point.
//
// Some callers cannot allocate device memory at all: code embedded in a host
// application that owns the whole device heap and hands out no allocator,
// or code on a latency-critical path where a device allocation (which can
// synchronise the device) is not allowed.  For them fic_encode_noalloc keeps
// the encoder's scratch -- the image descriptor, the look-back status words
// of the stream packer and the ticket counter -- in this file-scope device
// array instead of a caller workspace.  Every GPU that loads the library
// holds the array (about 256 KiB) until the process exits.  The image's
// tensor map (for the TMA window loads) lives in the same array.
#include <mutex>

namespace {

struct NoAllocScratch {
    fic::TmaMap map;
    fic::EncDesc desc;
    uint32_t ticket;
    uint32_t pad[63];
    uint32_t status[FIC_NOALLOC_MAX_STRIPS];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_noalloc_mutex;
NoAllocScratch *g_noalloc_addr[fic::kMaxDevices] = {};

// The array's name is only a host-side stand-in: the device address must be
// asked for, once per device, with that device current.
int noalloc_scratch_for_current_device(NoAllocScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= fic::kMaxDevices) return FIC_ECUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FIC_ECUDA;
        g_noalloc_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_noalloc_addr[dev];
    return FIC_OK;
}

}  // namespace

extern "C" int fic_encode_noalloc(const uint8_t *d_img, int width, int height, const fic_params *p,
                                  fic_stream *out, void *stream) {
    using namespace fic;
    int rc = fic_validate(width, height, p);
    if (rc) return rc;
    if (p->mode != FIC_NOSEARCH && p->mode != FIC_MNS) return FIC_EBADPARAM;  // centred-domain modes only
    if (p->bmin < 4) return FIC_EBADPARAM;  // leaves of 4 x 4 pixels or more
    if (!d_img || (reinterpret_cast<uintptr_t>(d_img) & 15) || !out) return FIC_EBADPARAM;
    if (!out->records || !out->tile_offsets || !out->split || !out->info || out->capacity <= 0)
        return FIC_EBADPARAM;
    if ((reinterpret_cast<uintptr_t>(out->records) & 15) || (reinterpret_cast<uintptr_t>(out->info) & 7))
        return FIC_EBADPARAM;
    const int bmax = p->bmax;
    const int tops = mns_strip_width(bmax) / bmax;
    const int tw = width / bmax, th = height / bmax;
    const int spr = (tw + tops - 1) / tops;
    const long long nstrips = (long long)spr * th;
    if (nstrips > FIC_NOALLOC_MAX_STRIPS) return FIC_EBADSIZE;  // larger than the static scratch
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        // the descriptor is staged from this call's own host memory, which a
        // captured graph could not replay: refuse to be captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FIC_ECUDA;
        if (cs != cudaStreamCaptureStatusNone) return FIC_EBADPARAM;
    }
    NoAllocScratch *scr = nullptr;
    rc = noalloc_scratch_for_current_device(&scr);
    if (rc) return rc;

    int L = 1;
    for (int b = p->bmax; b > p->bmin; b >>= 1) ++L;
    EncDesc d;
    memset(&d, 0, sizeof(d));
    d.img = d_img;
    d.rec = out->records;
    d.tile_off = out->tile_offsets;
    d.split = out->split;
    d.info = out->info;
    for (int j = 0; j < 4; ++j) {
        const double t = p->thr_rms[j < L ? j : L - 1];
        d.t2q[j] = (int64_t)(t * t * 256.0 + 0.5);
    }
    d.W = width;
    d.H = height;
    d.tw = tw;
    d.th = th;
    d.spr = spr;
    d.strip_base = 0;
    d.nstrips = (int)nstrips;
    d.capacity = out->capacity;
    d.mode = p->mode;
    d.bmin = p->bmin;
    d.L = L;
    d.phase2 = p->phase2 ? 1 : 0;
    d.phase2_domain = p->phase2_domain ? 1 : 0;
    d.s_bits = p->s_bits;
    d.o_bits = p->o_bits;
    d.local_radius = p->local_radius;
    d.local_step = p->local_step;
    d.bmax = bmax;
    d.slot_recs = 64;
    {
        const int bw = bmax == 32 ? WinBox<32>::W : (bmax == 16 ? WinBox<16>::W : WinBox<8>::W);
        d.boxw = bw < width ? bw : width;
    }
    d.map = &scr->map;
    TmaMap map;
    rc = make_tma_map(&map, d_img, width, height, d.boxw, 2 * bmax);
    if (rc) return rc;
    out->width = width;
    out->height = height;
    out->params = *p;
    out->ntop = tw * th;

    // The descriptor is staged from host memory; the status words, the ticket
    // and the stream's info block are cleared by the init kernel of the launch.
    if (cudaMemcpyAsync(&scr->map, &map, sizeof(map), cudaMemcpyHostToDevice, st) != cudaSuccess) return FIC_ECUDA;
    if (cudaMemcpyAsync(&scr->desc, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess) return FIC_ECUDA;
    return launch_mns_encode(bmax, &scr->desc, 1, (int)nstrips, scr->status, &scr->ticket, st) == cudaSuccess
               ? FIC_OK
               : FIC_ECUDA;
}
