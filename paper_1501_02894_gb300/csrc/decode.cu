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
// 1024-pixel strip, lane = 8x4 patch, two 4x4 half-patches per lane).
//   * decode_setup_kernel (once per decode): for every half-patch, the
//     transform that covers it (the strip's leaves tile its bmin cells in
//     canonical order, so a 64-bit mask of their first cells ranks a cell's
//     leaf with one popcount) packed into one word: window column/row of its
//     domain values, block side, contrast byte, luminance; plus a per-strip
//     word.  It also writes the first iterate (from 128: the luminances).
//   * decode_d4_iter_kernel (centred streams, once per later iteration):
//     iterates on 2x2-sum images (below); decode_iter_kernel (other streams):
//     stages the decimated window of the previous pixel iterate.  Both read
//     16 domain values per half-patch, reduce Sd4 per transform with xor
//     shuffles, then per pixel one dp2a (select + multiply + offset), one
//     shift and half of a saturating pack.
// Domains that are not centred (local / exhaustive search, isometries) are
// read from global memory instead of the staged window.
#include "fic_internal.cuh"

namespace fic {

template <int BMAX>
struct DGeom {
    static constexpr int SW = 1024 / BMAX;
    static constexpr int PC = SW / 8;
    static constexpr int PR = BMAX / 4;
    static constexpr int TOPS = SW / BMAX;
    // words per window row: the window's width (32, 48, 80 2x2 sums) and,
    // for BMAX 32, 4 words of padding so that the lanes of patch rows 4
    // apart (rows 16 words apart) fall in different shared-memory banks
    static constexpr int NP = BMAX == 32 ? 20 : (BMAX == 16 ? 24 : 40);
    static constexpr int WORDS = BMAX * NP;
    static constexpr int UPR = BMAX == 32 ? 4 : (BMAX == 16 ? 8 : 16);
    // lane bit that swaps the order of a row's two word loads, so that one
    // load instruction touches words of both parities: with the padding
    // above, at most two lanes of a leaf share a bank
    __device__ static int bank_key(int pr) { return BMAX == 32 ? (pr >> 1) & 1 : pr & 1; }
};

constexpr int kDecWarps = 8;


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

// Clamp two signed values to [0, 255] and pack them, with the upper half
// taken from `hi`: result bytes (b, a, hi.byte0, hi.byte1).
__device__ __forceinline__ uint32_t pack_sat_u8(int a, int b, uint32_t hi) {
    uint32_t d;
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(hi));
    return d;
}

// Four output pixels of one row: p = (c * d4 + K) >> 9, clamped, packed.
// dp2a with the contrast in one byte of the second operand picks one 16-bit
// d4 of the pair and multiplies-adds it in one instruction.
__device__ __forceinline__ uint32_t row_pixels(uint32_t p01, uint32_t p23, int cb0, int cb1, int K) {
    const int m0 = __dp2a_lo((int)p01, cb0, K) >> 9;
    const int m1 = __dp2a_lo((int)p01, cb1, K) >> 9;
    const int m2 = __dp2a_lo((int)p23, cb0, K) >> 9;
    const int m3 = __dp2a_lo((int)p23, cb1, K) >> 9;
    return pack_sat_u8(m1, m0, pack_sat_u8(m3, m2, 0u));
}

// Per-strip word of the decode tables.
struct StripInfo {
    const uint8_t *buf[2];
    int32_t W;
    uint32_t sxy;    // sx0 | sy0 << 16
    uint32_t axy;    // ax0 | ry0 << 16   (window origin, pixels)
    uint32_t misc;   // upr | nvalid << 8 | centred << 16
};

// Per-strip word of the 2x2-sum iteration (centred streams).
struct StripD4 {
    uint16_t *d4[2];       // ping-pong 2x2-sum images, (W/2) x (H/2)
    uint8_t *out;          // pixels, written by the last iteration
    const TmaMap *map[2];  // tensor maps of d4[0], d4[1] (box 2*NP x BMAX)
    uint32_t *info;        // the stream's info block (device error bits)
    int32_t W;             // pixels
    uint32_t sxy;          // sx0 | sy0 << 16
    uint32_t wxy;          // window origin in 2x2-sum units: c_base | r_base << 16
    uint32_t misc;         // nvalid << 8
};
static_assert(sizeof(StripD4) == 64, "strip word: one 64-byte bulk copy");

// 2x2 sums of two rows of four pixels each: (p0+p1+q0+q1) | (p2+p3+q2+q3) << 16.
__device__ __forceinline__ uint32_t sum2x2(uint32_t a, uint32_t b) {
    const uint32_t lo = __dp4a(a, 0x00000101u, __dp4a(b, 0x00000101u, 0u));
    const uint32_t hi = __dp4a(a, 0x01010000u, __dp4a(b, 0x01010000u, 0u));
    return __byte_perm(lo, hi, 0x5410);
}

// Per-lane transform words of the 2x2-sum path (one uint4 per lane and
// strip, written by the setup kernel):
//   x, y  fast words of the two half-patches (c | rr << 8 | lg << 16 | cbyte << 24)
//   z     their luminances O0 | O1 << 16 (signed 16-bit)
//   w     the lane's element offset in the (W/2) x (H/2) 2x2-sum images (its
//         top-left 2x2 sum), or kNoLane for a lane outside the image
// so that an iteration needs, per strip, only the image's 2x2-sum base and
// width besides its window.
constexpr uint32_t kNoLane = 0xffffffffu;

__device__ __forceinline__ int lum16(uint32_t z, int h) { return (int)(int16_t)(h ? (z >> 16) : (z & 0xffffu)); }

// First iteration from x0 = 128: every pixel is its transform's luminance.
// `last`: write the pixels (the only iteration) instead of their 2x2 sums.
template <int BMAX>
__device__ __forceinline__ void first_d4(uint4 tf, uint16_t *d4o, uint8_t *out, int W, uint32_t sxy, bool last,
                                         int lane) {
    constexpr int PC = DGeom<BMAX>::PC;
    if (tf.w == kNoLane) return;
    const int O0 = min(max(lum16(tf.z, 0), 0), 255), O1 = min(max(lum16(tf.z, 1), 0), 255);
    if (last) {
        const int pr = lane / PC, pc = lane % PC;
        const int sx0 = (int)(sxy & 0xffffu), sy0 = (int)(sxy >> 16);
        uint8_t *o = out + (size_t)(sy0 + 4 * pr) * W + sx0 + 8 * pc;
        const uint32_t w0 = (uint32_t)O0 * 0x01010101u, w1 = (uint32_t)O1 * 0x01010101u;
#pragma unroll
        for (int i = 0; i < 4; ++i) *reinterpret_cast<uint2 *>(o + (size_t)i * W) = make_uint2(w0, w1);
    } else {
        const int W2 = W >> 1;
        uint16_t *o = d4o + tf.w;
        const uint32_t w0 = (uint32_t)(4 * O0) * 0x00010001u, w1 = (uint32_t)(4 * O1) * 0x00010001u;
#pragma unroll
        for (int j = 0; j < 2; ++j) *reinterpret_cast<uint2 *>(o + (size_t)j * W2) = make_uint2(w0, w1);
    }
}

// Per-half-patch words: fast word (c | rr << 8 | lg << 16 | cbyte << 24, O)
// and, for domains outside the window, (dx | dy << 16, u0 | v0 << 8 | iso << 16).
__device__ __forceinline__ uint32_t fast_word(int c, int rr, int lg, int cc) {
    return (uint32_t)c | ((uint32_t)rr << 8) | ((uint32_t)lg << 16) | ((uint32_t)(cc & 0xff) << 24);
}

// Transform words of one strip (the lookup of every half-patch's transform
// in the strip's records), written to the decode tables.
template <int BMAX, bool D4>
__device__ __forceinline__ void setup_strip(const DecDesc *__restrict__ descs, int count, const int *s_base, int g,
                                            uint4 *recs, void *sinfo, uint4 *tfw, uint4 *tgw,
                                            int first_kind, int lane) {
    using G = DGeom<BMAX>;
    constexpr int PC = G::PC;
    const int pr = lane / PC, pc = lane % PC;
    const int img = find_image_s(s_base, descs, count, g);
    const DecDesc &D = descs[img];
    const int W = D.W, H = D.H, tw = D.tw;
    const int s = g - D.strip_base;
    const int row = s / D.spr, sc = s - row * D.spr;
    const int sy0 = row * BMAX, sx0 = sc * G::SW;
    const int top0 = row * tw + sc * G::TOPS;
    const int nvalid = min(G::TOPS, tw - sc * G::TOPS);
    const int lane_top = (8 * pc) / BMAX;
    const bool valid = lane_top < nvalid;
    const int bmin = D.bmin;
    const int lgbmin = 31 - __clz(bmin);  // bmin is a power of two: divisions are shifts
    const int cpt_side = BMAX >> lgbmin, cpt = cpt_side * cpt_side;
    const bool centred = (D.mode == FIC_NOSEARCH || D.mode == FIC_MNS);
    const int ko1 = (1 << D.o_bits) - 1;
    // L(q) = floor((510 q + ko1) / (2 ko1)) by a multiply-high (exact for q <= ko1 <= 255)
    const uint32_t lmagic = c_lum_magic[D.o_bits];
    const int rx0 = clampi(sx0 - BMAX / 2, 0, W - 2 * BMAX);
    const int xl = sx0 + (nvalid - 1) * BMAX;
    const int rx1 = clampi(xl - BMAX / 2, 0, W - 2 * BMAX) + 2 * BMAX;
    const int ax0 = rx0 & ~15, ax1 = (rx1 + 15) & ~15;
    const int ry0 = clampi(sy0 - BMAX / 2, 0, H - 2 * BMAX);
    const int c_base = ax0 >> 1, r_base = ry0 >> 1;

    const uint32_t rbeg = D.tile_off[top0], rend = D.tile_off[top0 + nvalid];
    const int nrec = min((int)(rend - rbeg), 64);
    // the strip's leaves tile its (at most 64) bmin cells in canonical order:
    // a 64-bit mask of their first cells ranks any cell's covering leaf
    __syncwarp();
    unsigned long long occ = 0;
    for (int i = lane; i < nrec; i += 32) {
        const uint4 r = *reinterpret_cast<const uint4 *>(D.rec + rbeg + i);
        recs[i] = r;
        const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16);
        const int lt = x / BMAX - sc * G::TOPS;
        const int key = min(lt * cpt + (int)morton3((x % BMAX) >> lgbmin, (y % BMAX) >> lgbmin), 63);
        occ |= 1ull << key;
    }
    occ = ((unsigned long long)__reduce_or_sync(0xffffffffu, (uint32_t)(occ >> 32)) << 32) |
          __reduce_or_sync(0xffffffffu, (uint32_t)occ);
    __syncwarp();
    uint32_t fw[2] = {0u, 0u}, gw[2] = {0u, 0u}, hw[2] = {0u, 0u};
    int Ow[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!valid || nrec <= 0) continue;
        const int px = 8 * pc + 4 * h, py = 4 * pr;  // in strip
        const int tx = px - lane_top * BMAX;
        const int key = min(lane_top * cpt + (int)morton3(tx >> lgbmin, py >> lgbmin), 63);
        const unsigned long long upto = key == 63 ? ~0ull : ((2ull << key) - 1ull);
        const int lo = max(__popcll(occ & upto) - 1, 0);  // last leaf starting at or before the cell
        const uint4 r = recs[min(lo, nrec - 1)];
        const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16);
        const int level = (int)(r.y & 0xffu), phase = (int)((r.y >> 8) & 0xffu);
        const int k = (int)((r.y >> 16) & 0xffu), q = (int)(r.y >> 24);
        const int B = BMAX >> (level - 1);
        const int Oi = (int)__umulhi((uint32_t)(510 * q + ko1), lmagic);
        int t_x, t_y, t_lg, t_dx, t_dy, t_c, t_O, t_iso;
        if (phase == 1) {
            t_x = x;
            t_y = y;
            t_lg = 31 - __clz(B);
            t_dx = (int)(r.w & 0xffffu);
            t_dy = (int)(r.w >> 16);
            t_c = contrast_code(k, D.s_bits);
            t_O = Oi;
            t_iso = (int)(r.z >> 24);
        } else {
            const int hb = B >> 1;
            const int ax = sx0 + px, ay = sy0 + py;
            const int sb = (ax - x >= hb ? 1 : 0) | (ay - y >= hb ? 2 : 0);
            const int d0 = (int)(int8_t)(r.z & 0xffu), d1 = (int)(int8_t)((r.z >> 8) & 0xffu),
                      d2 = (int)(int8_t)((r.z >> 16) & 0xffu);
            const int O0 = Oi + d0, O1 = Oi + d1, O2 = Oi + d2;
            const int O3 = 4 * Oi - (O0 + O1 + O2);  // eq. (1)
            t_O = sb == 0 ? O0 : (sb == 1 ? O1 : (sb == 2 ? O2 : O3));
            t_x = x + (sb & 1) * hb;
            t_y = y + (sb >> 1) * hb;
            t_lg = 31 - __clz(hb);
            if (D.phase2_domain) {  // quadrant sb of the block's own centred domain
                t_dx = centred_origin(x, B, W) + (sb & 1) * B;
                t_dy = centred_origin(y, B, H) + (sb >> 1) * B;
            } else {
                t_dx = centred_origin(t_x, hb, W);
                t_dy = centred_origin(t_y, hb, H);
            }
            t_c = phase2_code(level, (k >> sb) & 1);
            t_iso = 0;
        }
        const int u0 = sx0 + px - t_x, v0 = sy0 + py - t_y;
        const int c = centred ? (t_dx >> 1) + u0 - c_base : 0;
        const int rr = centred ? (t_dy >> 1) + v0 - r_base : 0;
        fw[h] = fast_word(c, rr, t_lg, t_c);
        Ow[h] = t_O;
        gw[h] = (uint32_t)t_dx | ((uint32_t)t_dy << 16);
        hw[h] = (uint32_t)u0 | ((uint32_t)v0 << 8) | ((uint32_t)t_iso << 16);
    }
    if (D4) {
        const uint32_t off =
            valid ? (uint32_t)(((sy0 >> 1) + 2 * pr) * (W >> 1) + (sx0 >> 1) + 4 * pc) : kNoLane;
        const uint4 tf = make_uint4(fw[0], fw[1], ((uint32_t)Ow[0] & 0xffffu) | ((uint32_t)Ow[1] << 16), off);
        tfw[(size_t)g * 32 + lane] = tf;
        // the first iteration from 128 needs only the luminance: written here
        if (first_kind)
            first_d4<BMAX>(tf, D.d4[0], D.buf[0], W, (uint32_t)sx0 | ((uint32_t)sy0 << 16), first_kind == 3, lane);
    } else {
        tfw[(size_t)g * 32 + lane] = make_uint4(fw[0], (uint32_t)Ow[0], fw[1], (uint32_t)Ow[1]);
        if (!centred) tgw[(size_t)g * 32 + lane] = make_uint4(gw[0], hw[0], gw[1], hw[1]);
    }
    if (lane == 0) {
        if (D4) {
            StripD4 si;
            si.d4[0] = D.d4[0];
            si.d4[1] = D.d4[1];
            si.out = D.buf[0];
            si.map[0] = D.map[0];
            si.map[1] = D.map[1];
            si.info = D.info;
            si.W = W;
            si.sxy = (uint32_t)sx0 | ((uint32_t)sy0 << 16);
            si.wxy = (uint32_t)c_base | ((uint32_t)r_base << 16);
            si.misc = (uint32_t)nvalid << 8;
            static_cast<StripD4 *>(sinfo)[g] = si;
        } else {
            StripInfo si;
            si.buf[0] = D.buf[0];
            si.buf[1] = D.buf[1];
            si.W = W;
            si.sxy = (uint32_t)sx0 | ((uint32_t)sy0 << 16);
            si.axy = (uint32_t)ax0 | ((uint32_t)ry0 << 16);
            si.misc = (uint32_t)((ax1 - ax0) >> 4) | ((uint32_t)nvalid << 8) | ((centred ? 1u : 0u) << 16);
            static_cast<StripInfo *>(sinfo)[g] = si;
        }
    }
}

template <int BMAX, bool D4>
__global__ void __launch_bounds__(kDecWarps * 32)
    decode_setup_kernel(const DecDesc *__restrict__ descs, int count, int total_strips, void *sinfo, uint4 *tfw,
                        uint4 *tgw, int first_kind, uint32_t *bar) {
    __shared__ int s_base[kImgTable];
    __shared__ uint4 s_recs[kDecWarps][64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the descriptors come from the host (uploaded when the plan was made)
    if (count <= kImgTable)
        for (int i = threadIdx.x; i < count; i += blockDim.x) s_base[i] = descs[i].strip_base;
    // Programmatic dependent launch: the table above may be built while the
    // previous kernel (the stream packer, or whatever wrote the records)
    // finishes; nothing of the decode's workspace or of its inputs is read
    // or written before that kernel has completed.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (bar && blockIdx.x == 0 && threadIdx.x == 0) {
        bar[0] = 0u;  // grid-barrier words of the single-launch iterations
        bar[1] = 0u;
    }
    __syncthreads();
    const int gwarps = gridDim.x * kDecWarps;
    for (int g = blockIdx.x * kDecWarps + warp; g < total_strips; g += gwarps)
        setup_strip<BMAX, D4>(descs, count, s_base, g, s_recs[warp], sinfo, tfw, tgw, first_kind, lane);
}

// First iteration from x0 = 128: d4 - mean d4 = 0, every pixel is its
// transform's luminance (clamped).
template <int BMAX>
__device__ __forceinline__ void first_strip(const StripInfo &si, uint4 tf, int src_sel, int lane) {
    using G = DGeom<BMAX>;
    constexpr int PC = G::PC;
    const int pr = lane / PC, pc = lane % PC;
    const int sx0 = (int)(si.sxy & 0xffffu), sy0 = (int)(si.sxy >> 16);
    const int nvalid = (int)((si.misc >> 8) & 0xffu);
    if ((8 * pc) / BMAX >= nvalid) return;
    uint8_t *out = const_cast<uint8_t *>(src_sel ? si.buf[0] : si.buf[1]) + (size_t)(sy0 + 4 * pr) * si.W + sx0 + 8 * pc;
    const int O0 = (int)tf.y, O1 = (int)tf.w;
    const uint32_t w0 = pack_sat_u8(O0, O0, pack_sat_u8(O0, O0, 0u));
    const uint32_t w1 = pack_sat_u8(O1, O1, pack_sat_u8(O1, O1, 0u));
#pragma unroll
    for (int i = 0; i < 4; ++i) *reinterpret_cast<uint2 *>(out + (size_t)i * si.W) = make_uint2(w0, w1);
}

// Decimated domain values (16 per half-patch, packed pairs) of centred
// transforms, read from the staged window, and the halves' partial Sd4.
template <int BMAX>
__device__ __forceinline__ void load_centred(const uint32_t (&fw)[2], const uint32_t *d4e, uint32_t (&dv)[2][4][2],
                                             int (&part)[2], int key) {
    constexpr int NP = DGeom<BMAX>::NP;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = (int)(fw[h] & 0xffu), rr = (int)((fw[h] >> 8) & 0xffu);
        const uint32_t *base = d4e + rr * NP + (c >> 1);
        const uint32_t *bk = base + key, *bn = base + (key ^ 1);
        const bool odd = c & 1;
        // the pair at 16-bit offset `odd` of (e1:e0) and of (e2:e1) by byte
        // permutes; (t0, t1) hold (e0, e1), or (e1, e0) when key is set
        const uint32_t s0 = key ? (odd ? 0x1076u : 0x7654u) : (odd ? 0x5432u : 0x3210u);
        const uint32_t s1 = odd ? 0x5432u : 0x3210u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t t0 = bk[i * NP], t1 = bn[i * NP];
            const uint32_t t2 = odd ? base[i * NP + 2] : 0u;
            const uint32_t e1 = key ? t0 : t1;
            dv[h][i][0] = __byte_perm(t0, t1, s0);
            dv[h][i][1] = __byte_perm(e1, t2, s1);
        }
        uint32_t pk = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) pk += dv[h][i][0] + dv[h][i][1];
        part[h] = (int)((pk & 0xffffu) + (pk >> 16));
    }
}

// Output pixels of both half-patches, rows packed 4 per word: Sd4 per
// transform (halves of one lane first for sides >= 8, then the lane group
// of the transform; every lane runs the same shuffles), then
// p = (c d4 + K) >> 9 with K = floor((512 n O - c Sd4 + 256 n) / n).
template <int BMAX>
__device__ __forceinline__ void transform_rows(const uint32_t (&fw)[2], const int (&Ov)[2],
                                               const uint32_t (&dv)[2][4][2], const int (&part)[2],
                                               uint32_t (&w)[4][2]) {
    constexpr int PC = DGeom<BMAX>::PC;
    const unsigned FULL = 0xffffffffu;
    const int lg0 = (int)((fw[0] >> 16) & 0xffu), lg1 = (int)((fw[1] >> 16) & 0xffu);
    int sd4[2];
    {
        const bool big = lg0 >= 3;  // a transform of side >= 8 covers both halves
        const int B = 1 << lg0;
        const int gx = big ? B / 8 : 1, gy = big ? B / 4 : 1;
        int v = part[0] + part[1];
        if (BMAX == 32 && __all_sync(FULL, lg0 == 5)) {
            // one transform covers the whole strip (a 32x32 leaf): one reduction
            v = __reduce_add_sync(FULL, v);
        } else {
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
        }
        sd4[0] = big ? v : part[0];
        sd4[1] = big ? v : part[1];
    }
    int K[2], cb0[2], cb1[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int lg2n = 2 * (h ? lg1 : lg0);
        const int c = (int)(int8_t)(fw[h] >> 24);
        K[h] = (Ov[h] * (1 << (9 + lg2n)) + (1 << (8 + lg2n)) - c * sd4[h]) >> lg2n;
        cb0[h] = (int)(fw[h] >> 24);
        cb1[h] = (int)((fw[h] >> 24) << 8);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        w[i][0] = row_pixels(dv[0][i][0], dv[0][i][1], cb0[0], cb1[0], K[0]);
        w[i][1] = row_pixels(dv[1][i][0], dv[1][i][1], cb0[1], cb1[1], K[1]);
    }
}

// One strip of one iteration after the first; for centred domains the
// decimated window of the previous iterate is already staged in d4e.
template <int BMAX>
__device__ __forceinline__ void iterate_strip(const StripInfo &si, uint4 tf, const uint4 *__restrict__ tgw_row,
                                              int src_sel, const uint32_t *d4e, int lane) {
    using G = DGeom<BMAX>;
    constexpr int PC = G::PC;
    const int pr = lane / PC, pc = lane % PC;
    const int W = si.W;
    const int sx0 = (int)(si.sxy & 0xffffu), sy0 = (int)(si.sxy >> 16);
    const int nvalid = (int)((si.misc >> 8) & 0xffu);
    const bool centred = (si.misc >> 16) & 1u;
    const bool valid = (8 * pc) / BMAX < nvalid;
    const uint8_t *src = src_sel ? si.buf[1] : si.buf[0];
    uint8_t *out = const_cast<uint8_t *>(src_sel ? si.buf[0] : si.buf[1]) + (size_t)(sy0 + 4 * pr) * W + sx0 + 8 * pc;
    const uint32_t fw[2] = {tf.x, tf.z};
    const int Ov[2] = {(int)tf.y, (int)tf.w};

    uint32_t dv[2][4][2];  // [half][row][pair]
    int part[2] = {0, 0};
    if (!valid) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < 4; ++i) dv[h][i][0] = dv[h][i][1] = 0u;
    } else if (centred) {
        load_centred<BMAX>(fw, d4e, dv, part, G::bank_key(pr));
    } else {
        // domains outside the window (local / exhaustive search, isometries)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 gg = tgw_row[lane];
            const uint32_t gd = h ? gg.z : gg.x, ge = h ? gg.w : gg.y;
            const int dx = (int)(gd & 0xffffu), dy = (int)(gd >> 16);
            const int u0 = (int)(ge & 0xffu), v0 = (int)((ge >> 8) & 0xffu), iso = (int)((ge >> 16) & 0xffu);
            const int B = 1 << ((fw[h] >> 16) & 0xffu);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t vals[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    int su, sv;
                    iso_src(iso, B, u0 + e, v0 + i, su, sv);
                    const uint8_t *p = src + (size_t)(dy + 2 * sv) * W + dx + 2 * su;
                    vals[e] = (uint32_t)p[0] + p[1] + p[W] + p[W + 1];
                }
                dv[h][i][0] = vals[0] | (vals[1] << 16);
                dv[h][i][1] = vals[2] | (vals[3] << 16);
            }
            uint32_t pk = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) pk += dv[h][i][0] + dv[h][i][1];
            part[h] = (int)((pk & 0xffffu) + (pk >> 16));
        }
    }
    uint32_t w[4][2];
    transform_rows<BMAX>(fw, Ov, dv, part, w);
    if (valid) {
#pragma unroll
        for (int i = 0; i < 4; ++i) *reinterpret_cast<uint2 *>(out + (size_t)i * W) = make_uint2(w[i][0], w[i][1]);
    }
}

template <int BMAX>
__global__ void __launch_bounds__(kDecWarps * 32, 4)
    decode_iter_kernel(const StripInfo *__restrict__ sinfo, const uint4 *__restrict__ tfw,
                       const uint4 *__restrict__ tgw, int total_strips, int src_sel, int first) {
    using G = DGeom<BMAX>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *d4e = reinterpret_cast<uint32_t *>(smem) + warp * G::WORDS;
    const int gwarps = gridDim.x * kDecWarps;
    for (int g = blockIdx.x * kDecWarps + warp; g < total_strips; g += gwarps) {
        const StripInfo si = sinfo[g];
        const uint4 tf = tfw[(size_t)g * 32 + lane];
        if (first) {
            first_strip<BMAX>(si, tf, src_sel, lane);
            continue;
        }
        __syncwarp();
        if ((si.misc >> 16) & 1u)
            stage_window<BMAX, G::UPR, G::NP>(src_sel ? si.buf[1] : si.buf[0], si.W, (int)(si.axy >> 16), (int)(si.axy & 0xffffu),
                                              (int)(si.misc & 0xffu), d4e, lane);
        __syncwarp();
        iterate_strip<BMAX>(si, tf, tgw + (size_t)g * 32, src_sel, d4e, lane);
    }
}

// ---------------------------------------------------------------------------
// 2x2-sum iteration for centred streams (no-search / MNS).
//
// A centred domain starts at even coordinates (x - B/2 with B >= 4, clamped
// to the even W - 2B), so every decimated value the decoder reads is a value
// of the previous iterate's 2x2-sum image on the even grid.  Between the
// first and the last iteration the decoder therefore keeps that (W/2) x (H/2)
// uint16 image instead of the pixels: an iteration fetches the strip's window
// of 2x2 sums by TMA straight into the layout the lanes read (no decimation
// pass), computes the output pixels exactly as above, and stores the 2x2
// sums of those clamped pixels -- the values the next iteration would form
// from them.  Only the last iteration writes pixels.  Each warp prefetches
// its next strip's window into a second buffer while it computes.

template <int BMAX>
__device__ __forceinline__ void iterate_d4(uint4 tf, const uint32_t *win, uint16_t *d4o, int W, bool last,
                                           const StripD4 *sp, int lane) {
    constexpr int PC = DGeom<BMAX>::PC;
    const int pr = lane / PC, pc = lane % PC;
    const bool valid = tf.w != kNoLane;
    const uint32_t fw[2] = {tf.x, tf.y};
    const int Ov[2] = {lum16(tf.z, 0), lum16(tf.z, 1)};
    uint32_t dv[2][4][2];
    int part[2] = {0, 0};
    if (valid) {
        load_centred<BMAX>(fw, win, dv, part, DGeom<BMAX>::bank_key(pr));
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < 4; ++i) dv[h][i][0] = dv[h][i][1] = 0u;
    }
    uint32_t w[4][2];
    transform_rows<BMAX>(fw, Ov, dv, part, w);
    if (!valid) return;
    if (last) {
        const uint32_t sxy = sp->sxy;
        const int sx0 = (int)(sxy & 0xffffu), sy0 = (int)(sxy >> 16);
        uint8_t *out = sp->out + (size_t)(sy0 + 4 * pr) * W + sx0 + 8 * pc;
#pragma unroll
        for (int i = 0; i < 4; ++i) *reinterpret_cast<uint2 *>(out + (size_t)i * W) = make_uint2(w[i][0], w[i][1]);
    } else {
        const int W2 = W >> 1;
        uint16_t *o = d4o + tf.w;
#pragma unroll
        for (int j = 0; j < 2; ++j)
            *reinterpret_cast<uint2 *>(o + (size_t)j * W2) =
                make_uint2(sum2x2(w[2 * j][0], w[2 * j + 1][0]), sum2x2(w[2 * j][1], w[2 * j + 1][1]));
    }
}

// Window double buffer of one warp across the iterations of a launch: the
// buffer the next copy lands in and the phase each buffer's barrier waits for.
struct D4Ring {
    uint32_t par0 = 0, par1 = 0;
    int b = 0;
};

// One iteration over this warp's strips (strips g, g + gstep, ...): reads the
// 2x2-sum image `src`, writes the other one (or the pixels when `last`).
// Lane 0 loads the box coordinates of a strip two strips ahead and issues
// each window copy one strip ahead, so that issuing never waits on a global
// load.  With PDL the previous kernel's output is read only after
// griddepcontrol.wait.  Returns false if a copy did not land (the stream's
// error bit is raised and the warp's copies in flight are waited for, bounded).
template <int BMAX, bool PDL>
__device__ __forceinline__ bool d4_pass(const StripD4 *__restrict__ sinfo, const uint4 *__restrict__ tfw,
                                        int total_strips, int g, int gstep, int src, bool last, bool after_setup,
                                        uint32_t *win0, uint32_t *win1, uint64_t *bar, D4Ring &R, int lane) {
    constexpr uint32_t WB = (uint32_t)DGeom<BMAX>::WORDS * 4u;  // one window: BMAX rows x NP words
    const unsigned FULL = 0xffffffffu;
    const int dst = src ^ 1;
    auto coords = [&](int gi, const TmaMap *&map, uint32_t &wxy) {
        const StripD4 *sn = sinfo + gi;
        map = src ? sn->map[1] : sn->map[0];
        wxy = sn->wxy;
    };
    auto issue = [&](int b, const TmaMap *map, uint32_t wxy) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + b, WB);
        tma_load_2d(b ? win1 : win0, map, (int)(wxy & 0xffffu), (int)(wxy >> 16), bar + b);
    };
    const TmaMap *nmap = nullptr, *m0 = nullptr;
    uint32_t nwxy = 0, w0 = 0;
    // With PDL, everything before griddepcontrol.wait may overlap the
    // previous kernel, whose output is read only after the wait.  The strip
    // tables come from the setup kernel: right after it (`after_setup`) they
    // are that kernel's output and are read after the wait like the rest;
    // in later iterations an earlier iteration's wait has already made them
    // visible, so their first coordinates are fetched before the wait.
    const bool early = !PDL || !after_setup;
    if (early && lane == 0 && g < total_strips) {
        coords(g, m0, w0);
        if (g + gstep < total_strips) coords(g + gstep, nmap, nwxy);
    }
    if (PDL) {
        // the next kernel may be scheduled as this one's CTAs retire
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    if (!early && lane == 0 && g < total_strips) {
        coords(g, m0, w0);
        if (g + gstep < total_strips) coords(g + gstep, nmap, nwxy);
    }
    if (lane == 0 && g < total_strips) issue(R.b, m0, w0);
    for (; g < total_strips; g += gstep) {
        const int gn = g + gstep;
        const int b = R.b;
        const StripD4 *sp = sinfo + g;
        uint16_t *const d4o = dst ? sp->d4[1] : sp->d4[0];
        const int W = sp->W;
        const uint4 tf = tfw[(size_t)g * 32 + lane];
        if (gn < total_strips) {
            if (lane == 0) {
                issue(b ^ 1, nmap, nwxy);
                if (gn + gstep < total_strips) coords(gn + gstep, nmap, nwxy);
            }
        }
        const uint32_t par = b ? R.par1 : R.par0;
        const bool arrived = mbar_wait(bar + b, par, kMbarLimit);
        if (!__all_sync(FULL, arrived)) {
            // give both buffers' copies a bounded chance to land, then leave
            if (lane == 0) {
                raise_error(sp->info, FIC_DEVERR_TIMEOUT);
                mbar_wait(bar + b, par, kMbarLimit);
                if (gn < total_strips) mbar_wait(bar + (b ^ 1), b ? R.par0 : R.par1, kMbarLimit);
            }
            __syncwarp();
            return false;
        }
        if (b) R.par1 ^= 1u;
        else R.par0 ^= 1u;
        iterate_d4<BMAX>(tf, b ? win1 : win0, d4o, W, last, sp, lane);
        __syncwarp();
        R.b = b ^ 1;
    }
    return true;
}

// Per-warp windows of the 2x2-sum kernels (two buffers of BMAX rows x NP
// words, 128-byte aligned) and their barriers.
template <int BMAX>
__device__ __forceinline__ void d4_windows(uint8_t *smem, uint64_t (*s_bar)[2], int warp, int lane, uint32_t *&win0,
                                           uint32_t *&win1) {
    constexpr uint32_t WB = (uint32_t)DGeom<BMAX>::WORDS * 4u;
    uint8_t *base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    win0 = reinterpret_cast<uint32_t *>(base + (size_t)(2 * warp) * WB);
    win1 = reinterpret_cast<uint32_t *>(base + (size_t)(2 * warp + 1) * WB);
    if (lane == 0) {
        mbar_init(&s_bar[warp][0], 1);
        mbar_init(&s_bar[warp][1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// One iteration after the first (the setup kernel writes the first).  kind
// bit 1: the last iteration (writes pixels); bit 2: the launch right after
// the setup kernel.  src: the 2x2-sum image read (0/1); the other one is
// written.
template <int BMAX>
__global__ void __launch_bounds__(kDecWarps * 32, 4)
    decode_d4_iter_kernel(const StripD4 *__restrict__ sinfo, const uint4 *__restrict__ tfw, int total_strips, int src,
                          int kind) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar[kDecWarps][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool last = (kind >> 1) & 1, after_setup = (kind >> 2) & 1;
    const int gstep = gridDim.x * kDecWarps;
    const int g = blockIdx.x * kDecWarps + warp;
    uint32_t *win0, *win1;
    d4_windows<BMAX>(smem, s_bar, warp, lane, win0, win1);
    D4Ring R;
    d4_pass<BMAX, true>(sinfo, tfw, total_strips, g, gstep, src, last, after_setup, win0, win1, s_bar[warp], R,
                        lane);
}

// Grid barrier of the single-launch decoder: one arrival per CTA on a
// counter, then a bounded wait until every CTA of the launch has arrived
// `round` times (the grid is co-resident: cooperative launch).  bar[0]:
// arrivals, bar[1]: abort flag (a CTA that failed sets it so that the others
// leave at their next barrier instead of waiting out the limit).  Called by
// one thread per CTA between __syncthreads; false on abort or timeout.
__device__ __forceinline__ bool grid_barrier(uint32_t *bar, uint32_t target) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    for (unsigned n = 0; n < kSpinLimit; ++n) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) return true;
        if (ld_volatile(bar + 1)) return false;
        if (n > 4) __nanosleep(32);
    }
    return false;
}

// All iterations after the first in one cooperative launch: iteration it
// (1 <= it < iters) reads 2x2-sum image (it - 1) & 1 and writes the other,
// the last one writes the pixels; a grid barrier separates iterations (every
// write of one iteration before any read of the next, every read of one
// before the next overwrites its source).  The same strips stay with the
// same warp throughout, and the launches and grid ramps of the
// one-launch-per-iteration schedule are saved.  bar[0..1] are zeroed by the
// setup kernel.
template <int BMAX>
__global__ void __launch_bounds__(kDecWarps * 32, 4)
    decode_d4_loop_kernel(const StripD4 *__restrict__ sinfo, const uint4 *__restrict__ tfw, int total_strips,
                          int iters, uint32_t *bar) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar[kDecWarps][2];
    __shared__ int s_abort;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gstep = gridDim.x * kDecWarps;
    const int g0 = blockIdx.x * kDecWarps + warp;
    if (threadIdx.x == 0) s_abort = 0;
    uint32_t *win0, *win1;
    d4_windows<BMAX>(smem, s_bar, warp, lane, win0, win1);
    D4Ring R;
    uint32_t target = 0;
    for (int it = 1; it < iters; ++it) {
        const bool last = it == iters - 1;
        if (!d4_pass<BMAX, false>(sinfo, tfw, total_strips, g0, gstep, (it - 1) & 1, last, false, win0, win1,
                                  s_bar[warp], R, lane) &&
            lane == 0)
            atomicExch(&s_abort, 1);
        if (last) break;
        // this thread's stores (generic proxy) before the next iteration's
        // window copies (async proxy) on any SM
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_abort) st_volatile(bar + 1, 1u);
            target += gridDim.x;
            if (!grid_barrier(bar, target)) {
                st_volatile(bar + 1, 1u);
                s_abort = 1;
            }
        }
        __syncthreads();
        if (s_abort) {
            // every stream with a strip here learns that the decode stopped
            if (lane == 0)
                for (int g = g0; g < total_strips; g += gstep) raise_error(sinfo[g].info, FIC_DEVERR_TIMEOUT);
            return;
        }
        if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
    }
}

size_t decode_d4_smem_bytes(int bmax) {
    const int words = bmax == 32 ? DGeom<32>::WORDS : (bmax == 16 ? DGeom<16>::WORDS : DGeom<8>::WORDS);
    return (size_t)kDecWarps * 2 * words * sizeof(uint32_t) + 128;
}

// Box width (in 2x2 sums) of the decoder's window loads.
int decode_d4_box(int bmax) { return 2 * (bmax == 32 ? DGeom<32>::NP : (bmax == 16 ? DGeom<16>::NP : DGeom<8>::NP)); }

size_t decode_table_bytes_per_strip() { return sizeof(StripInfo) + 2 * 32 * sizeof(uint4); }

size_t decode_smem_bytes(int bmax) {
    int words = bmax == 32 ? DGeom<32>::WORDS : (bmax == 16 ? DGeom<16>::WORDS : DGeom<8>::WORDS);
    return (size_t)kDecWarps * words * sizeof(uint32_t);
}

// Decode: the table setup kernel, then one launch per iteration.
template <int BMAX>
static cudaError_t dlaunch_t(const DecDesc *descs, int count, int total_strips, void *tables, int iters, bool d4,
                             const DecTune &tune, cudaStream_t st) {
    // launch facts per kernel and device (the iteration kernels also get their shared-memory limit)
    static KernelSlots ks_setup_d4, ks_setup_px, ks_iter, ks_d4, ks_loop;
    const size_t smem = decode_smem_bytes(BMAX), smem_d4 = decode_d4_smem_bytes(BMAX);
    int sms = 0, per = 0;
    const size_t info_bytes = d4 ? sizeof(StripD4) : sizeof(StripInfo);
    uint4 *tfw = reinterpret_cast<uint4 *>(static_cast<uint8_t *>(tables) + info_bytes * (size_t)total_strips);
    uint4 *tgw = tfw + (size_t)total_strips * 32;
    const int need = (total_strips + kDecWarps - 1) / kDecWarps;
    // the 2x2-sum path keeps no far-domain words: its grid-barrier words sit there
    const bool single = d4 && tune.single_launch && iters >= 2;
    uint32_t *bar = single ? reinterpret_cast<uint32_t *>(tgw) : nullptr;
    if (d4) {
        cudaError_t e = kernel_slots(ks_setup_d4, (const void *)decode_setup_kernel<BMAX, true>, kDecWarps * 32, 0,
                                     sms, per);
        if (e != cudaSuccess) return e;
        const int gs = sms * per;
        // the setup kernel also writes the first iterate (pixels when it is the only one)
        e = launch_pdl(decode_setup_kernel<BMAX, true>, need < gs ? need : gs, kDecWarps * 32, 0, st, descs, count,
                       total_strips, tables, tfw, tgw, iters == 1 ? 3 : 1, bar);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = kernel_slots(ks_setup_px, (const void *)decode_setup_kernel<BMAX, false>, kDecWarps * 32, 0,
                                     sms, per);
        if (e != cudaSuccess) return e;
        const int gs = sms * per;
        e = launch_pdl(decode_setup_kernel<BMAX, false>, need < gs ? need : gs, kDecWarps * 32, 0, st, descs, count,
                       total_strips, tables, tfw, tgw, 0, (uint32_t *)nullptr);
        if (e != cudaSuccess) return e;
    }
    stage_mark(st, "decode_setup_kernel");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (single) {
        // iterations 1 .. iters-1 in one cooperative launch (grid barriers
        // between iterations need every CTA resident)
        const StripD4 *sinfo = static_cast<const StripD4 *>(tables);
        e = kernel_slots(ks_loop, (const void *)decode_d4_loop_kernel<BMAX>, kDecWarps * 32, smem_d4, sms, per);
        if (e != cudaSuccess) return e;
        const int k = tune.ctas_per_sm > 0 && tune.ctas_per_sm < per ? tune.ctas_per_sm : per;
        const int grid = need < sms * k ? need : sms * k;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kDecWarps * 32);
        cfg.dynamicSmemBytes = smem_d4;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, decode_d4_loop_kernel<BMAX>, sinfo, (const uint4 *)tfw, total_strips, iters, bar);
        stage_mark(st, "decode_d4_loop_kernel");
        if (e == cudaSuccess) e = cudaGetLastError();
        return e;
    }
    if (d4) {
        const StripD4 *sinfo = static_cast<const StripD4 *>(tables);
        e = kernel_slots(ks_d4, (const void *)decode_d4_iter_kernel<BMAX>, kDecWarps * 32, smem_d4, sms, per);
        if (e != cudaSuccess) return e;
        const int k = tune.ctas_per_sm > 0 && tune.ctas_per_sm < per ? tune.ctas_per_sm : per;
        const int grid = need < sms * k ? need : sms * k;
        // iterations are launched as programmatic dependents of the previous
        // kernel (their prologue overlaps its tail; see the kernel)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kDecWarps * 32);
        cfg.dynamicSmemBytes = smem_d4;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        for (int it = 1; it < iters; ++it) {
            // iteration it >= 1 reads image (it - 1) & 1; the first (in the setup kernel) wrote image 0
            const int kind = (it == iters - 1 ? 2 : 0) | (it == 1 ? 4 : 0);
            e = cudaLaunchKernelEx(&cfg, decode_d4_iter_kernel<BMAX>, sinfo, (const uint4 *)tfw, total_strips,
                                   (it - 1) & 1, kind);
            stage_mark(st, "decode_d4_iter_kernel");
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const StripInfo *sinfo = static_cast<const StripInfo *>(tables);
    e = kernel_slots(ks_iter, (const void *)decode_iter_kernel<BMAX>, kDecWarps * 32, smem, sms, per);
    if (e != cudaSuccess) return e;
    const int k = tune.ctas_per_sm > 0 && tune.ctas_per_sm < per ? tune.ctas_per_sm : per;
    const int gi = sms * k;
    const int grid = need < gi ? need : gi;
    for (int it = 0; it < iters; ++it) {
        const int src_sel = (iters - it) & 1;  // the last iteration writes buf[0] (the output)
        decode_iter_kernel<BMAX><<<grid, kDecWarps * 32, smem, st>>>(sinfo, tfw, tgw, total_strips, src_sel, it == 0);
        stage_mark(st, "decode_iter_kernel");
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Transform-per-thread iteration, for streams whose leaves go down to 2 x 2
// pixels (the paper's 16 -> 2 quadtree; the strip kernels above assume every
// 4 x 4 half-patch is covered by one transform).  One thread applies one
// stored transform (a phase-2 leaf: its four sub-block transforms, eq. (1))
// to the previous iterate: Sd4 over its decimated domain, then every pixel
// p = clamp(floor((512 n O + c (n d4 - Sd4) + 256 n) / (512 n))), the same
// fixed-point rule as the strip kernels.  Leaves tile the image, so every
// pixel of the next iterate is written.  Transforms whose range or domain
// would leave the image are skipped (a stream from the encoder has none).
__device__ __forceinline__ int d4_at(const uint8_t *x, int W, int px, int py) {
    const uint8_t *p = x + (size_t)py * W + px;
    return (int)p[0] + (int)p[1] + (int)p[W] + (int)p[W + 1];
}

__device__ void apply_leaf_transform(const uint8_t *__restrict__ x, uint8_t *__restrict__ y, int W, int H, int rx,
                                     int ry, int B, int dx, int dy, int iso, int c, int O) {
    if (rx < 0 || ry < 0 || rx + B > W || ry + B > H || dx < 0 || dy < 0 || dx + 2 * B > W || dy + 2 * B > H) return;
    const int lgB = 31 - __clz(B);
    const long long n = (long long)B * B;
    long long sd = 0;
    for (int v = 0; v < B; ++v)
        for (int u = 0; u < B; ++u) sd += d4_at(x, W, dx + 2 * u, dy + 2 * v);
    const long long base = 512 * n * O - (long long)c * sd + 256 * n;
    for (int v = 0; v < B; ++v) {
        for (int u = 0; u < B; ++u) {
            int su, sv;
            iso_src(iso, B, u, v, su, sv);
            const long long num = base + (long long)c * n * d4_at(x, W, dx + 2 * su, dy + 2 * sv);
            long long pix = num >> (9 + 2 * lgB);  // 512 n is a power of two: floor division
            pix = pix < 0 ? 0 : (pix > 255 ? 255 : pix);
            y[(size_t)(ry + v) * W + rx + u] = (uint8_t)pix;
        }
    }
}

__global__ void __launch_bounds__(256)
    decode_leaf_kernel(const DecDesc *__restrict__ descs, int src) {
    const DecDesc &D = descs[blockIdx.y];
    const int nrec = (int)D.tile_off[D.tw * D.th];
    const uint8_t *x = D.buf[src];
    uint8_t *y = D.buf[src ^ 1];
    const int bmax = D.W / D.tw, ko1 = (1 << D.o_bits) - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nrec; i += gridDim.x * blockDim.x) {
        const uint4 r = *reinterpret_cast<const uint4 *>(D.rec + i);
        const int rx = (int)(r.x & 0xffffu), ry = (int)(r.x >> 16);
        const int level = (int)(r.y & 0xffu), phase = (int)((r.y >> 8) & 0xffu);
        const int k = (int)((r.y >> 16) & 0xffu), q = (int)(r.y >> 24);
        const int iso = (int)(r.z >> 24);
        const int dx = (int)(r.w & 0xffffu), dy = (int)(r.w >> 16);
        if (level < 1 || level > D.L) continue;
        const int B = bmax >> (level - 1);
        const int O = (int)__umulhi((uint32_t)(510 * q + ko1), c_lum_magic[D.o_bits]);  // L(q)
        if (phase == 1) {
            apply_leaf_transform(x, y, D.W, D.H, rx, ry, B, dx, dy, iso, contrast_code(k, D.s_bits), O);
        } else {
            const int h = B / 2;
            const int d0 = (int)(int8_t)(r.z & 0xffu), d1 = (int)(int8_t)((r.z >> 8) & 0xffu);
            const int d2 = (int)(int8_t)((r.z >> 16) & 0xffu);
            const int Ok[4] = {O + d0, O + d1, O + d2, O - (d0 + d1 + d2)};  // eq. (1)
            for (int sb = 0; sb < 4; ++sb) {
                const int sx = rx + (sb & 1) * h, sy = ry + (sb >> 1) * h;
                int sdx, sdy;
                if (D.phase2_domain) {
                    sdx = centred_origin(rx, B, D.W) + (sb & 1) * B;
                    sdy = centred_origin(ry, B, D.H) + (sb >> 1) * B;
                } else {
                    sdx = centred_origin(sx, h, D.W);
                    sdy = centred_origin(sy, h, D.H);
                }
                apply_leaf_transform(x, y, D.W, D.H, sx, sy, h, sdx, sdy, 0, phase2_code(level, (k >> sb) & 1),
                                     Ok[sb]);
            }
        }
    }
}

// `hdec`: the host copy of the descriptors (the iterate buffers of the
// memset); `max_recs`: the largest record capacity of the batch.
cudaError_t launch_decode_leaves(const DecDesc *d_descs, const DecDesc *hdec, int count, int max_recs, int iters,
                                 cudaStream_t st) {
    if (iters < 1 || count < 1 || count > 65535) return cudaErrorInvalidValue;
    // iteration t writes buffer (iters - 1 - t) & 1: the last one writes buf[0]
    const int first_src = ((iters - 1) & 1) ^ 1;
    for (int i = 0; i < count; ++i) {
        const cudaError_t e =
            cudaMemsetAsync(hdec[i].buf[first_src], 128, (size_t)hdec[i].W * (size_t)hdec[i].H, st);
        if (e != cudaSuccess) return e;
    }
    int gx = (max_recs + 255) / 256;
    gx = gx < 1 ? 1 : (gx > 4096 ? 4096 : gx);
    for (int t = 0; t < iters; ++t) {
        const int src = ((iters - 1 - t) & 1) ^ 1;
        decode_leaf_kernel<<<dim3(gx, count), 256, 0, st>>>(d_descs, src);
        stage_mark(st, "decode_leaf_kernel");
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_decode(int bmax, const DecDesc *d_descs, int count, int total_strips, void *tables, int iters,
                          bool d4, const DecTune &tune, cudaStream_t st) {
    switch (bmax) {
    case 32: return dlaunch_t<32>(d_descs, count, total_strips, tables, iters, d4, tune, st);
    case 16: return dlaunch_t<16>(d_descs, count, total_strips, tables, iters, d4, tune, st);
    case 8: return dlaunch_t<8>(d_descs, count, total_strips, tables, iters, d4, tune, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fic
