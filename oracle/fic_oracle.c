/*
 * fic_oracle.c -- TEST INFRASTRUCTURE: the CPU oracle of the fractal coder.
 *
 * This is a plain, slow and deliberately unoptimised restatement of the
 * modified no-search (MNS) fractal encoder of Salarian, Mohamadinia and
 * Rasekhi ("A Modified No Search Algorithm for Fractal Image Compression"),
 * of the comparison modes it is measured against (no-search, local search,
 * exhaustive search with isometries) and of an iterated decoder.  It exists
 * only so that tests, the smoke check and the benchmark's CPU-baseline leg
 * can check and time the CUDA library; the product path never calls it and
 * it shares no code, header or table with the CUDA sources.
 *
 * Everything is integer arithmetic (int64 where needed) so that results are
 * exact.  Wherever the paper is silent the reading taken is stated at the
 * function that implements it.
 *
 * Notation (paper Section 1 and 3): a range block R is B x B pixels of the
 * image, a domain block D is 2B x 2B and is reduced to B x B by the mean of
 * every 2x2 group of pixels ("mean filter to four neighbor pixels",
 * Section 3).  Here that mean is kept as the integer 2x2 SUM d4 = 4*mean, so
 * that all moments stay integers.  n = B*B.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NOSEARCH 0
#define ORC_MNS 1
#define ORC_LOCAL 2
#define ORC_EXHAUSTIVE 3

#define ORC_OK 0
#define ORC_EBADSIZE -1
#define ORC_EBADPARAM -2
#define ORC_ECAPACITY -3
#define ORC_ENOMEM -4

typedef struct {
    int32_t mode;
    int32_t bmax, bmin;
    double thr_rms[4];
    int32_t s_bits, o_bits;
    int32_t phase2;
    int32_t local_radius, local_step;
    int32_t dom_step;
    int32_t isometries;
    int32_t phase2_domain; /* 0: sub-blocks use their own centred domains; 1: the
                              quadrants of the parent's (alternative reading) */
} orc_params;

/* One leaf of the quadtree, i.e. one stored transform (16 bytes). */
typedef struct {
    uint16_t x, y;     /* range top-left, pixels */
    uint8_t level;     /* 1 = largest block */
    uint8_t phase;     /* 1 = phase-1 transform, 2 = phase-2 group of four */
    uint8_t k;         /* phase 1: contrast code; phase 2: the four 1-bit choices */
    uint8_t q;         /* luminance code (phase 2: the block mean code q_i) */
    int8_t d[3];       /* phase 2: O_k - O_i for sub-blocks 1..3 */
    uint8_t iso;       /* isometry applied to the decimated domain */
    uint16_t dx, dy;   /* domain top-left, pixels */
} orc_leaf;

typedef struct {
    int64_t sr, srr, sd, sdd, sdr;
} orc_moments;

/* ------------------------------------------------------------------ */
/* Small integer helpers                                                */

static int64_t floor_div(int64_t a, int64_t b) {
    /* floor(a / b) for b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int ilog2_ceil(long v) {
    int b = 0;
    while ((1L << b) < v) b++;
    return b;
}

/* ------------------------------------------------------------------ */
/* Codebooks (Section 3.3 stores a quantised contrast and luminance)    */

/* Contrast s is coded on 2^s_bits uniform cells of [-1, 1); the code is the
 * cell midpoint, so |s| <= 1 - 1/2^s_bits < 1 (contractive).  Kept in fixed
 * point c = 128*s: c_k = (2k - (K-1)) * (128/K), K = 2^s_bits.  With 5 bits
 * this is c_k = 4(2k - 31), k = 0..31. */
int64_t orc_contrast(int k, int s_bits) {
    int K = 1 << s_bits;
    return (int64_t)(2 * k - (K - 1)) * (128 / K);
}

/* Luminance (offset) codes: 2^o_bits levels spread over 0..255,
 * L(q) = round(255 q / (Ko-1)).  With 7 bits, L(q) = floor((510q+127)/254);
 * with 8 bits, L(q) = q. */
int64_t orc_luminance(int q, int o_bits) {
    int64_t Ko1 = (1 << o_bits) - 1;
    return (510 * (int64_t)q + Ko1) / (2 * Ko1);
}

/* Phase-2 contrast sets (Section 3.2): {.2,.5} at level 1, {.4,.65} at
 * level 2, {.5,.9} at level 3, in the same fixed point c = round(128 s). */
int64_t orc_phase2_contrast(int level, int bit) {
    static const int64_t sets[3][2] = {{26, 64}, {51, 83}, {64, 115}};
    return sets[level - 1][bit];
}

/* Bits for the signed mean differences O_k - O_i (Section 3.3: five bits at
 * the first level, six at the other levels, one of them the sign). */
int orc_phase2_mbits(int level) { return level == 1 ? 5 : 6; }

/* ------------------------------------------------------------------ */
/* Geometry                                                             */

/* Number of range blocks of side n in an N x N image, (N/n)^2, and of
 * domain blocks of side 2n when every position is allowed, (N-2n+1)^2
 * (Section 1). */
int64_t orc_count_ranges(int W, int H, int n) { return (int64_t)(W / n) * (H / n); }
int64_t orc_count_domains(int W, int H, int n, int step) {
    if (2 * n > W || 2 * n > H) return 0;
    return (int64_t)((W - 2 * n) / step + 1) * ((H - 2 * n) / step + 1);
}

/* The no-search domain: the 2B x 2B block that has the same centre as the
 * range (Section 3, "take the domain block with the same center of the range
 * one"; Fig. 1b).  The paper does not say what happens at the image border;
 * the block is shifted inside the image (clamped). */
int orc_centred(int x, int B, int W) { return clampi(x - B / 2, 0, W - 2 * B); }

/* Isometry applied to a B x B decimated domain block: the transformed block
 * at (u, v) (column u, row v) takes the source element returned here.
 * 0 identity, 1 rotation by 90 degrees (clockwise), 2 rotation by 180,
 * 3 rotation by 270, 4 mirror across the vertical axis, 5 mirror across the
 * horizontal axis, 6 transpose, 7 anti-transpose. */
void orc_iso_source(int iso, int B, int u, int v, int *su, int *sv) {
    int m = B - 1;
    switch (iso) {
    case 0: *su = u;     *sv = v;     break;
    case 1: *su = v;     *sv = m - u; break;
    case 2: *su = m - u; *sv = m - v; break;
    case 3: *su = m - v; *sv = u;     break;
    case 4: *su = m - u; *sv = v;     break;
    case 5: *su = u;     *sv = m - v; break;
    case 6: *su = v;     *sv = u;     break;
    default: *su = m - v; *sv = m - u; break;
    }
}

/* 2x2 sum of the domain pixels under decimated element (u, v). */
static int64_t d4_at(const uint8_t *img, int W, int dx, int dy, int u, int v) {
    const uint8_t *p = img + (size_t)(dy + 2 * v) * W + (dx + 2 * u);
    return (int64_t)p[0] + p[1] + p[W] + p[W + 1];
}

/* Moments of one range/domain pair: sums of r, r^2, d4, d4^2 and r*d4 over
 * the n = B*B pixel pairs (the quantities a least-squares affine fit of D
 * to R needs, Section 1 and 3). */
void orc_moments_of(const uint8_t *img, int W, int x, int y, int B, int dx, int dy,
                    int iso, orc_moments *m) {
    memset(m, 0, sizeof(*m));
    for (int v = 0; v < B; v++) {
        for (int u = 0; u < B; u++) {
            int64_t r = img[(size_t)(y + v) * W + (x + u)];
            int su, sv;
            orc_iso_source(iso, B, u, v, &su, &sv);
            int64_t d = d4_at(img, W, dx, dy, su, sv);
            m->sr += r;
            m->srr += r * r;
            m->sd += d;
            m->sdd += d * d;
            m->sdr += r * d;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Collage error of a coded transform                                   */

/* The transform maps the decimated domain onto the range as
 *     rhat = O + s * (d - mean(d)),   d = d4 / 4,
 * i.e. the luminance O is the block mean the paper's phase 2 works with
 * (Section 3.1, eq. 1) and only s is searched (Section 3).  With c = 128 s,
 * n*512^2*SSE is the integer
 *     E = 512^2 (n Srr - Sr^2) - 1024 c (n Sdr - Sd Sr)
 *         + c^2 (n Sdd - Sd^2) + 512^2 (Sr - n O)^2.               */
int64_t orc_error(const orc_moments *m, int64_t n, int64_t c, int64_t O) {
    int64_t ncrr = n * m->srr - m->sr * m->sr;
    int64_t ncdr = n * m->sdr - m->sd * m->sr;
    int64_t ncdd = n * m->sdd - m->sd * m->sd;
    int64_t e = m->sr - n * O;
    return 262144 * ncrr - 1024 * c * ncdr + c * c * ncdd + 262144 * e * e;
}

/* Threshold test "error smaller than E_i" (Section 3), with E_i an RMS per
 * pixel: SSE < T^2 n, i.e. E < T^2 n^2 512^2.  T^2 is taken in units of
 * 1/256 (exact for any T that is a multiple of 1/16). */
int64_t orc_threshold(double thr_rms, int64_t n) {
    double t2 = thr_rms * thr_rms * 256.0;
    int64_t t2q = (int64_t)(t2 + 0.5);
    return t2q * n * n * 1024;
}

/* Best phase-1 codes for one pair: the contrast code k and luminance code q
 * that minimise E (Section 3, "find the best value for contrast factor").
 * E separates into a part that depends only on c and a part that depends
 * only on O, so the joint minimum is the pair of separate minima; each is
 * found by scanning its whole codebook.  Ties: smaller |c|, then c > 0;
 * smaller q. */
void orc_best_codes(const orc_moments *m, int64_t n, int s_bits, int o_bits,
                    int *k_out, int *q_out, int64_t *e_out) {
    int64_t ncdr = n * m->sdr - m->sd * m->sr;
    int64_t ncdd = n * m->sdd - m->sd * m->sd;
    int K = 1 << s_bits, Ko = 1 << o_bits;
    int bk = -1;
    int64_t bg = 0, bc = 0;
    for (int k = 0; k < K; k++) {
        int64_t c = orc_contrast(k, s_bits);
        int64_t g = c * c * ncdd - 1024 * c * ncdr;
        int64_t ac = c < 0 ? -c : c, abc = bc < 0 ? -bc : bc;
        if (bk < 0 || g < bg || (g == bg && (ac < abc || (ac == abc && c > 0)))) {
            bk = k; bg = g; bc = c;
        }
    }
    int bq = -1;
    int64_t bh = 0;
    for (int q = 0; q < Ko; q++) {
        int64_t e = m->sr - n * orc_luminance(q, o_bits);
        int64_t h = e * e;
        if (bq < 0 || h < bh) { bq = q; bh = h; }
    }
    *k_out = bk;
    *q_out = bq;
    *e_out = orc_error(m, n, orc_contrast(bk, s_bits), orc_luminance(bq, o_bits));
}

/* ------------------------------------------------------------------ */
/* Domain search per mode (phase 1)                                     */

typedef struct {
    int k, q, dx, dy, iso;
    int64_t e;
    orc_moments m;
} orc_fit;

static void fit_pair(const uint8_t *img, int W, const orc_params *p, int x, int y, int B,
                     int dx, int dy, int iso, orc_fit *f) {
    orc_moments_of(img, W, x, y, B, dx, dy, iso, &f->m);
    orc_best_codes(&f->m, (int64_t)B * B, p->s_bits, p->o_bits, &f->k, &f->q, &f->e);
    f->dx = dx; f->dy = dy; f->iso = iso;
}

/* Phase-1 search of one range.
 *  no-search / MNS phase 1 (Section 3): the single centred domain;
 *  local search (Section 2): domains around the centred one, offsets in
 *     [-R, R] with step S in x and y (81 candidates for R=16, S=4), those
 *     that leave the image skipped, no isometries;
 *  exhaustive search (Section 1): every domain at a multiple of dom_step,
 *     every isometry.
 * The smallest E wins; ties go to the candidate met first (offset or domain
 * raster order, then isometry).  Returns the number of candidates tried. */
int orc_search(const uint8_t *img, int W, int H, const orc_params *p, int x, int y, int B,
               orc_fit *best) {
    int cx = orc_centred(x, B, W), cy = orc_centred(y, B, H);
    int tried = 0;
    orc_fit f;
    if (p->mode == ORC_NOSEARCH || p->mode == ORC_MNS) {
        fit_pair(img, W, p, x, y, B, cx, cy, 0, best);
        return 1;
    }
    if (p->mode == ORC_LOCAL) {
        int R = p->local_radius, S = p->local_step;
        for (int oy = -R; oy <= R; oy += S) {
            for (int ox = -R; ox <= R; ox += S) {
                int dx = cx + ox, dy = cy + oy;
                if (dx < 0 || dy < 0 || dx + 2 * B > W || dy + 2 * B > H) continue;
                fit_pair(img, W, p, x, y, B, dx, dy, 0, &f);
                if (tried == 0 || f.e < best->e) *best = f;
                tried++;
            }
        }
        return tried;
    }
    /* exhaustive */
    int S = p->dom_step;
    for (int dy = 0; dy + 2 * B <= H; dy += S) {
        for (int dx = 0; dx + 2 * B <= W; dx += S) {
            for (int iso = 0; iso < p->isometries; iso++) {
                fit_pair(img, W, p, x, y, B, dx, dy, iso, &f);
                if (tried == 0 || f.e < best->e) *best = f;
                tried++;
            }
        }
    }
    return tried;
}

/* ------------------------------------------------------------------ */
/* MNS phase 2 (Sections 3.1 - 3.3)                                     */

/* Domain of phase-2 sub-block sb (TL, TR, BL, BR) of block (x, y, B): the
 * paper does not say which domain a sub-block uses.  Reading 0: its own
 * centred domain (the no-search rule at the sub-block size).  Reading 1:
 * the matching quadrant of the parent block's centred domain, i.e. the
 * parent's 2B x 2B domain cut into four B x B quarters. */
static void phase2_domain_of(const orc_params *p, int W, int H, int x, int y, int B, int sb, int *dx, int *dy) {
    int h = B / 2;
    if (p->phase2_domain) {
        *dx = orc_centred(x, B, W) + (sb & 1) * B;
        *dy = orc_centred(y, B, H) + (sb >> 1) * B;
    } else {
        *dx = orc_centred(x + (sb & 1) * h, h, W);
        *dy = orc_centred(y + (sb >> 1) * h, h, H);
    }
}

/* Phase 2 of a block that failed phase 1 at level j < L ("Technique 1").
 * O_i is the block's quantised mean (its phase-1 luminance code q_i).  The
 * four sub-blocks (TL, TR, BL, BR) have means O_k; their differences to O_i
 * are rounded half up to integers and must fit the signed M-bit field of
 * Section 3.3 (|delta| <= 2^(M-1) - 1): that is read as the paper's "small
 * enough".  O_4 is not stored but derived by eq. (1): O_4 = 4 O_i - sum of
 * O_1..O_3.  Each sub-block is fitted to its own centred domain (the
 * no-search rule of Section 3 applied at the sub-block size) with s taken
 * from the level's two-element set (Section 3.2, one bit each).  Phase 2
 * succeeds when every sub-block passes the level's threshold.
 * Returns 1 on success and fills the leaf. */
int orc_phase2(const uint8_t *img, int W, int H, const orc_params *p, int level, int x, int y,
               int B, int q_i, orc_leaf *leaf) {
    int h = B / 2;
    int64_t n4 = (int64_t)h * h;
    int64_t Oi = orc_luminance(q_i, p->o_bits);
    int64_t thr = orc_threshold(p->thr_rms[level - 1], n4);
    int dmax = (1 << (orc_phase2_mbits(level) - 1)) - 1;
    int64_t delta[4];
    orc_moments ms[4];
    for (int sb = 0; sb < 4; sb++) {
        int sx = x + (sb & 1) * h, sy = y + (sb >> 1) * h;
        int dx, dy;
        phase2_domain_of(p, W, H, x, y, B, sb, &dx, &dy);
        orc_moments_of(img, W, sx, sy, h, dx, dy, 0, &ms[sb]);
        /* round-half-up of (mean_k - O_i) = floor((2(Sr_k - n4 O_i) + n4) / (2 n4)) */
        delta[sb] = floor_div(2 * (ms[sb].sr - n4 * Oi) + n4, 2 * n4);
        if (delta[sb] > dmax || delta[sb] < -dmax) return 0;
    }
    int64_t O[4];
    O[0] = Oi + delta[0];
    O[1] = Oi + delta[1];
    O[2] = Oi + delta[2];
    O[3] = 4 * Oi - (O[0] + O[1] + O[2]); /* eq. (1) */
    int bits = 0;
    for (int sb = 0; sb < 4; sb++) {
        int64_t e0 = orc_error(&ms[sb], n4, orc_phase2_contrast(level, 0), O[sb]);
        int64_t e1 = orc_error(&ms[sb], n4, orc_phase2_contrast(level, 1), O[sb]);
        int64_t e = e0;
        if (e1 < e0) { bits |= 1 << sb; e = e1; }
        if (!(e < thr)) return 0;
    }
    leaf->phase = 2;
    leaf->k = (uint8_t)bits;
    leaf->q = (uint8_t)q_i;
    leaf->d[0] = (int8_t)delta[0];
    leaf->d[1] = (int8_t)delta[1];
    leaf->d[2] = (int8_t)delta[2];
    return 1;
}

/* ------------------------------------------------------------------ */
/* Quadtree encoder (Section 3)                                         */

static int nlevels(const orc_params *p) {
    int L = 1;
    for (int b = p->bmax; b > p->bmin; b >>= 1) L++;
    return L;
}

static int is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int orc_check(int W, int H, const orc_params *p) {
    if (!is_pow2(p->bmax) || !is_pow2(p->bmin) || p->bmin < 2 || p->bmin > p->bmax) return ORC_EBADPARAM;
    if (nlevels(p) > 4) return ORC_EBADPARAM;
    if (p->s_bits < 1 || p->s_bits > 7 || p->o_bits < 1 || p->o_bits > 8) return ORC_EBADPARAM;
    if (p->mode < 0 || p->mode > 3) return ORC_EBADPARAM;
    if (p->mode == ORC_LOCAL && (p->local_step <= 0 || p->local_radius < 0)) return ORC_EBADPARAM;
    if (p->mode == ORC_EXHAUSTIVE && (p->dom_step <= 0 || p->isometries < 1 || p->isometries > 8))
        return ORC_EBADPARAM;
    if (W <= 0 || H <= 0 || W % p->bmax || H % p->bmax || W < 2 * p->bmax || H < 2 * p->bmax ||
        W > 65535 || H > 65535)
        return ORC_EBADSIZE;
    return ORC_OK;
}

/* Interleave the bits of (bx, by), x in the low bit: the depth-first order
 * TL, TR, BL, BR of the quadtree. */
static uint32_t morton(uint32_t bx, uint32_t by) {
    uint32_t z = 0;
    for (int b = 0; b < 16; b++) {
        z |= ((bx >> b) & 1u) << (2 * b);
        z |= ((by >> b) & 1u) << (2 * b + 1);
    }
    return z;
}

typedef struct {
    uint64_t key;
    orc_leaf leaf;
} keyed_leaf;

static int cmp_keyed(const void *a, const void *b) {
    uint64_t ka = ((const keyed_leaf *)a)->key, kb = ((const keyed_leaf *)b)->key;
    return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

/* The encoder of Section 3, level by level: every top-level range block is
 * fitted (phase 1); a block whose error is below the level's threshold, or
 * that is at the last level, is stored; otherwise (MNS only, levels before
 * the last) phase 2 is tried; a block that fails both is split into four and
 * its children form the next level's list.
 *
 * Output: leaves in the canonical order (top-level blocks in raster order,
 * then depth-first TL, TR, BL, BR inside each), and one 32-bit split mask
 * per top-level block (bit 0: the block itself, bits 1..4: its four
 * children, bits 5..20: the sixteen grandchildren, each group in depth-first
 * order; a set bit means the node was split).  *fits counts the
 * range-domain fits evaluated. */
int orc_encode(const uint8_t *img, int W, int H, const orc_params *p, orc_leaf *out, int cap,
               uint32_t *split, int *nleaves, int64_t *fits) {
    int rc = orc_check(W, H, p);
    if (rc) return rc;
    int L = nlevels(p);
    int tw = W / p->bmax, th = H / p->bmax;
    int ntop = tw * th;
    int64_t maxleaves = (int64_t)(W / p->bmin) * (H / p->bmin);
    int *list = (int *)malloc(sizeof(int) * 2 * (size_t)maxleaves);
    int *next = (int *)malloc(sizeof(int) * 2 * (size_t)maxleaves);
    keyed_leaf *kl = (keyed_leaf *)malloc(sizeof(keyed_leaf) * (size_t)maxleaves);
    if (!list || !next || !kl) {
        free(list); free(next); free(kl);
        return ORC_ENOMEM;
    }
    memset(split, 0, sizeof(uint32_t) * (size_t)ntop);
    int64_t nfits = 0;
    int count = 0, nl = 0;
    for (int ty = 0; ty < th; ty++)
        for (int tx = 0; tx < tw; tx++) {
            list[2 * count] = tx * p->bmax;
            list[2 * count + 1] = ty * p->bmax;
            count++;
        }
    int B = p->bmax;
    for (int level = 1; level <= L; level++, B >>= 1) {
        int64_t n = (int64_t)B * B;
        int64_t thr = orc_threshold(p->thr_rms[level - 1], n);
        int ncount = 0;
        for (int i = 0; i < count; i++) {
            int x = list[2 * i], y = list[2 * i + 1];
            int X = x / p->bmax, Y = y / p->bmax;
            uint32_t z = morton((uint32_t)((x % p->bmax) / B), (uint32_t)((y % p->bmax) / B));
            uint32_t zf = morton((uint32_t)((x % p->bmax) / p->bmin), (uint32_t)((y % p->bmax) / p->bmin));
            orc_fit f;
            nfits += orc_search(img, W, H, p, x, y, B, &f);
            orc_leaf leaf;
            memset(&leaf, 0, sizeof(leaf));
            leaf.x = (uint16_t)x;
            leaf.y = (uint16_t)y;
            leaf.level = (uint8_t)level;
            leaf.dx = (uint16_t)f.dx;
            leaf.dy = (uint16_t)f.dy;
            leaf.iso = (uint8_t)f.iso;
            int stored = 0;
            if (f.e < thr || level == L) {
                leaf.phase = 1;
                leaf.k = (uint8_t)f.k;
                leaf.q = (uint8_t)f.q;
                stored = 1;
            } else if (p->mode == ORC_MNS && p->phase2 && level < L) {
                nfits += 4;
                stored = orc_phase2(img, W, H, p, level, x, y, B, f.q, &leaf);
            }
            if (stored) {
                if (nl >= cap) {
                    free(list); free(next); free(kl);
                    return ORC_ECAPACITY;
                }
                kl[nl].key = ((uint64_t)(Y * tw + X) << 32) | zf;
                kl[nl].leaf = leaf;
                nl++;
            } else {
                uint32_t bit = (uint32_t)(((1u << (2 * (level - 1))) - 1) / 3) + z;
                split[Y * tw + X] |= 1u << bit;
                int h = B / 2;
                for (int c = 0; c < 4; c++) {
                    next[2 * ncount] = x + (c & 1) * h;
                    next[2 * ncount + 1] = y + (c >> 1) * h;
                    ncount++;
                }
            }
        }
        int *t = list;
        list = next;
        next = t;
        count = ncount;
    }
    qsort(kl, (size_t)nl, sizeof(keyed_leaf), cmp_keyed);
    for (int i = 0; i < nl; i++) out[i] = kl[i].leaf;
    *nleaves = nl;
    if (fits) *fits = nfits;
    free(list); free(next); free(kl);
    return ORC_OK;
}

/* Phase-1 search of a chosen set of ranges, independently of the quadtree
 * (used to sample very large searches).  xs/ys/bs give each range. */
int orc_search_ranges(const uint8_t *img, int W, int H, const orc_params *p, int count,
                      const int32_t *xs, const int32_t *ys, const int32_t *bs, int32_t *k,
                      int32_t *q, int32_t *dx, int32_t *dy, int32_t *iso, int64_t *e) {
    for (int i = 0; i < count; i++) {
        orc_fit f;
        orc_search(img, W, H, p, xs[i], ys[i], bs[i], &f);
        k[i] = f.k; q[i] = f.q; dx[i] = f.dx; dy[i] = f.dy; iso[i] = f.iso; e[i] = f.e;
    }
    return ORC_OK;
}

/* Exposed for tests: moments and best codes for one explicit pair. */
void orc_fit_pair(const uint8_t *img, int W, int x, int y, int B, int dx, int dy, int iso,
                  int s_bits, int o_bits, int64_t *mom5, int32_t *k, int32_t *q, int64_t *e) {
    orc_moments m;
    orc_moments_of(img, W, x, y, B, dx, dy, iso, &m);
    int kk, qq;
    orc_best_codes(&m, (int64_t)B * B, s_bits, o_bits, &kk, &qq, e);
    mom5[0] = m.sr; mom5[1] = m.srr; mom5[2] = m.sd; mom5[3] = m.sdd; mom5[4] = m.sdr;
    *k = kk;
    *q = qq;
}

/* ------------------------------------------------------------------ */
/* Decoder                                                              */

/* Apply one transform to the current image x (read) and write its block into
 * y: every output pixel is round-half-up(O + s (d - mean(d))) computed on the
 * decimated (and isometry-mapped) domain of x, clipped to [0, 255]:
 *     p = floor((512 n O + c (n d4 - Sd4) + 256 n) / (512 n)).          */
static void apply_transform(const uint8_t *x, uint8_t *y, int W, int rx, int ry, int B, int dx,
                            int dy, int iso, int64_t c, int64_t O) {
    int64_t n = (int64_t)B * B;
    int64_t sd = 0;
    for (int v = 0; v < B; v++)
        for (int u = 0; u < B; u++) sd += d4_at(x, W, dx, dy, u, v);
    for (int v = 0; v < B; v++) {
        for (int u = 0; u < B; u++) {
            int su, sv;
            orc_iso_source(iso, B, u, v, &su, &sv);
            int64_t d = d4_at(x, W, dx, dy, su, sv);
            int64_t num = 512 * n * O + c * (n * d - sd) + 256 * n;
            int64_t pix = floor_div(num, 512 * n);
            if (pix < 0) pix = 0;
            if (pix > 255) pix = 255;
            y[(size_t)(ry + v) * W + (rx + u)] = (uint8_t)pix;
        }
    }
}

/* The paper does not describe its decoder beyond the iterated function
 * system it relies on (Section 1).  This one starts from mid-grey (128) and
 * applies every stored transform to the previous iterate (Jacobi update) a
 * fixed number of times. */
int orc_decode(const orc_leaf *leaves, int nleaves, int W, int H, const orc_params *p, int iters,
               uint8_t *out) {
    int L = nlevels(p);
    uint8_t *cur = (uint8_t *)malloc((size_t)W * H);
    uint8_t *nxt = (uint8_t *)malloc((size_t)W * H);
    if (!cur || !nxt) {
        free(cur); free(nxt);
        return ORC_ENOMEM;
    }
    memset(cur, 128, (size_t)W * H);
    memcpy(nxt, cur, (size_t)W * H);
    for (int it = 0; it < iters; it++) {
        for (int i = 0; i < nleaves; i++) {
            const orc_leaf *lf = &leaves[i];
            int B = p->bmax >> (lf->level - 1);
            if (lf->level < 1 || lf->level > L) continue;
            if (lf->phase == 1) {
                apply_transform(cur, nxt, W, lf->x, lf->y, B, lf->dx, lf->dy, lf->iso,
                                orc_contrast(lf->k, p->s_bits), orc_luminance(lf->q, p->o_bits));
            } else {
                int h = B / 2;
                int64_t Oi = orc_luminance(lf->q, p->o_bits);
                int64_t O[4];
                O[0] = Oi + lf->d[0];
                O[1] = Oi + lf->d[1];
                O[2] = Oi + lf->d[2];
                O[3] = 4 * Oi - (O[0] + O[1] + O[2]);
                for (int sb = 0; sb < 4; sb++) {
                    int sx = lf->x + (sb & 1) * h, sy = lf->y + (sb >> 1) * h;
                    int dx, dy;
                    phase2_domain_of(p, W, H, lf->x, lf->y, B, sb, &dx, &dy);
                    apply_transform(cur, nxt, W, sx, sy, h, dx, dy, 0,
                                    orc_phase2_contrast(lf->level, (lf->k >> sb) & 1), O[sb]);
                }
            }
        }
        uint8_t *t = cur;
        cur = nxt;
        nxt = t;
    }
    memcpy(out, cur, (size_t)W * H);
    free(cur);
    free(nxt);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Bit accounting (Sections 3.3 and 3.4)                                */

/* Bits of the stored stream, per leaf:
 *   payload: phase 1 s_bits + o_bits; phase 2 o_bits (O_i) + 3 M-bit mean
 *            differences + 4 one-bit contrast choices (Section 3.3);
 *            local search adds the candidate index, exhaustive search the
 *            domain index and the isometry;
 *   +1 phase bit at levels where phase 2 is possible (Section 3.3);
 *   +ceil(log2 L) level bits, except that, with Technique 2 (Section 3.4),
 *    only the first of the four sibling leaves at the last level pays them.
 * Leaves must be in the canonical order.  Returns the total bit count. */
int64_t orc_bits(const orc_leaf *leaves, int nleaves, int W, int H, const orc_params *p,
                 int technique2) {
    int L = nlevels(p);
    int lbits = ilog2_ceil(L);
    int64_t total = 0;
    int extra = 0;
    if (p->mode == ORC_LOCAL) {
        int per = 2 * (p->local_radius / p->local_step) + 1;
        extra = ilog2_ceil((long)per * per);
    } else if (p->mode == ORC_EXHAUSTIVE) {
        extra = ilog2_ceil((long)orc_count_domains(W, H, p->bmin, p->dom_step)) +
                ilog2_ceil(p->isometries);
    }
    for (int i = 0; i < nleaves; i++) {
        const orc_leaf *lf = &leaves[i];
        int64_t b;
        if (lf->phase == 1) b = p->s_bits + p->o_bits + extra;
        else b = p->o_bits + 3 * orc_phase2_mbits(lf->level) + 4;
        if (p->mode == ORC_MNS && p->phase2 && lf->level < L) b += 1;
        int pay_level = 1;
        if (technique2 && L > 1 && lf->level == L) {
            int B = p->bmax >> (L - 1);
            int first = ((lf->x / B) % 2 == 0) && ((lf->y / B) % 2 == 0);
            pay_level = first;
        }
        if (pay_level) b += lbits;
        total += b;
    }
    return total;
}

/* Number of candidate domains the search of one range tries (81 for an
 * interior range under local search with radius 16 and step 4, Section 2). */
int orc_count_candidates(const uint8_t *img, int W, int H, const orc_params *p, int x, int y,
                         int B) {
    orc_fit f;
    return orc_search(img, W, H, p, x, y, B, &f);
}

/* ------------------------------------------------------------------ */
/* Bitstream: the stored parameters of Section 3.3 with the level-id rule
 * of Technique 2 (Section 3.4).
 *
 * Layout (a reading: the paper gives the fields and their widths, not an
 * order): bits are appended least-significant first into 32-bit words (bit
 * i of the stream is bit i % 32 of word i / 32).  Leaves follow the
 * canonical order; per leaf:
 *   level - 1          ceil(log2 L) bits; with Technique 2 a last-level
 *                      leaf that is not the first (top-left) of its group
 *                      of four has none (its level is implied)
 *   phase              1 bit (0: phase 1, 1: phase 2) at levels < L when
 *                      MNS phase 2 is on
 *   phase 1            k (s_bits), q (o_bits), then the domain: local
 *                      search the offset index ((oy + R)/step * per +
 *                      (ox + R)/step, per = 2R/step + 1) in ceil(log2 per^2)
 *                      bits; exhaustive search the domain's raster index on
 *                      the step grid (ceil(log2 count) bits) and the
 *                      isometry (ceil(log2 isometries) bits)
 *   phase 2            q_i (o_bits), the three differences O_k - O_i (M
 *                      bits each, two's complement, M of Section 3.3), the
 *                      four contrast choices (4 bits, bit b = sub-block b)
 * Positions, block sides and centred domains are implied by the order.
 * tile_bits[t] is the first bit of top-level block t (tile_bits[ntop] = the
 * total): an index that lets a reader start at any block. */

static void put_bits(uint32_t *w, int64_t *pos, uint32_t v, int nb) {
    for (int i = 0; i < nb; i++, (*pos)++)
        if ((v >> i) & 1u) w[*pos >> 5] |= 1u << (*pos & 31);
}

static uint32_t get_bits(const uint32_t *w, int64_t *pos, int nb) {
    uint32_t v = 0;
    for (int i = 0; i < nb; i++, (*pos)++) v |= ((w[*pos >> 5] >> (*pos & 31)) & 1u) << i;
    return v;
}

typedef struct {
    int L, lbits, phase_bit_on, extra_kind;
    int per, rstep, local_bits;   /* local search */
    int ndx, dom_bits, iso_bits;  /* exhaustive search */
} bit_layout;

static void layout_of(int W, int H, const orc_params *p, bit_layout *b) {
    b->L = nlevels(p);
    b->lbits = ilog2_ceil(b->L);
    b->phase_bit_on = p->mode == ORC_MNS && p->phase2;
    b->extra_kind = p->mode == ORC_LOCAL ? 1 : (p->mode == ORC_EXHAUSTIVE ? 2 : 0);
    b->rstep = p->local_step > 0 ? p->local_radius / p->local_step : 0;
    b->per = 2 * b->rstep + 1;
    b->local_bits = ilog2_ceil((long)b->per * b->per);
    b->ndx = p->dom_step > 0 ? (W - 2 * p->bmin) / p->dom_step + 1 : 0;
    b->dom_bits = b->extra_kind == 2 ? ilog2_ceil((long)orc_count_domains(W, H, p->bmin, p->dom_step)) : 0;
    b->iso_bits = b->extra_kind == 2 ? ilog2_ceil(p->isometries) : 0;
}

/* Bits of the stream of `leaves` (canonical order).  words[0..nwords) must
 * be zero; returns ORC_ECAPACITY when they are too few. */
int orc_serialize(const orc_leaf *leaves, int nleaves, int W, int H, const orc_params *p, int technique2,
                  uint32_t *words, int64_t nwords, uint64_t *tile_bits, int64_t *nbits) {
    int rc = orc_check(W, H, p);
    if (rc) return rc;
    bit_layout b;
    layout_of(W, H, p, &b);
    int tw = W / p->bmax, ntop = tw * (H / p->bmax);
    int64_t pos = 0;
    int t_next = 0;
    for (int i = 0; i < nleaves; i++) {
        const orc_leaf *lf = &leaves[i];
        int t = (lf->y / p->bmax) * tw + lf->x / p->bmax;
        while (t_next <= t) tile_bits[t_next++] = (uint64_t)pos;
        int B = p->bmax >> (lf->level - 1);
        /* worst case of one leaf: 8 + 1 + 8 + 3 * 7 + 4 + 32 bits */
        if ((pos + 80) / 32 + 1 > nwords) return ORC_ECAPACITY;
        int first = ((lf->x / B) % 2 == 0) && ((lf->y / B) % 2 == 0);
        if (!(technique2 && b.L > 1 && lf->level == b.L && !first)) put_bits(words, &pos, lf->level - 1u, b.lbits);
        if (b.phase_bit_on && lf->level < b.L) put_bits(words, &pos, lf->phase == 2 ? 1u : 0u, 1);
        if (lf->phase == 1) {
            put_bits(words, &pos, lf->k, p->s_bits);
            put_bits(words, &pos, lf->q, p->o_bits);
            if (b.extra_kind == 1) {
                int ox = lf->dx - orc_centred(lf->x, B, W), oy = lf->dy - orc_centred(lf->y, B, H);
                int idx = (oy / p->local_step + b.rstep) * b.per + (ox / p->local_step + b.rstep);
                put_bits(words, &pos, (uint32_t)idx, b.local_bits);
            } else if (b.extra_kind == 2) {
                int idx = (lf->dy / p->dom_step) * b.ndx + lf->dx / p->dom_step;
                put_bits(words, &pos, (uint32_t)idx, b.dom_bits);
                put_bits(words, &pos, lf->iso, b.iso_bits);
            }
        } else {
            int M = orc_phase2_mbits(lf->level);
            put_bits(words, &pos, lf->q, p->o_bits);
            for (int k = 0; k < 3; k++) put_bits(words, &pos, (uint32_t)lf->d[k] & ((1u << M) - 1u), M);
            put_bits(words, &pos, lf->k, 4);
        }
    }
    while (t_next <= ntop) tile_bits[t_next++] = (uint64_t)pos;
    *nbits = pos;
    return ORC_OK;
}

/* Read a stream back: leaves in canonical order with every record field
 * (positions from the order, centred domains recomputed), split masks, the
 * tile index.  ORC_EBADPARAM for a stream that does not tile the image. */
int orc_parse(const uint32_t *words, int64_t nbits, int W, int H, const orc_params *p, int technique2,
              orc_leaf *out, int cap, uint32_t *split, uint64_t *tile_bits, int *nleaves) {
    int rc = orc_check(W, H, p);
    if (rc) return rc;
    bit_layout b;
    layout_of(W, H, p, &b);
    int tw = W / p->bmax, th = H / p->bmax;
    int cells = p->bmax / p->bmin;
    int64_t pos = 0;
    int n = 0;
    for (int t = 0; t < tw * th; t++) {
        tile_bits[t] = (uint64_t)pos;
        split[t] = 0;
        int tx = (t % tw) * p->bmax, ty = (t / tw) * p->bmax;
        int c = 0;
        while (c < cells * cells) {
            int cx = 0, cy = 0;
            for (int k = 0; k < 8; k++) {
                cx |= ((c >> (2 * k)) & 1) << k;
                cy |= ((c >> (2 * k + 1)) & 1) << k;
            }
            int level;
            if (technique2 && b.L > 1 && (c & 3) != 0) level = b.L;
            else level = (int)get_bits(words, &pos, b.lbits) + 1;
            if (level < 1 || level > b.L) return ORC_EBADPARAM;
            int B = p->bmax >> (level - 1);
            int span = (B / p->bmin) * (B / p->bmin);
            if (c % span != 0 || n >= cap || pos > nbits) return ORC_EBADPARAM;
            orc_leaf lf;
            memset(&lf, 0, sizeof(lf));
            lf.x = (uint16_t)(tx + cx * p->bmin);
            lf.y = (uint16_t)(ty + cy * p->bmin);
            lf.level = (uint8_t)level;
            lf.dx = (uint16_t)orc_centred(lf.x, B, W);
            lf.dy = (uint16_t)orc_centred(lf.y, B, H);
            int phase = 1;
            if (b.phase_bit_on && level < b.L) phase = get_bits(words, &pos, 1) ? 2 : 1;
            lf.phase = (uint8_t)phase;
            if (phase == 1) {
                lf.k = (uint8_t)get_bits(words, &pos, p->s_bits);
                lf.q = (uint8_t)get_bits(words, &pos, p->o_bits);
                if (b.extra_kind == 1) {
                    int idx = (int)get_bits(words, &pos, b.local_bits);
                    if (idx >= b.per * b.per) return ORC_EBADPARAM;
                    lf.dx = (uint16_t)(lf.dx + (idx % b.per - b.rstep) * p->local_step);
                    lf.dy = (uint16_t)(lf.dy + (idx / b.per - b.rstep) * p->local_step);
                } else if (b.extra_kind == 2) {
                    int idx = (int)get_bits(words, &pos, b.dom_bits);
                    lf.dx = (uint16_t)((idx % b.ndx) * p->dom_step);
                    lf.dy = (uint16_t)((idx / b.ndx) * p->dom_step);
                    lf.iso = (uint8_t)get_bits(words, &pos, b.iso_bits);
                }
            } else {
                int M = orc_phase2_mbits(level);
                lf.q = (uint8_t)get_bits(words, &pos, p->o_bits);
                for (int k = 0; k < 3; k++) {
                    int v = (int)get_bits(words, &pos, M);
                    if (v >= (1 << (M - 1))) v -= 1 << M;  /* two's complement */
                    lf.d[k] = (int8_t)v;
                }
                lf.k = (uint8_t)get_bits(words, &pos, 4);
            }
            if (pos > nbits) return ORC_EBADPARAM;
            for (int a = 1; a < level; a++)
                split[t] |= 1u << (((1u << (2 * (a - 1))) - 1) / 3 + (uint32_t)(c >> (2 * (b.L - a))));
            out[n++] = lf;
            c += span;
        }
    }
    tile_bits[tw * th] = (uint64_t)pos;
    if (pos != nbits) return ORC_EBADPARAM;
    *nleaves = n;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Resolution-independent decoding (Section 1: the stored transforms are a
 * description of the image at no particular resolution).  Rescaling a
 * stream by 2^shift (shift = +1 or -1) multiplies every position, block
 * side and domain position by 2^shift and keeps the codes; decoding the
 * result renders the attractor on a grid 2^shift times finer or coarser.
 * Returns ORC_EBADPARAM when a rescaled quantity is not an integer or the
 * block sides leave 4 <= bmin, bmax <= 32 (the sides the decoder handles). */
int orc_rescale(const orc_leaf *in, int n, int W, int H, const orc_params *p, int shift, orc_leaf *out,
                orc_params *po, int *W2, int *H2) {
    if (shift != 1 && shift != -1) return ORC_EBADPARAM;
    *po = *p;
    if (shift > 0) {
        po->bmax = p->bmax * 2;
        po->bmin = p->bmin * 2;
        po->local_radius = p->local_radius * 2;
        po->local_step = p->local_step * 2;
        po->dom_step = p->dom_step * 2;
        *W2 = W * 2;
        *H2 = H * 2;
    } else {
        if (p->bmin % 2 || W % 2 || H % 2 || p->local_radius % 2 || p->local_step % 2 || p->dom_step % 2)
            return ORC_EBADPARAM;
        po->bmax = p->bmax / 2;
        po->bmin = p->bmin / 2;
        po->local_radius = p->local_radius / 2;
        po->local_step = p->local_step / 2;
        po->dom_step = p->dom_step / 2;
        *W2 = W / 2;
        *H2 = H / 2;
    }
    if (po->bmin < 4 || po->bmax > 32) return ORC_EBADPARAM;
    for (int i = 0; i < n; i++) {
        orc_leaf lf = in[i];
        int v[4] = {lf.x, lf.y, lf.dx, lf.dy};
        for (int k = 0; k < 4; k++) {
            if (shift < 0 && v[k] % 2) return ORC_EBADPARAM;
            v[k] = shift > 0 ? v[k] * 2 : v[k] / 2;
        }
        lf.x = (uint16_t)v[0];
        lf.y = (uint16_t)v[1];
        lf.dx = (uint16_t)v[2];
        lf.dy = (uint16_t)v[3];
        out[i] = lf;
    }
    return ORC_OK;
}
