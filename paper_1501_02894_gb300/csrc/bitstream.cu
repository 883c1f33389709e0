// bitstream.cu -- the stored parameters of Section 3.3 as a bitstream, with
// the level ids of Technique 2 (Section 3.4), written and read on the device.
//
// Layout (the paper gives the fields and their widths, not an order; this
// is the order chosen): bits are appended least-significant first into
// 32-bit words; leaves follow the stream's canonical order; per leaf
//   level - 1   ceil(log2 L) bits, absent (Technique 2) for a last-level
//               leaf that is not the top-left one of its group of four
//   phase       1 bit at levels < L when MNS phase 2 is on
//   phase 1     k (s_bits), q (o_bits); local search: the offset index on
//               the (2R/step + 1)^2 grid; exhaustive search: the domain's
//               raster index on the step grid and the isometry
//   phase 2     q_i (o_bits), three M-bit two's-complement differences
//               (M = 5 at level 1, 6 below), four contrast-choice bits.
// Positions, block sides and centred domains follow from the order and are
// not stored.  tile_bits[t] (uint64) is the first bit of top-level block t,
// tile_bits[ntop] the total: an index that lets the reader parse every
// block independently.
//
// Writer: a warp per top-level block sizes its leaves (warp sum), a scan
// over each stream's blocks gives the index (and zeroes its words), and the
// warp then writes every leaf's fields at its bit offset with atomicOr
// (fields may straddle words and blocks may share a word).  Reader: a thread
// per block parses it twice -- once to count its leaves (scanned into tile
// offsets), once to write the records, split masks and the record count.
// Every kernel covers a whole batch of streams (up to kBitBatch per launch,
// their descriptors passed by value as the kernel's parameter), so writing
// or reading any number of streams takes three launches per kBitBatch.
#include "fic_internal.cuh"

namespace fic {

namespace {

__host__ __device__ inline int ceil_log2(long long v) {
    int b = 0;
    while ((1LL << b) < v) ++b;
    return b;
}

// Field widths of one stream.
struct BitLayout {
    int W, H, bmax, bmin, L, lbits, phase_bit, s_bits, o_bits, mode;
    int rstep, per, local_bits, step, ndx, dom_bits, iso_bits, technique2;
};

BitLayout make_layout(int W, int H, const fic_params &p, int technique2) {
    BitLayout b;
    b.W = W;
    b.H = H;
    b.bmax = p.bmax;
    b.bmin = p.bmin;
    b.L = 1;
    for (int s = p.bmax; s > p.bmin; s >>= 1) ++b.L;
    b.lbits = ceil_log2(b.L);
    b.phase_bit = p.mode == FIC_MNS && p.phase2;
    b.s_bits = p.s_bits;
    b.o_bits = p.o_bits;
    b.mode = p.mode;
    b.rstep = p.local_step > 0 ? p.local_radius / p.local_step : 0;
    b.per = 2 * b.rstep + 1;
    b.local_bits = p.mode == FIC_LOCAL ? ceil_log2((long long)b.per * b.per) : 0;
    b.step = p.mode == FIC_LOCAL ? p.local_step : p.dom_step;
    b.ndx = p.dom_step > 0 ? (W - 2 * p.bmin) / p.dom_step + 1 : 0;
    const int ndy = p.dom_step > 0 ? (H - 2 * p.bmin) / p.dom_step + 1 : 0;
    b.dom_bits = p.mode == FIC_EXHAUSTIVE ? ceil_log2((long long)b.ndx * ndy) : 0;
    b.iso_bits = p.mode == FIC_EXHAUSTIVE ? ceil_log2(p.isometries) : 0;
    b.technique2 = technique2 ? 1 : 0;
    return b;
}

// The fields of one record as (value, width) pairs in stream order; returns
// their count.
__device__ __forceinline__ int leaf_fields(const BitLayout &b, uint4 r, uint32_t (&v)[9], int (&n)[9]) {
    const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16);
    const int level = (int)(r.y & 0xffu), phase = (int)((r.y >> 8) & 0xffu);
    const int k = (int)((r.y >> 16) & 0xffu), q = (int)(r.y >> 24);
    const int B = b.bmax >> (level - 1);
    int f = 0;
    const bool first = ((x / B) & 1) == 0 && ((y / B) & 1) == 0;
    if (!(b.technique2 && b.L > 1 && level == b.L && !first)) {
        v[f] = (uint32_t)(level - 1);
        n[f++] = b.lbits;
    }
    if (b.phase_bit && level < b.L) {
        v[f] = phase == 2 ? 1u : 0u;
        n[f++] = 1;
    }
    if (phase == 1) {
        v[f] = (uint32_t)k;
        n[f++] = b.s_bits;
        v[f] = (uint32_t)q;
        n[f++] = b.o_bits;
        const int dx = (int)(r.w & 0xffffu), dy = (int)(r.w >> 16);
        if (b.mode == FIC_LOCAL) {
            const int ox = dx - centred_origin(x, B, b.W), oy = dy - centred_origin(y, B, b.H);
            v[f] = (uint32_t)((oy / b.step + b.rstep) * b.per + (ox / b.step + b.rstep));
            n[f++] = b.local_bits;
        } else if (b.mode == FIC_EXHAUSTIVE) {
            v[f] = (uint32_t)((dy / b.step) * b.ndx + dx / b.step);
            n[f++] = b.dom_bits;
            v[f] = (r.z >> 24) & 0xffu;
            n[f++] = b.iso_bits;
        }
    } else {
        const int M = level == 1 ? 5 : 6;
        v[f] = (uint32_t)q;
        n[f++] = b.o_bits;
        for (int i = 0; i < 3; ++i) {
            v[f] = (r.z >> (8 * i)) & ((1u << M) - 1u);  // the int8 difference's low M bits
            n[f++] = M;
        }
        v[f] = (uint32_t)k & 15u;
        n[f++] = 4;
    }
    return f;
}

__device__ __forceinline__ int leaf_bits(const BitLayout &b, uint4 r) {
    uint32_t v[9];
    int n[9];
    const int f = leaf_fields(b, r, v, n);
    int s = 0;
    for (int i = 0; i < f; ++i) s += n[i];
    return s;
}

__device__ __forceinline__ void put_bits(uint32_t *w, unsigned long long pos, uint32_t v, int nb) {
    if (nb == 0) return;
    const unsigned long long i = pos >> 5;
    const int sh = (int)(pos & 31);
    if (v << sh) atomicOr(w + i, v << sh);
    if (sh + nb > 32 && (v >> (32 - sh))) atomicOr(w + i + 1, v >> (32 - sh));
}

__device__ __forceinline__ uint32_t get_bits(const uint32_t *w, unsigned long long pos, int nb, long long nwords) {
    if (nb == 0) return 0u;
    const long long i = (long long)(pos >> 5);
    const int sh = (int)(pos & 31);
    const uint32_t lo = i < nwords ? w[i] : 0u;
    const uint32_t hi = i + 1 < nwords ? w[i + 1] : 0u;
    const unsigned long long both = ((unsigned long long)hi << 32) | lo;
    return (uint32_t)(both >> sh) & (nb == 32 ? 0xffffffffu : ((1u << nb) - 1u));
}

// ---- batches

constexpr int kBitBatch = 48;  // streams per launch (descriptors travel as the kernel parameter)

// One stream of a batch.
struct BitDesc {
    BitLayout b;
    int ntop;
    const fic_record *rec;        // serialize: the stream's records and tile offsets
    const uint32_t *toff;
    uint32_t *words;              // serialize: output words (nwords, zeroed here)
    const uint32_t *words_in;     // parse: input words
    long long nwords;
    unsigned long long *tile_bits;     // serialize: output index; parse: input index (read only)
    unsigned long long *sizes;         // workspace: per block bits (serialize) or leaf counts (parse)
    unsigned long long *first;         // workspace (parse): exclusive scan of the counts
    fic_record *out_rec;          // parse outputs
    uint32_t *out_toff, *out_split, *out_info;
};

struct BitBatch {
    int count;
    int tops_base[kBitBatch + 1];  // first global block index of each stream
    BitDesc d[kBitBatch];
};

// The stream of global block g and its local index.
__device__ __forceinline__ int batch_stream(const BitBatch &B, int g) {
    int lo = 0, hi = B.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.tops_base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Exclusive scan of one stream's n uint64 values into out[0..n] (out[n] =
// total) by one CTA: each thread sums a contiguous slice, the CTA scans the
// slice sums, and each thread writes its slice.  Returns (to every thread)
// whether any value had its top bit set (a block that does not parse).
__device__ bool cta_scan(const unsigned long long *__restrict__ in, int n, unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s_part[1024];
    __shared__ int s_bad;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) s_bad = 0;
    __syncthreads();
    const int per = (n + nt - 1) / nt;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    unsigned long long s = 0;
    bool bad = false;
    for (int i = lo; i < hi; ++i) {
        const unsigned long long v = in[i];
        bad = bad || (v >> 63);
        s += v;
    }
    if (bad) s_bad = 1;
    s_part[t] = s;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const unsigned long long v = t >= off ? s_part[t - off] : 0ull;
        __syncthreads();
        s_part[t] += v;
        __syncthreads();
    }
    unsigned long long acc = s_part[t] - s;
    for (int i = lo; i < hi; ++i) {
        out[i] = acc;
        acc += in[i];
    }
    if (t == nt - 1) out[n] = s_part[t];
    __syncthreads();
    return s_bad != 0;
}

// ---- writer

__global__ void tile_size_kernel(const __grid_constant__ BitBatch B) {
    const int lane = threadIdx.x & 31;
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (g >= B.tops_base[B.count]) return;
    const BitDesc &D = B.d[batch_stream(B, g)];
    const int t = g - B.tops_base[batch_stream(B, g)];
    const uint32_t beg = D.toff[t], end = D.toff[t + 1];
    unsigned long long s = 0;
    for (uint32_t i = beg + lane; i < end; i += 32)
        s += (unsigned)leaf_bits(D.b, *reinterpret_cast<const uint4 *>(D.rec + i));
    for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) D.sizes[t] = s;
}

// kSerZeroCtas CTAs per stream (blockIdx.y): each zeroes a slice of the
// stream's words (the writer ORs its fields in); the first also scans the
// block sizes into the index.
constexpr int kSerZeroCtas = 8;
__global__ void __launch_bounds__(1024) ser_scan_kernel(const __grid_constant__ BitBatch B) {
    const BitDesc &D = B.d[blockIdx.x];
    const long long per = (D.nwords + kSerZeroCtas - 1) / kSerZeroCtas;
    const long long lo = per * blockIdx.y, hi = min(D.nwords, lo + per);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) D.words[i] = 0u;
    if (blockIdx.y == 0) cta_scan(D.sizes, D.ntop, D.tile_bits);
}

__global__ void write_kernel(const __grid_constant__ BitBatch B) {
    const int lane = threadIdx.x & 31;
    const int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (g >= B.tops_base[B.count]) return;
    const int si = batch_stream(B, g);
    const BitDesc &D = B.d[si];
    const int t = g - B.tops_base[si];
    const BitLayout &b = D.b;
    const uint32_t beg = D.toff[t], end = D.toff[t + 1];
    unsigned long long base = D.tile_bits[t];
    for (uint32_t i0 = beg; i0 < end; i0 += 32) {
        const uint32_t i = i0 + lane;
        const bool has = i < end;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        uint32_t v[9];
        int n[9];
        int f = 0, s = 0;
        if (has) {
            r = *reinterpret_cast<const uint4 *>(D.rec + i);
            f = leaf_fields(b, r, v, n);
            for (int j = 0; j < f; ++j) s += n[j];
        }
        // exclusive prefix of the leaf sizes over the lanes
        int incl = s;
        for (int m = 1; m < 32; m <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, m);
            if (lane >= m) incl += o;
        }
        unsigned long long pos = base + (unsigned)(incl - s);
        for (int j = 0; j < f; ++j) {
            put_bits(D.words, pos, v[j], n[j]);
            pos += (unsigned)n[j];
        }
        base += (unsigned)__shfl_sync(0xffffffffu, incl, 31);
    }
}

// ---- reader

// Parse top-level block t from its first bit.  WRITE = false: only count
// the leaves (returns the count, or -1 for a block that does not tile);
// WRITE = true: also store the records at out + first and the split mask.
template <bool WRITE>
__device__ int parse_tile(const BitLayout &b, const uint32_t *words, long long nwords, unsigned long long pos,
                          unsigned long long end, int t, fic_record *out, uint32_t *split) {
    const int tw = b.W / b.bmax;
    const int tx = (t % tw) * b.bmax, ty = (t / tw) * b.bmax;
    const int cells = b.bmax / b.bmin;
    int c = 0, count = 0;
    uint32_t mask = 0;
    while (c < cells * cells) {
        int cx = 0, cy = 0;
        for (int k = 0; k < 3; ++k) {
            cx |= ((c >> (2 * k)) & 1) << k;
            cy |= ((c >> (2 * k + 1)) & 1) << k;
        }
        int level;
        if (b.technique2 && b.L > 1 && (c & 3) != 0) {
            level = b.L;
        } else {
            level = (int)get_bits(words, pos, b.lbits, nwords) + 1;
            pos += (unsigned)b.lbits;
        }
        if (level > b.L) return -1;
        const int B = b.bmax >> (level - 1);
        const int span = (B / b.bmin) * (B / b.bmin);
        if (c % span) return -1;
        const int x = tx + cx * b.bmin, y = ty + cy * b.bmin;
        int phase = 1;
        if (b.phase_bit && level < b.L) {
            phase = get_bits(words, pos, 1, nwords) ? 2 : 1;
            pos += 1;
        }
        uint32_t k = 0, q = 0, dz = 0, iso = 0;
        int dx = centred_origin(x, B, b.W), dy = centred_origin(y, B, b.H);
        if (phase == 1) {
            k = get_bits(words, pos, b.s_bits, nwords);
            pos += (unsigned)b.s_bits;
            q = get_bits(words, pos, b.o_bits, nwords);
            pos += (unsigned)b.o_bits;
            if (b.mode == FIC_LOCAL) {
                const int idx = (int)get_bits(words, pos, b.local_bits, nwords);
                pos += (unsigned)b.local_bits;
                if (idx >= b.per * b.per) return -1;
                dx += (idx % b.per - b.rstep) * b.step;
                dy += (idx / b.per - b.rstep) * b.step;
            } else if (b.mode == FIC_EXHAUSTIVE) {
                const int idx = (int)get_bits(words, pos, b.dom_bits, nwords);
                pos += (unsigned)b.dom_bits;
                dx = (idx % b.ndx) * b.step;
                dy = (idx / b.ndx) * b.step;
                iso = get_bits(words, pos, b.iso_bits, nwords);
                pos += (unsigned)b.iso_bits;
            }
        } else {
            const int M = level == 1 ? 5 : 6;
            q = get_bits(words, pos, b.o_bits, nwords);
            pos += (unsigned)b.o_bits;
            for (int i = 0; i < 3; ++i) {
                int d = (int)get_bits(words, pos, M, nwords);
                pos += (unsigned)M;
                if (d >= (1 << (M - 1))) d -= 1 << M;
                dz |= ((uint32_t)d & 0xffu) << (8 * i);
            }
            k = get_bits(words, pos, 4, nwords);
            pos += 4;
        }
        if (pos > end) return -1;
        if (WRITE) {
            *reinterpret_cast<uint4 *>(out + count) =
                make_uint4((uint32_t)x | ((uint32_t)y << 16),
                           (uint32_t)level | ((uint32_t)phase << 8) | (k << 16) | (q << 24), dz | (iso << 24),
                           (uint32_t)dx | ((uint32_t)dy << 16));
            for (int a = 1; a < level; ++a)
                mask |= 1u << (((1u << (2 * (a - 1))) - 1) / 3 + (uint32_t)(c >> (2 * (b.L - a))));
        }
        ++count;
        c += span;
    }
    if (pos != end) return -1;
    if (WRITE) split[t] = mask;
    return count;
}

// The leaf boundaries of a block follow from the leaves' headers alone (the
// level id, when stored, and the phase bit fix a leaf's size), so the reader
// splits parsing in two: lane 0 walks the headers -- the only serial part --
// recording where each leaf's fields start, and then every lane decodes
// leaves of its own.  A block has at most 64 leaves ((bmax / bmin)^2).
struct LeafPos {
    uint32_t pos;   // first bit of the leaf's fields after its header (relative to the staged words)
    uint16_t c;     // its first bmin cell (Morton index inside the top-level block)
    uint8_t level, phase;
};
constexpr int kTileLeaves = 64;

// 32 bits of staged words starting at bit `pos` (the buffer holds four zero
// words past the staged ones: every read of a walk starts less than 96 bits
// past the block's end, which lies in the staged words).
__device__ __forceinline__ uint32_t bits32(const uint32_t *w, uint32_t pos) {
    return __funnelshift_r(w[pos >> 5], w[(pos >> 5) + 1], pos & 31);
}

// Walk the headers of a block in staged words (positions relative to the
// first staged word); returns its leaf count, or -1 for a block that does
// not tile (or, with OUT, holds more than `cap` leaves).  A leaf at level
// `level` covers 4^(L - level) bmin cells (bmax / bmin = 2^(L - 1)), its
// header is the level id (omitted under Technique 2 inside a group of four)
// and the phase bit, and its fields have a fixed length for each phase and
// level, so the walk reads only the headers.
template <bool OUT>
__device__ int walk_tile(const BitLayout &b, const uint32_t *words, uint32_t pos, uint32_t end, LeafPos *out,
                         int cap) {
    const int L = b.L, lbits = b.lbits;
    const bool t2 = b.technique2 && L > 1, pbit = b.phase_bit, local = b.mode == FIC_LOCAL;
    const int ncells = 1 << (2 * (L - 1));
    const uint32_t lmask = (1u << lbits) - 1u;
    const uint32_t len1 = (uint32_t)(b.s_bits + b.o_bits) + (local ? (uint32_t)b.local_bits : 0u) +
                          (b.mode == FIC_EXHAUSTIVE ? (uint32_t)(b.dom_bits + b.iso_bits) : 0u);
    const uint32_t len2_top = (uint32_t)b.o_bits + 3u * 5u + 4u, len2 = (uint32_t)b.o_bits + 3u * 6u + 4u;
    const uint32_t lskip = (uint32_t)(b.s_bits + b.o_bits), lbm = (1u << b.local_bits) - 1u;
    const uint32_t pp = (uint32_t)(b.per * b.per);
    int c = 0, count = 0;
    while (c < ncells) {
        const uint32_t hb = bits32(words, pos);
        int level = L;
        uint32_t used = 0;
        if (!(t2 && (c & 3) != 0)) {
            level = (int)(hb & lmask) + 1;
            used = (uint32_t)lbits;
        }
        if (level > L) return -1;
        const int span_lg = 2 * (L - level);
        if (c & ((1 << span_lg) - 1)) return -1;
        int phase = 1;
        if (pbit && level < L) {
            phase = ((hb >> used) & 1u) ? 2 : 1;
            ++used;
        }
        pos += used;
        if (OUT) {
            if (count >= cap) return -1;
            out[count].pos = pos;
            out[count].c = (uint16_t)c;
            out[count].level = (uint8_t)level;
            out[count].phase = (uint8_t)phase;
        }
        if (phase == 1) {
            if (local && (bits32(words, pos + lskip) & lbm) >= pp) return -1;
            pos += len1;
        } else {
            pos += level == 1 ? len2_top : len2;
        }
        if (pos > end) return -1;
        ++count;
        c += 1 << span_lg;
    }
    return pos == end ? count : -1;
}

// The next nb (<= 32) bits of staged words at `pos`, advancing it.
__device__ __forceinline__ uint32_t take_bits(const uint32_t *w, uint32_t &pos, int nb) {
    const uint32_t v = nb ? bits32(w, pos) & (0xffffffffu >> (32 - nb)) : 0u;
    pos += (uint32_t)nb;
    return v;
}

// The record of one walked leaf of top-level block t (staged words).
__device__ uint4 decode_leaf(const BitLayout &b, const uint32_t *words, const LeafPos &lp, int t) {
    const int tw = b.W / b.bmax;
    const int tx = (t % tw) * b.bmax, ty = (t / tw) * b.bmax;
    const int c = lp.c, level = lp.level, phase = lp.phase;
    int cx = 0, cy = 0;
    for (int k = 0; k < 3; ++k) {
        cx |= ((c >> (2 * k)) & 1) << k;
        cy |= ((c >> (2 * k + 1)) & 1) << k;
    }
    const int B = b.bmax >> (level - 1);
    const int x = tx + cx * b.bmin, y = ty + cy * b.bmin;
    uint32_t pos = lp.pos;
    uint32_t k = 0, q = 0, dz = 0, iso = 0;
    int dx = centred_origin(x, B, b.W), dy = centred_origin(y, B, b.H);
    if (phase == 1) {
        k = take_bits(words, pos, b.s_bits);
        q = take_bits(words, pos, b.o_bits);
        if (b.mode == FIC_LOCAL) {
            const int idx = (int)take_bits(words, pos, b.local_bits);
            dx += (idx % b.per - b.rstep) * b.step;
            dy += (idx / b.per - b.rstep) * b.step;
        } else if (b.mode == FIC_EXHAUSTIVE) {
            const int idx = (int)take_bits(words, pos, b.dom_bits);
            dx = (idx % b.ndx) * b.step;
            dy = (idx / b.ndx) * b.step;
            iso = take_bits(words, pos, b.iso_bits);
        }
    } else {
        const int M = level == 1 ? 5 : 6;
        q = take_bits(words, pos, b.o_bits);
        for (int i = 0; i < 3; ++i) {
            int d = (int)take_bits(words, pos, M);
            if (d >= (1 << (M - 1))) d -= 1 << M;
            dz |= ((uint32_t)d & 0xffu) << (8 * i);
        }
        k = take_bits(words, pos, 4);
    }
    return make_uint4((uint32_t)x | ((uint32_t)y << 16), (uint32_t)level | ((uint32_t)phase << 8) | (k << 16) | (q << 24),
                      dz | (iso << 24), (uint32_t)dx | ((uint32_t)dy << 16));
}

// The reader's passes read a block bit by bit: the warp that owns a block
// first copies the block's words into shared memory (coalesced).
constexpr int kParseWarps = 4;
constexpr int kBlockWords = 320;  // words staged per block (larger blocks read global memory)

// Stage the words holding bits [beg, end) of a block, then four zero words
// (reads past the stream's last word give zeros, as get_bits does); returns
// the first staged word, or -1 when the block does not fit the buffer
// (kBlockWords + 4 words).
__device__ __forceinline__ long long stage_block_words(const BitDesc &D, unsigned long long beg, unsigned long long end,
                                                       uint32_t *sw, int lane, int &nstaged) {
    const long long w0 = (long long)(beg >> 5);
    const long long w1 = min(D.nwords, (long long)((end + 63) >> 5));  // + the word a field may reach into
    nstaged = (int)(w1 - w0);
    if (nstaged > kBlockWords || nstaged < 0) return -1;
    for (int i = lane; i < nstaged + 4; i += 32) sw[i] = i < nstaged ? D.words_in[w0 + i] : 0u;
    __syncwarp();
    return w0;
}

__global__ void __launch_bounds__(kParseWarps * 32) parse_count_kernel(const __grid_constant__ BitBatch B) {
    __shared__ uint32_t s_words[kParseWarps][kBlockWords + 4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * kParseWarps + warp;
    if (g >= B.tops_base[B.count]) return;
    const int si = batch_stream(B, g);
    const BitDesc &D = B.d[si];
    const int t = g - B.tops_base[si];
    const unsigned long long beg = D.tile_bits[t], end = D.tile_bits[t + 1];
    int n = -1;
    if (end >= beg && end <= (unsigned long long)D.nwords * 32ull) {
        int nst = 0;
        const long long w0 = stage_block_words(D, beg, end, s_words[warp], lane, nst);
        if (lane == 0)
            n = w0 >= 0 ? walk_tile<false>(D.b, s_words[warp], (uint32_t)(beg - 32ull * (unsigned long long)w0),
                                           (uint32_t)(end - 32ull * (unsigned long long)w0), nullptr, 0)
                        : parse_tile<false>(D.b, D.words_in, D.nwords, beg, end, t, nullptr, nullptr);
    }
    // a block that does not parse is marked by the top bit (the scan finds it)
    if (lane == 0) D.sizes[t] = n < 0 ? (1ull << 63) : (unsigned long long)n;
}

// One CTA per stream: tile offsets of the records, the info block.
__global__ void __launch_bounds__(1024) parse_scan_kernel(const __grid_constant__ BitBatch B) {
    const BitDesc &D = B.d[blockIdx.x];
    const bool bad = cta_scan(D.sizes, D.ntop, D.first);
    if (threadIdx.x == 0) {
        const uint32_t total = bad ? 0u : (uint32_t)D.first[D.ntop];
        D.out_info[FIC_INFO_RECORDS] = total;
        D.out_info[FIC_INFO_ERROR] = bad ? FIC_DEVERR_FORMAT : 0u;
        D.out_info[FIC_INFO_FITS_LO] = 0u;
        D.out_info[FIC_INFO_FITS_HI] = 0u;
        for (int w = FIC_INFO_FITS_HI + 1; w < FIC_INFO_WORDS; ++w) D.out_info[w] = 0u;
        D.out_toff[D.ntop] = total;
    }
}

__global__ void __launch_bounds__(kParseWarps * 32) parse_write_kernel(const __grid_constant__ BitBatch B) {
    __shared__ uint32_t s_words[kParseWarps][kBlockWords + 4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * kParseWarps + warp;
    if (g >= B.tops_base[B.count]) return;
    const int si = batch_stream(B, g);
    const BitDesc &D = B.d[si];
    const int t = g - B.tops_base[si];
    const bool bad = D.out_info[FIC_INFO_ERROR] & FIC_DEVERR_FORMAT;
    if (lane == 0) {
        D.out_toff[t] = bad ? 0u : (uint32_t)D.first[t];
        D.out_split[t] = 0u;
    }
    if (bad) return;
    const unsigned long long beg = D.tile_bits[t], end = D.tile_bits[t + 1];
    int nst = 0;
    const long long w0 = stage_block_words(D, beg, end, s_words[warp], lane, nst);
    if (w0 < 0) {
        if (lane == 0) parse_tile<true>(D.b, D.words_in, D.nwords, beg, end, t, D.out_rec + D.first[t], D.out_split);
        return;
    }
    // lane 0 walks the headers, then the lanes decode the leaves
    __shared__ LeafPos s_leaf[kParseWarps][kTileLeaves];
    int n = 0;
    if (lane == 0)
        n = walk_tile<true>(D.b, s_words[warp], (uint32_t)(beg - 32ull * (unsigned long long)w0),
                            (uint32_t)(end - 32ull * (unsigned long long)w0), s_leaf[warp], kTileLeaves);
    n = __shfl_sync(0xffffffffu, n, 0);  // the count pass found the same blocks well formed
    __syncwarp();
    uint32_t mask = 0;
    fic_record *out = D.out_rec + D.first[t];
    for (int i = lane; i < n; i += 32) {
        const LeafPos lp = s_leaf[warp][i];
        *reinterpret_cast<uint4 *>(out + i) = decode_leaf(D.b, s_words[warp], lp, t);
        for (int a = 1; a < lp.level; ++a)
            mask |= 1u << (((1u << (2 * (a - 1))) - 1) / 3 + (uint32_t)(lp.c >> (2 * (D.b.L - a))));
    }
    mask = __reduce_or_sync(0xffffffffu, mask);
    if (lane == 0) D.out_split[t] = mask;
}

}  // namespace

}  // namespace fic

using namespace fic;

extern "C" {

int64_t fic_bitstream_max_words(int width, int height, const fic_params *p) {
    int32_t ntop = 0, cap = 0;
    if (!p || fic_stream_sizes(width, height, p, &ntop, &cap)) return 0;
    return 2 * (int64_t)cap + 2;  // 64 bits per record bound the widest leaf
}

size_t fic_bitstream_workspace_bytes(int width, int height, const fic_params *p) {
    int32_t ntop = 0, cap = 0;
    if (!p || fic_stream_sizes(width, height, p, &ntop, &cap)) return 0;
    return 8 * ((size_t)ntop + 1) * 2;
}

// Launch the three kernels of a writer (parse = false) or reader batch.
static int run_batch(BitBatch &B, bool parse, cudaStream_t s) {
    B.tops_base[0] = 0;
    for (int i = 0; i < B.count; ++i) B.tops_base[i + 1] = B.tops_base[i] + B.d[i].ntop;
    const int tops = B.tops_base[B.count];
    if (B.count == 0) return FIC_OK;
    if (!parse) {
        const int warps_per_cta = 8;
        const int grid = (tops + warps_per_cta - 1) / warps_per_cta;
        tile_size_kernel<<<grid, warps_per_cta * 32, 0, s>>>(B);
        ser_scan_kernel<<<dim3(B.count, kSerZeroCtas), 1024, 0, s>>>(B);
        write_kernel<<<grid, warps_per_cta * 32, 0, s>>>(B);
    } else {
        const int grid = (tops + kParseWarps - 1) / kParseWarps;
        parse_count_kernel<<<grid, kParseWarps * 32, 0, s>>>(B);
        parse_scan_kernel<<<B.count, 1024, 0, s>>>(B);
        parse_write_kernel<<<grid, kParseWarps * 32, 0, s>>>(B);
    }
    return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

// Each stream's scans at a 256-byte aligned offset; the last one needs only
// its own size (so a batch of one needs fic_bitstream_workspace_bytes).
size_t fic_bitstream_batch_workspace_bytes(const fic_stream *sts, int count) {
    if (!sts || count <= 0) return 0;
    size_t n = 0;
    for (int i = 0; i < count; ++i) {
        const size_t one = fic_bitstream_workspace_bytes(sts[i].width, sts[i].height, &sts[i].params);
        if (one == 0) return 0;
        n += i == count - 1 ? one : (one + 255) & ~(size_t)255;
    }
    return n;
}

int fic_serialize_batch(const fic_stream *sts, int count, int technique2, uint32_t *const *d_words,
                        const int64_t *nwords, uint64_t *const *d_tile_bits, void *d_workspace, size_t ws_bytes,
                        void *stream) {
    if (!sts || count <= 0 || !d_words || !nwords || !d_tile_bits || !d_workspace) return FIC_EBADPARAM;
    if (ws_bytes < fic_bitstream_batch_workspace_bytes(sts, count)) return FIC_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *ws = static_cast<uint8_t *>(d_workspace);
    BitBatch B;
    B.count = 0;
    for (int i = 0; i < count; ++i) {
        const fic_stream *st = &sts[i];
        if (!st->records || !st->tile_offsets || !d_words[i] || !d_tile_bits[i]) return FIC_EBADPARAM;
        const int rc = fic_validate_stream(st->width, st->height, &st->params);
        if (rc) return rc;
        if (nwords[i] < fic_bitstream_max_words(st->width, st->height, &st->params)) return FIC_ENOMEM;
        BitDesc &D = B.d[B.count++];
        D.b = make_layout(st->width, st->height, st->params, technique2);
        D.ntop = st->ntop;
        D.rec = st->records;
        D.toff = st->tile_offsets;
        D.words = d_words[i];
        D.words_in = nullptr;
        D.nwords = nwords[i];
        D.tile_bits = reinterpret_cast<unsigned long long *>(d_tile_bits[i]);
        D.sizes = reinterpret_cast<unsigned long long *>(ws);
        D.first = nullptr;
        D.out_rec = nullptr;
        D.out_toff = D.out_split = D.out_info = nullptr;
        ws += (fic_bitstream_workspace_bytes(st->width, st->height, &st->params) + 255) & ~(size_t)255;
        if (B.count == kBitBatch || i == count - 1) {
            const int rc2 = run_batch(B, false, s);
            if (rc2) return rc2;
            B.count = 0;
        }
    }
    return FIC_OK;
}

int fic_parse_batch(const uint32_t *const *d_words, const int64_t *nwords, const uint64_t *const *d_tile_bits,
                    int technique2, fic_stream *outs, int count, void *d_workspace, size_t ws_bytes, void *stream) {
    if (!outs || count <= 0 || !d_words || !nwords || !d_tile_bits || !d_workspace) return FIC_EBADPARAM;
    if (ws_bytes < fic_bitstream_batch_workspace_bytes(outs, count)) return FIC_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *ws = static_cast<uint8_t *>(d_workspace);
    BitBatch B;
    B.count = 0;
    for (int i = 0; i < count; ++i) {
        fic_stream *out = &outs[i];
        if (!out->records || !out->tile_offsets || !out->split || !out->info || !d_words[i] || !d_tile_bits[i] ||
            nwords[i] <= 0)
            return FIC_EBADPARAM;
        const int rc = fic_validate_stream(out->width, out->height, &out->params);
        if (rc) return rc;
        int32_t ntop = 0, cap = 0;
        fic_stream_sizes(out->width, out->height, &out->params, &ntop, &cap);
        if (out->ntop != ntop || out->capacity < cap) return FIC_ECAPACITY;
        BitDesc &D = B.d[B.count++];
        D.b = make_layout(out->width, out->height, out->params, technique2);
        D.ntop = ntop;
        D.rec = nullptr;
        D.toff = nullptr;
        D.words = nullptr;
        D.words_in = d_words[i];
        D.nwords = nwords[i];
        D.tile_bits = const_cast<unsigned long long *>(reinterpret_cast<const unsigned long long *>(d_tile_bits[i]));
        D.sizes = reinterpret_cast<unsigned long long *>(ws);
        D.first = D.sizes + ntop + 1;
        D.out_rec = out->records;
        D.out_toff = out->tile_offsets;
        D.out_split = out->split;
        D.out_info = out->info;
        ws += (fic_bitstream_workspace_bytes(out->width, out->height, &out->params) + 255) & ~(size_t)255;
        if (B.count == kBitBatch || i == count - 1) {
            const int rc2 = run_batch(B, true, s);
            if (rc2) return rc2;
            B.count = 0;
        }
    }
    return FIC_OK;
}

int fic_serialize(const fic_stream *st, int technique2, uint32_t *d_words, int64_t nwords, uint64_t *d_tile_bits,
                  void *d_workspace, size_t ws_bytes, void *stream) {
    if (!st || !d_words || !d_tile_bits || !d_workspace || !st->records || !st->tile_offsets) return FIC_EBADPARAM;
    int rc = fic_validate_stream(st->width, st->height, &st->params);
    if (rc) return rc;
    if (nwords < fic_bitstream_max_words(st->width, st->height, &st->params) ||
        ws_bytes < fic_bitstream_workspace_bytes(st->width, st->height, &st->params))
        return FIC_ENOMEM;
    return fic_serialize_batch(st, 1, technique2, &d_words, &nwords, &d_tile_bits, d_workspace, ws_bytes, stream);
}

int fic_parse(const uint32_t *d_words, int64_t nwords, const uint64_t *d_tile_bits, int technique2, fic_stream *out,
              void *d_workspace, size_t ws_bytes, void *stream) {
    if (!out || !d_words || !d_tile_bits || !d_workspace || !out->records || !out->tile_offsets || !out->split ||
        !out->info || nwords <= 0)
        return FIC_EBADPARAM;
    int rc = fic_validate_stream(out->width, out->height, &out->params);
    if (rc) return rc;
    int32_t ntop = 0, cap = 0;
    fic_stream_sizes(out->width, out->height, &out->params, &ntop, &cap);
    if (out->ntop != ntop || out->capacity < cap) return FIC_ECAPACITY;
    if (ws_bytes < fic_bitstream_workspace_bytes(out->width, out->height, &out->params)) return FIC_ENOMEM;
    return fic_parse_batch(&d_words, &nwords, &d_tile_bits, technique2, out, 1, d_workspace, ws_bytes, stream);
}

}  // extern "C"
