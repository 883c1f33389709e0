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
// over the blocks gives the index, and the warp then writes every leaf's
// fields at its bit offset with atomicOr (fields may straddle words and
// blocks may share a word).  Reader: a thread per block parses it twice --
// once to count its leaves (scanned into tile offsets), once to write the
// records, split masks and the record count.
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

// ---- writer

__global__ void tile_size_kernel(BitLayout b, const fic_record *__restrict__ rec, const uint32_t *__restrict__ toff,
                                 int ntop, unsigned long long *__restrict__ sizes) {
    const int lane = threadIdx.x & 31;
    const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= ntop) return;
    const uint32_t beg = toff[t], end = toff[t + 1];
    unsigned long long s = 0;
    for (uint32_t i = beg + lane; i < end; i += 32) s += (unsigned)leaf_bits(b, *reinterpret_cast<const uint4 *>(rec + i));
    for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) sizes[t] = s;
}

__global__ void write_kernel(BitLayout b, const fic_record *__restrict__ rec, const uint32_t *__restrict__ toff,
                             int ntop, const unsigned long long *__restrict__ tile_bits, uint32_t *__restrict__ words) {
    const int lane = threadIdx.x & 31;
    const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= ntop) return;
    const uint32_t beg = toff[t], end = toff[t + 1];
    unsigned long long base = tile_bits[t];
    for (uint32_t i0 = beg; i0 < end; i0 += 32) {
        const uint32_t i = i0 + lane;
        const bool has = i < end;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        uint32_t v[9];
        int n[9];
        int f = 0, s = 0;
        if (has) {
            r = *reinterpret_cast<const uint4 *>(rec + i);
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
            put_bits(words, pos, v[j], n[j]);
            pos += (unsigned)n[j];
        }
        base += (unsigned)__shfl_sync(0xffffffffu, incl, 31);
    }
}

// Exclusive scan of n uint64 values into out[0..n] (out[n] = total) by one
// CTA: each thread sums a contiguous slice, the CTA scans the slice sums,
// and each thread writes its slice.
__global__ void scan_kernel(const unsigned long long *__restrict__ in, int n, unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s_part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    unsigned long long s = 0;
    for (int i = lo; i < hi; ++i) s += in[i];
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

__global__ void parse_count_kernel(BitLayout b, const uint32_t *__restrict__ words, long long nwords,
                                   const unsigned long long *__restrict__ tile_bits, int ntop,
                                   unsigned long long *__restrict__ counts, uint32_t *__restrict__ info) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntop; t += gridDim.x * blockDim.x) {
        const unsigned long long beg = tile_bits[t], end = tile_bits[t + 1];
        int n = -1;
        if (end >= beg && end <= (unsigned long long)nwords * 32ull)
            n = parse_tile<false>(b, words, nwords, beg, end, t, nullptr, nullptr);
        if (n < 0) {
            atomicOr(info + FIC_INFO_ERROR, FIC_DEVERR_FORMAT);
            n = 0;
        }
        counts[t] = (unsigned long long)n;
    }
}

__global__ void parse_write_kernel(BitLayout b, const uint32_t *__restrict__ words, long long nwords,
                                   const unsigned long long *__restrict__ tile_bits, int ntop,
                                   const unsigned long long *__restrict__ first, fic_record *__restrict__ rec,
                                   uint32_t *__restrict__ toff, uint32_t *__restrict__ split,
                                   uint32_t *__restrict__ info) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntop; t += gridDim.x * blockDim.x) {
        toff[t] = (uint32_t)first[t];
        split[t] = 0u;
        if (info[FIC_INFO_ERROR] & FIC_DEVERR_FORMAT) continue;
        parse_tile<true>(b, words, nwords, tile_bits[t], tile_bits[t + 1], t, rec + first[t], split);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        toff[ntop] = (uint32_t)first[ntop];
        info[FIC_INFO_RECORDS] = (uint32_t)first[ntop];
        info[FIC_INFO_FITS_LO] = 0u;
        info[FIC_INFO_FITS_HI] = 0u;
    }
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

int fic_serialize(const fic_stream *st, int technique2, uint32_t *d_words, int64_t nwords, uint64_t *d_tile_bits,
                  void *d_workspace, size_t ws_bytes, void *stream) {
    if (!st || !d_words || !d_tile_bits || !d_workspace || !st->records || !st->tile_offsets) return FIC_EBADPARAM;
    int rc = fic_validate_stream(st->width, st->height, &st->params);
    if (rc) return rc;
    if (nwords < fic_bitstream_max_words(st->width, st->height, &st->params) ||
        ws_bytes < fic_bitstream_workspace_bytes(st->width, st->height, &st->params))
        return FIC_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const BitLayout b = make_layout(st->width, st->height, st->params, technique2);
    const int ntop = st->ntop;
    unsigned long long *sizes = static_cast<unsigned long long *>(d_workspace);
    if (cudaMemsetAsync(d_words, 0, (size_t)nwords * 4, s) != cudaSuccess) return FIC_ECUDA;
    const int warps_per_cta = 8;
    const int grid = (ntop + warps_per_cta - 1) / warps_per_cta;
    tile_size_kernel<<<grid, warps_per_cta * 32, 0, s>>>(b, st->records, st->tile_offsets, ntop, sizes);
    scan_kernel<<<1, 1024, 0, s>>>(sizes, ntop, reinterpret_cast<unsigned long long *>(d_tile_bits));
    write_kernel<<<grid, warps_per_cta * 32, 0, s>>>(b, st->records, st->tile_offsets, ntop,
                                                     reinterpret_cast<const unsigned long long *>(d_tile_bits),
                                                     d_words);
    return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
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
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const BitLayout b = make_layout(out->width, out->height, out->params, technique2);
    unsigned long long *counts = static_cast<unsigned long long *>(d_workspace);
    unsigned long long *first = counts + ntop + 1;
    if (cudaMemsetAsync(out->info, 0, FIC_INFO_WORDS * 4, s) != cudaSuccess) return FIC_ECUDA;
    const int threads = 128;
    int grid = (ntop + threads - 1) / threads;
    grid = grid < 1 ? 1 : grid;
    const unsigned long long *tb = reinterpret_cast<const unsigned long long *>(d_tile_bits);
    parse_count_kernel<<<grid, threads, 0, s>>>(b, d_words, nwords, tb, ntop, counts, out->info);
    scan_kernel<<<1, 1024, 0, s>>>(counts, ntop, first);
    parse_write_kernel<<<grid, threads, 0, s>>>(b, d_words, nwords, tb, ntop, first, out->records, out->tile_offsets,
                                                out->split, out->info);
    return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

}  // extern "C"
