// pack.cuh -- one warp packs one chunk of 32 strips: the chunk's stream
// offset by a decoupled look-back over the image's earlier chunks, the tile
// offsets of its top-level blocks, the image's totals when it is the
// image's last chunk, and the copy of its record slots into the stream.
// Used by the MNS encoder, whose warp that completes a chunk's last strip
// packs the chunk (so no separate pack launch is needed).
#pragma once

#include "fic_internal.cuh"

namespace fic {

constexpr uint32_t kPkAgg = 1u << 30, kPkIncl = 2u << 30, kPkVal = (1u << 30) - 1;

// Loads of what other warps wrote (after their fence and the chunk counter):
// at L2, not through this SM's L1.
__device__ __forceinline__ uint2 ld_cg2(const uint2 *p) { return __ldcg(p); }
__device__ __forceinline__ uint4 ld_cg4(const fic_record *p) { return __ldcg(reinterpret_cast<const uint4 *>(p)); }

// Returns false when the look-back wait ran out (the image's error bit is
// raised and nothing is copied).  Chunk status words start at zero.
__device__ __forceinline__ bool pack_chunk_warp(const EncDesc &D, int cl, uint32_t *__restrict__ pstatus, int lane) {
    const unsigned FULL = 0xffffffffu;
    const int c = D.chunk_base + cl;
    const int s = cl * 32 + lane;
    const bool in = s < D.nstrips;
    const uint2 st = in ? ld_cg2(D.stats + s) : make_uint2(0u, 0u);
    const uint32_t cnt = st.x;
    uint32_t incl = cnt;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        const uint32_t o = __shfl_up_sync(FULL, incl, m);
        if (lane >= m) incl += o;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    uint32_t prefix = 0;
    bool ok = true;
    if (cl == 0) {
        if (lane == 0) st_volatile(pstatus + c, kPkIncl | tot);
    } else {
        if (lane == 0) st_volatile(pstatus + c, kPkAgg | tot);
        int p = c - 1;
        for (;;) {
            const int idx = p - lane;
            const bool inimg = idx >= D.chunk_base;
            uint32_t v = inimg ? ld_volatile(pstatus + idx) : kPkIncl;
            unsigned it = 0;
            while (!__all_sync(FULL, v != 0u) && ++it < kSpinLimit) {
                __nanosleep(64);
                if (v == 0u) v = ld_volatile(pstatus + idx);
            }
            if (!__all_sync(FULL, v != 0u)) {
                ok = false;
                break;
            }
            const uint32_t inc = __ballot_sync(FULL, (v & ~kPkVal) == kPkIncl);
            const int first = inc ? __ffs(inc) - 1 : 32;
            prefix += __reduce_add_sync(FULL, (lane <= first) ? (v & kPkVal) : 0u);
            if (inc) break;
            p -= 32;
        }
        if (lane == 0 && ok) st_volatile(pstatus + c, kPkIncl | (prefix + tot));
    }
    __threadfence();  // what the chunks before published is read below
    const uint32_t excl = prefix + incl - cnt;
    if (ok && in) {
        // the encoder stored each top-level block's offset inside its strip
        const int tops = 1024 / (D.bmax * D.bmax);
        const int row = s / D.spr, sc = s - row * D.spr;
        const int top0 = row * D.tw + sc * tops;
        const int nvalid = min(tops, D.tw - sc * tops);
        for (int t = 0; t < nvalid; ++t) atomicAdd(D.tile_off + top0 + t, excl);  // at L2: written by other warps
    }
    if (cl == D.nchunks - 1) {
        // the image's last chunk: totals, fits and error bits of all its strips
        unsigned long long fsum = 0;
        uint32_t err = ok ? 0u : FIC_DEVERR_TIMEOUT;
        for (int t = lane; t < D.nstrips; t += 32) {
            const uint2 v = ld_cg2(D.stats + t);
            fsum += v.y & 0x7fffffffu;
            err |= (v.y >> 31) ? FIC_DEVERR_TIMEOUT : 0u;
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) fsum += __shfl_xor_sync(FULL, fsum, m);
        err = __reduce_or_sync(FULL, err);
        if (ok && prefix + tot > (uint32_t)D.capacity) err |= FIC_DEVERR_CAPACITY;
        if (lane == 0) {
            // the info block is written here only (it may hold anything before)
            D.info[FIC_INFO_FITS_LO] = (uint32_t)fsum;
            D.info[FIC_INFO_FITS_HI] = (uint32_t)(fsum >> 32);
            D.info[FIC_INFO_ERROR] = err;
            if (ok) {
                D.tile_off[D.tw * D.th] = prefix + tot;
                D.info[FIC_INFO_RECORDS] = prefix + tot;
            }
        }
    } else if (!ok && lane == 0) {
        raise_error(D.info, FIC_DEVERR_TIMEOUT);
    }
    if (!ok) return false;
    // records past the capacity are dropped (the image's last chunk reports it)
    // copy the 32 slots: lane-strided over each slot's records
    for (int j = 0; j < 32 && cl * 32 + j < D.nstrips; ++j) {
        const uint32_t n = __shfl_sync(FULL, cnt, j), off = __shfl_sync(FULL, excl, j);
        const fic_record *src = D.slots + (size_t)(cl * 32 + j) * D.slot_recs;
        for (uint32_t k = lane; k < n; k += 32) {
            if (off + k < (uint32_t)D.capacity) *reinterpret_cast<uint4 *>(D.rec + off + k) = ld_cg4(src + k);
        }
    }
    return true;
}

}  // namespace fic
