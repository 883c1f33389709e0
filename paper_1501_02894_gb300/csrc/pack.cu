// pack.cu -- compaction of the per-strip record slots into the canonical
// transform stream (leaves in top-level raster order, depth-first inside
// each top-level block; Section 3.4 relies on this order for Technique 2).
//
// The encoder writes the leaves of strip s to slot s (at most 64 records)
// and the strip's record count.  Here one CTA takes 32 consecutive strips of
// one image.  Every count is final when this kernel runs, so a chunk needs
// no other chunk's result: the CTA sums the counts of all of the image's
// earlier strips itself (each thread a strided share, then one block
// reduction) -- no look-back, no wait on another CTA.  Meanwhile its copy
// warps load the 32 slots' records into registers (coalesced 16-byte
// loads); warp 0 scans the chunk's counts, fixes the tile offsets, and the
// copy warps store the records at their stream offsets.  The image's last
// chunk also writes the stream's info block (record count, fits, device
// error bits), summing the fits of all of the image's strips in the same
// strided pass.
#include "fic_internal.cuh"

namespace fic {

constexpr int kPackWarps = 8;

__global__ void __launch_bounds__(kPackWarps * 32)
    pack_kernel(const EncDesc *__restrict__ descs, int count, int total_chunks, uint32_t *__restrict__ ticket) {
    __shared__ int s_cb[kImgTable];
    __shared__ uint32_t s_off[32];
    __shared__ uint32_t s_part[kPackWarps];
    __shared__ unsigned long long s_fits[kPackWarps];
    __shared__ uint32_t s_err[kPackWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const int c = blockIdx.x;
    // the decoder setup that may follow can be scheduled as this grid's CTAs
    // retire (it waits for this grid's completion before reading its output)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (count <= kImgTable)
        for (int i = threadIdx.x; i < count; i += blockDim.x) s_cb[i] = descs[i].chunk_base;
    __syncthreads();
    // the chunk's image
    int lo = 0;
    {
        int hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            const int cb = count <= kImgTable ? s_cb[mid] : descs[mid].chunk_base;
            if (cb <= c) lo = mid;
            else hi = mid - 1;
        }
    }
    // Programmatic dependent launch: the prologue above (descriptors written
    // by the host) may overlap the encoder's tail; everything the encoder
    // wrote is read after it has completed.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // the encoder's strip counter (dynamic schedule) is free again: reset it
    // for the next launch
    if (ticket && c == 0 && threadIdx.x == 0) *ticket = 0u;
    const EncDesc &D = descs[lo];
    const int cl = c - D.chunk_base;
    const bool last = cl == D.nchunks - 1;
    // copy warps: their slots' records into registers
    constexpr int kPer = (32 + kPackWarps - 2) / (kPackWarps - 1);  // slots per copy warp (5)
    uint4 pre[kPer][2];
    uint32_t pre_n[kPer];
    if (warp > 0) {
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int j = (warp - 1) + (kPackWarps - 1) * t;
            const int sidx = cl * 32 + j;
            const uint32_t n = (j < 32 && sidx < D.nstrips) ? D.stats[sidx].x : 0u;
            pre_n[t] = n;
            const fic_record *src = D.slots + (size_t)sidx * D.slot_recs;
            pre[t][0] = (uint32_t)lane < n ? *reinterpret_cast<const uint4 *>(src + lane) : make_uint4(0u, 0u, 0u, 0u);
            pre[t][1] = (uint32_t)lane + 32u < n ? *reinterpret_cast<const uint4 *>(src + lane + 32)
                                                : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    // records of the image's earlier strips (and, in the last chunk, the fits
    // and error flags of all of its strips)
    uint32_t part = 0, err = 0;
    unsigned long long fs = 0;
    {
        const int before = cl * 32, end = last ? D.nstrips : before;
        for (int i = threadIdx.x; i < end; i += kPackWarps * 32) {
            const uint2 v = D.stats[i];
            if (i < before) part += v.x;
            fs += v.y & 0x7fffffffu;
            err |= v.y >> 31;
        }
    }
    part = __reduce_add_sync(FULL, part);
    err = __reduce_or_sync(FULL, err);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) fs += __shfl_xor_sync(FULL, fs, m);
    if (lane == 0) {
        s_part[warp] = part;
        s_fits[warp] = fs;
        s_err[warp] = err;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t prefix = lane < kPackWarps ? s_part[lane] : 0u;
        prefix = __reduce_add_sync(FULL, prefix);
        const int s = cl * 32 + lane;
        const bool in = s < D.nstrips;
        const uint32_t cnt = in ? D.stats[s].x : 0u;
        uint32_t incl = cnt;
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            const uint32_t o = __shfl_up_sync(FULL, incl, m);
            if (lane >= m) incl += o;
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        const uint32_t excl = prefix + incl - cnt;
        s_off[lane] = excl;
        if (in) {
            // tile offsets: the encoder stored each block's offset inside its
            // strip (0 when a strip is one block)
            const int tops = 1024 / (D.bmax * D.bmax);
            const int row = s / D.spr, sc = s - row * D.spr;
            const int top0 = row * D.tw + sc * tops;
            if (tops == 1) {
                D.tile_off[top0] = excl;
            } else {
                const int nvalid = min(tops, D.tw - sc * tops);
                for (int t = 0; t < nvalid; ++t) D.tile_off[top0 + t] += excl;
            }
        }
        if (last) {
            unsigned long long fsum = lane < kPackWarps ? s_fits[lane] : 0ull;
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) fsum += __shfl_xor_sync(FULL, fsum, m);
            uint32_t e = __reduce_or_sync(FULL, lane < kPackWarps ? s_err[lane] : 0u) ? FIC_DEVERR_TIMEOUT : 0u;
            if (prefix + tot > (uint32_t)D.capacity) e |= FIC_DEVERR_CAPACITY;
            if (lane == 0) {
                // the info block is written here only (it may hold anything before)
                D.info[FIC_INFO_FITS_LO] = (uint32_t)fsum;
                D.info[FIC_INFO_FITS_HI] = (uint32_t)(fsum >> 32);
                D.info[FIC_INFO_ERROR] = e;
                D.tile_off[D.tw * D.th] = prefix + tot;
                D.info[FIC_INFO_RECORDS] = prefix + tot;
            }
        }
    }
    __syncthreads();
    if (warp == 0) return;
    // store the prefetched records at their stream offsets (records past
    // the capacity are dropped; the image's last chunk reports it)
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int j = (warp - 1) + (kPackWarps - 1) * t;
        if (j >= 32) break;
        const uint32_t n = pre_n[t], off = s_off[j];
        if ((uint32_t)lane < n && off + lane < (uint32_t)D.capacity)
            *reinterpret_cast<uint4 *>(D.rec + off + lane) = pre[t][0];
        if ((uint32_t)lane + 32u < n && off + lane + 32 < (uint32_t)D.capacity)
            *reinterpret_cast<uint4 *>(D.rec + off + lane + 32) = pre[t][1];
        // slots of 2 x 2 leaves hold up to 256 records: the rest directly
        if (n > 64u) {
            const fic_record *src = D.slots + (size_t)(cl * 32 + j) * D.slot_recs;
            for (uint32_t k = 64u + (uint32_t)lane; k < n; k += 32u)
                if (off + k < (uint32_t)D.capacity)
                    *reinterpret_cast<uint4 *>(D.rec + off + k) = *reinterpret_cast<const uint4 *>(src + k);
        }
    }
}

cudaError_t launch_pack(const EncDesc *d_descs, int count, int total_chunks, uint32_t *pack_status,
                        uint32_t *ticket, cudaStream_t st) {
    if (total_chunks <= 0) return cudaSuccess;
    // a programmatic dependent of the encoder kernel (see griddepcontrol.wait above)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total_chunks);
    cfg.blockDim = dim3(kPackWarps * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    (void)pack_status;  // the look-back words are used by fused packing only
    cudaError_t e = cudaLaunchKernelEx(&cfg, pack_kernel, d_descs, count, total_chunks, ticket);
    stage_mark(st, "pack_kernel");
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fic
