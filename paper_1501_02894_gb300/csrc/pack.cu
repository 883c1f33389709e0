// pack.cu -- compaction of the per-strip record slots into the canonical
// transform stream (leaves in top-level raster order, depth-first inside
// each top-level block; Section 3.4 relies on this order for Technique 2).
//
// The encoder writes the leaves of strip s to slot s (at most 64 records)
// and the strip's record count.  Here one CTA takes 32 consecutive strips of
// one image: warp 0 scans their counts and looks back over the image's
// earlier chunks (their counts are already final, so the look-back resolves
// in a few rounds), turns the encoder's per-strip tile offsets into stream
// offsets and adds the fit counts to the stream's info block; meanwhile the
// other seven warps load the 32 slots' records into registers (coalesced
// 16-byte loads), and store them at their stream offsets once warp 0 has
// them.  The info block of each stream (record count, fits, device error
// bits) is written here, by the image's last chunk.
#include "fic_internal.cuh"

namespace fic {

constexpr int kPackWarps = 8;
constexpr uint32_t kPAgg = 1u << 30, kPIncl = 2u << 30, kPVal = (1u << 30) - 1;
constexpr int kSlotRecs = 64;

// One CTA per chunk of 32 strips, in block order (lower chunks of an image
// are scheduled first, so a look-back only waits on chunks already running;
// the wait is bounded in any case).
__global__ void __launch_bounds__(kPackWarps * 32)
    pack_kernel(const EncDesc *__restrict__ descs, int count, int total_chunks, uint32_t *__restrict__ pstatus,
                uint32_t *__restrict__ ticket) {
    __shared__ int s_cb[kImgTable];
    __shared__ int s_ok;
    __shared__ uint32_t s_off[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const int c = blockIdx.x;
    // the decoder setup that may follow can be scheduled as this grid's CTAs
    // retire (it waits for this grid's completion before reading its output)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (count <= kImgTable)
        for (int i = threadIdx.x; i < count; i += blockDim.x) s_cb[i] = descs[i].chunk_base;
    __syncthreads();
    // the chunk's image (every warp: the copy warps prefetch below)
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
    // warps 1..7 load their slots' records while warp 0 resolves the offsets
    constexpr int kPer = (32 + kPackWarps - 2) / (kPackWarps - 1);  // slots per copy warp (5)
    uint4 pre[kPer][2];
    uint32_t pre_n[kPer];
    if (warp > 0) {
        const EncDesc &D = descs[lo];
        const int cl = c - D.chunk_base;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
            const int j = (warp - 1) + (kPackWarps - 1) * t;
            const int sidx = cl * 32 + j;
            const uint32_t n = (j < 32 && sidx < D.nstrips) ? D.stats[sidx].x : 0u;
            pre_n[t] = n;
            const fic_record *src = D.slots + (size_t)sidx * kSlotRecs;
            pre[t][0] = (uint32_t)lane < n ? *reinterpret_cast<const uint4 *>(src + lane) : make_uint4(0u, 0u, 0u, 0u);
            pre[t][1] = (uint32_t)lane + 32u < n ? *reinterpret_cast<const uint4 *>(src + lane + 32)
                                                : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (warp == 0) {
        const EncDesc &D = descs[lo];
        const int cl = c - D.chunk_base;
        const int s = cl * 32 + lane;
        const bool in = s < D.nstrips;
        const uint2 st = in ? D.stats[s] : make_uint2(0u, 0u);
        const uint32_t cnt = st.x;
        uint32_t incl = cnt;
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            const uint32_t o = __shfl_up_sync(FULL, incl, m);
            if (lane >= m) incl += o;
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        // look-back over the image's earlier chunks (their counts are final)
        uint32_t prefix = 0;
        int ok = 1;
        if (cl == 0) {
            if (lane == 0) st_volatile(pstatus + c, kPIncl | tot);
        } else {
            if (lane == 0) st_volatile(pstatus + c, kPAgg | tot);
            int p = c - 1;
            for (;;) {
                const int idx = p - lane;
                const bool inimg = idx >= D.chunk_base;
                uint32_t v = inimg ? ld_volatile(pstatus + idx) : kPIncl;
                unsigned it = 0;
                while (!__all_sync(FULL, v != 0u) && ++it < kSpinLimit) {
                    __nanosleep(32);
                    if (v == 0u) v = ld_volatile(pstatus + idx);
                }
                if (!__all_sync(FULL, v != 0u)) {
                    ok = 0;
                    break;
                }
                const uint32_t inc = __ballot_sync(FULL, (v & ~kPVal) == kPIncl);
                const int first = inc ? __ffs(inc) - 1 : 32;
                prefix += __reduce_add_sync(FULL, (lane <= first) ? (v & kPVal) : 0u);
                if (inc) break;
                p -= 32;
            }
            if (lane == 0 && ok) st_volatile(pstatus + c, kPIncl | (prefix + tot));
        }
        const uint32_t excl = prefix + incl - cnt;
        s_off[lane] = excl;
        if (lane == 0) s_ok = ok;
        if (ok && in) {
            // tile offsets: the encoder stored offsets inside the strip
            const int tops = 1024 / (D.bmax * D.bmax);
            const int row = s / D.spr, sc = s - row * D.spr;
            const int top0 = row * D.tw + sc * tops;
            const int nvalid = min(tops, D.tw - sc * tops);
            for (int t = 0; t < nvalid; ++t) D.tile_off[top0 + t] += excl;
        }
        if (cl == D.nchunks - 1) {
            // last chunk of the image: totals, fits and error bits of all its strips
            unsigned long long fsum = 0;
            uint32_t err = ok ? 0u : FIC_DEVERR_TIMEOUT;
            for (int t = lane; t < D.nstrips; t += 32) {
                const uint2 v = D.stats[t];
                fsum += v.y & 0x7fffffffu;
                err |= (v.y >> 31) ? FIC_DEVERR_TIMEOUT : 0u;
            }
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) fsum += __shfl_xor_sync(FULL, fsum, m);
            err = __reduce_or_sync(FULL, err);
            if (ok && prefix + tot > (uint32_t)D.capacity) err |= FIC_DEVERR_CAPACITY;
            if (lane == 0) {
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
    }
    __syncthreads();
    if (!s_ok || warp == 0) return;
    // store the prefetched records at their stream offsets (records past
    // the capacity are dropped; the image's last chunk reports it)
    const EncDesc &D = descs[lo];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int j = (warp - 1) + (kPackWarps - 1) * t;
        if (j >= 32) break;
        const uint32_t n = pre_n[t], off = s_off[j];
        if ((uint32_t)lane < n && off + lane < (uint32_t)D.capacity)
            *reinterpret_cast<uint4 *>(D.rec + off + lane) = pre[t][0];
        if ((uint32_t)lane + 32u < n && off + lane + 32 < (uint32_t)D.capacity)
            *reinterpret_cast<uint4 *>(D.rec + off + lane + 32) = pre[t][1];
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, pack_kernel, d_descs, count, total_chunks, pack_status, ticket);
    stage_mark(st, "pack_kernel");
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fic
