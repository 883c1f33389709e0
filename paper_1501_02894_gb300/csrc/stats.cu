// stats.cu -- stream utilities: position statistics and rescaling.
//
// Section 2 of the paper motivates local search with the distributions of
// the differences x_d - x_r and y_d - y_r between the position of each range
// block and the position of the domain block an exhaustive search picked
// for it (its Figs. 2 and 3).  fic_offset_histogram counts those
// differences over a stream's records on the device.
#include "fic_internal.cuh"

namespace fic {

// One thread per record; the record count is read from the stream's info
// block, so the launch needs no host synchronisation.
__global__ void offset_histogram_kernel(const fic_record *__restrict__ rec, const uint32_t *__restrict__ info,
                                        int capacity, int W, int H, uint32_t *__restrict__ hx,
                                        uint32_t *__restrict__ hy) {
    const uint32_t n = min(info[FIC_INFO_RECORDS], (uint32_t)capacity);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 r = *reinterpret_cast<const uint4 *>(rec + i);
        const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16);
        const int dx = (int)(r.w & 0xffffu), dy = (int)(r.w >> 16);
        const int bx = dx - x + W, by = dy - y + H;
        if (bx >= 0 && bx < 2 * W) atomicAdd(hx + bx, 1u);
        if (by >= 0 && by < 2 * H) atomicAdd(hy + by, 1u);
    }
}

// Rescale by 2^shift: positions and domains scaled, codes kept.  One
// thread per record; tile offsets (ntop + 1), split masks and the info
// block are copied (the top-level order is unchanged by the scaling).
__global__ void rescale_kernel(const fic_record *__restrict__ in, const uint32_t *__restrict__ toff_in,
                               const uint32_t *__restrict__ split_in, const uint32_t *__restrict__ info_in,
                               int capacity, int ntop, int shift, fic_record *__restrict__ out,
                               uint32_t *__restrict__ toff_out, uint32_t *__restrict__ split_out,
                               uint32_t *__restrict__ info_out) {
    const uint32_t n = min(info_in[FIC_INFO_RECORDS], (uint32_t)capacity);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (uint32_t i = tid; i < n; i += nt) {
        uint4 r = *reinterpret_cast<const uint4 *>(in + i);
        uint32_t xy = r.x, dxy = r.w;
        if (shift > 0) {
            xy = (xy & 0x7fff7fffu) << 1;
            dxy = (dxy & 0x7fff7fffu) << 1;
        } else {
            xy = (xy >> 1) & 0x7fff7fffu;
            dxy = (dxy >> 1) & 0x7fff7fffu;
        }
        r.x = xy;
        r.w = dxy;
        *reinterpret_cast<uint4 *>(out + i) = r;
    }
    for (int t = tid; t <= ntop; t += nt) {
        toff_out[t] = toff_in[t];
        if (t < ntop) split_out[t] = split_in[t];
    }
    if (tid < FIC_INFO_WORDS) info_out[tid] = info_in[tid];
}

}  // namespace fic

extern "C" int fic_rescale_params(int width, int height, const fic_params *p, int shift, int *width_out,
                                  int *height_out, fic_params *p_out) {
    if (!p || !width_out || !height_out || !p_out || (shift != 1 && shift != -1)) return FIC_EBADPARAM;
    int rc = fic_validate_stream(width, height, p);
    if (rc) return rc;
    fic_params q = *p;
    int W = width, H = height;
    if (shift > 0) {
        W *= 2;
        H *= 2;
        q.bmax *= 2;
        q.bmin *= 2;
        q.local_radius *= 2;
        q.local_step *= 2;
        q.dom_step *= 2;
    } else {
        if ((q.bmin | W | H | q.local_radius | q.local_step | q.dom_step) & 1) return FIC_EBADPARAM;
        W /= 2;
        H /= 2;
        q.bmax /= 2;
        q.bmin /= 2;
        q.local_radius /= 2;
        q.local_step /= 2;
        q.dom_step /= 2;
    }
    rc = fic_validate_stream(W, H, &q);
    if (rc) return FIC_EBADPARAM;
    *width_out = W;
    *height_out = H;
    *p_out = q;
    return FIC_OK;
}

extern "C" int fic_stream_rescale(const fic_stream *in, int shift, fic_stream *out, void *stream) {
    using namespace fic;
    if (!in || !out || !in->records || !in->tile_offsets || !in->split || !in->info || !out->records ||
        !out->tile_offsets || !out->split || !out->info)
        return FIC_EBADPARAM;
    int W = 0, H = 0;
    fic_params q;
    int rc = fic_rescale_params(in->width, in->height, &in->params, shift, &W, &H, &q);
    if (rc) return rc;
    if (out->width != W || out->height != H || out->params.bmax != q.bmax || out->params.bmin != q.bmin ||
        out->ntop != in->ntop || out->capacity < in->capacity)
        return FIC_EBADPARAM;
    const int threads = 256;
    int blocks = (in->capacity + threads - 1) / threads;
    blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
    rescale_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        in->records, in->tile_offsets, in->split, in->info, in->capacity, in->ntop, shift, out->records,
        out->tile_offsets, out->split, out->info);
    return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

extern "C" int fic_offset_histogram(const fic_stream *st, uint32_t *d_hx, uint32_t *d_hy, void *stream) {
    using namespace fic;
    if (!st || !d_hx || !d_hy || !st->records || !st->info || st->width <= 0 || st->height <= 0 || st->capacity < 0)
        return FIC_EBADPARAM;
    const int threads = 256;
    int blocks = (st->capacity + threads - 1) / threads;
    blocks = blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks);
    offset_histogram_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        st->records, st->info, st->capacity, st->width, st->height, d_hx, d_hy);
    return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded device waits every kernel uses: a spin on a word
// that nothing writes and an mbarrier wait for a transfer that never comes
// must both give up after their iteration limits and report it, leaving the
// context usable.  out[0] = 1 when the word spin gave up, out[1] = 1 when the
// mbarrier wait gave up, out[2] = the spin's iterations.
namespace fic {
__global__ void selftest_waits_kernel(const uint32_t *never, uint32_t *out, unsigned spin_limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    unsigned it = 0;
    uint32_t v = ld_volatile(never);
    while (v == 0u && ++it < spin_limit) {
        __nanosleep(32);
        v = ld_volatile(never);
    }
    out[0] = v == 0u ? 1u : 0u;
    out[2] = it;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16u);  // 16 bytes announced, none sent
    out[1] = mbar_wait(&bar, 0u, kMbarLimit) ? 0u : 1u;
}
}  // namespace fic

extern "C" int fic_selftest_waits(const uint32_t *d_never, uint32_t *d_out, void *stream) {
    if (!d_never || !d_out) return FIC_EBADPARAM;
    fic::selftest_waits_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(d_never, d_out, fic::kSpinLimit);
    return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}
