// stats.cu -- position statistics of a transform stream.
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

}  // namespace fic

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
