// transfer.cu -- the records of encoded streams to host memory without a
// round trip to the host.  How many records a stream holds is known only on
// the device (its info block), so a copy engine transfer would have to move
// the whole capacity or wait for the count; here one kernel reads each
// stream's count and copies exactly that many records (and the info block)
// through the device's mapping of the host buffers.
#include <vector>

#include "fic_internal.cuh"

namespace fic {

namespace {

constexpr int kXferBatch = 64;  // streams per launch (descriptors travel as the kernel parameter)

struct XferDesc {
    const uint4 *rec;       // the stream's records (device)
    uint4 *h_rec;           // destination (device address of page-locked host memory)
    const uint32_t *info;   // the stream's info block (device)
    uint32_t *h_info;       // destination of the info block, or null
    uint32_t capacity;
};

struct XferBatch {
    int count;
    XferDesc d[kXferBatch];
};

// blockIdx.y: the stream; the CTAs of x copy strided slices of its records.
__global__ void __launch_bounds__(256) records_to_host_kernel(const __grid_constant__ XferBatch B) {
    const XferDesc &D = B.d[blockIdx.y];
    const uint32_t n = min(D.info[FIC_INFO_RECORDS], D.capacity);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) D.h_rec[i] = D.rec[i];
    if (D.h_info && blockIdx.x == 0 && threadIdx.x < FIC_INFO_WORDS) D.h_info[threadIdx.x] = D.info[threadIdx.x];
}

// The device address of host memory the device can address (page-locked
// memory, or any host memory where the device reads the host's page
// tables), or null when it cannot (or the pointer is not aligned to `align`
// bytes).
template <typename T>
T *mapped(void *h, size_t align) {
    if (!h || (reinterpret_cast<uintptr_t>(h) & (align - 1))) return nullptr;
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        (void)cudaGetLastError();  // not addressable: clear the error the query recorded
        return nullptr;
    }
    return static_cast<T *>(d);
}

}  // namespace

}  // namespace fic

using namespace fic;

extern "C" {

int fic_records_to_host(const fic_stream *sts, int count, fic_record *const *h_records, uint32_t *const *h_info,
                        void *stream) {
    if (!sts || count <= 0 || !h_records) return FIC_EBADPARAM;
    // every argument is checked before anything is enqueued
    std::vector<XferDesc> ds((size_t)count);
    for (int i = 0; i < count; ++i) {
        const fic_stream *st = &sts[i];
        if (!st->records || !st->info || st->capacity < 0) return FIC_EBADPARAM;
        XferDesc &D = ds[(size_t)i];
        D.rec = reinterpret_cast<const uint4 *>(st->records);
        D.info = st->info;
        D.capacity = (uint32_t)st->capacity;
        D.h_rec = mapped<uint4>(h_records[i], 16);
        D.h_info = nullptr;
        if (!D.h_rec) return FIC_EBADPARAM;
        if (h_info) {
            D.h_info = mapped<uint32_t>(h_info[i], 4);
            if (!D.h_info) return FIC_EBADPARAM;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int b = 0; b < count; b += kXferBatch) {
        XferBatch B;
        B.count = count - b < kXferBatch ? count - b : kXferBatch;
        uint32_t max_cap = 1;
        for (int k = 0; k < B.count; ++k) {
            B.d[k] = ds[(size_t)(b + k)];
            if (B.d[k].capacity > max_cap) max_cap = B.d[k].capacity;
        }
        // about 2048 records per CTA of the batch's largest stream, at most 4 CTAs per stream: the
        // copy is bound by the link to the host, and fewer CTAs take fewer SM slots from kernels
        // running beside it (measured with 1, 2, 4 and 8 in a pipeline of encode-decode steps)
        const uint32_t per = (max_cap + 2047u) / 2048u;
        const int gx = per < 4u ? (int)per : 4;
        records_to_host_kernel<<<dim3(gx, B.count), 256, 0, s>>>(B);
        if (cudaGetLastError() != cudaSuccess) return FIC_ECUDA;
    }
    return FIC_OK;
}

}  // extern "C"
