// fic_internal.cuh -- device-side types and helpers shared by the kernels of
// libfic.so (not part of the public ABI).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fic.h"
#include "tma.cuh"

namespace fic {

// Bounded spin: a wait that has not finished after this many polls gives up,
// records FIC_DEVERR_TIMEOUT and lets the kernel return.
constexpr unsigned kSpinLimit = 1u << 22;
// Polls of an mbarrier before a TMA copy is declared lost.
constexpr unsigned kMbarLimit = 1u << 20;

// One image of an encode launch.
struct EncDesc {
    const uint8_t *img;
    fic_record *rec;
    uint32_t *tile_off;
    uint32_t *split;
    uint32_t *info;
    int64_t t2q[4];      // round(256 T_j^2) per level
    int32_t W, H;
    int32_t tw, th;      // top-level blocks per row / column
    int32_t spr;         // strips per top-block row
    int32_t strip_base;  // global index of this image's first strip
    int32_t nstrips;
    int32_t capacity;
    int32_t mode, bmin, L, phase2;
    int32_t s_bits, o_bits;
    int32_t local_radius, local_step;
    int32_t phase2_domain;  // 0: sub-blocks' own centred domains, 1: parent-domain quadrants
    const TmaMap *map;   // 2-D tensor map of the image (box: the strip's domain window)
    int32_t boxw;        // box width in pixels (= row pitch of the staged window)
    int32_t bmax;
    fic_record *slots;   // slot variant: slot_recs records per strip (workspace)
    int32_t slot_recs;   // records a strip can emit: 64, or 256 when bmin is 2
    uint2 *stats;        // slot variant: per strip (record count, fits)
    int32_t chunk_base;  // slot variant: first 32-strip chunk of the image (pack kernel)
    int32_t nchunks;
};

// Box of the TMA window load for strips of top-level side BMAX: columns
// (16-aligned) x rows.  The window of a strip is at most this wide.
template <int BMAX>
struct WinBox {
    static constexpr int W = BMAX == 32 ? 64 : (BMAX == 16 ? 96 : 160);
    static constexpr int H = 2 * BMAX;
};

// The driver's cuTensorMapEncodeTiled, looked up once per process through
// the runtime's entry-point query (thread safe); null if unavailable.
void *tensor_map_encoder();

// Build the tensor map of a W x H image of uint8 (elem_bytes 1) or uint16
// (elem_bytes 2) elements, rows W elements apart, for boxes of boxw x boxh
// elements (host side; the driver entry point is looked up once).
int make_tma_map(TmaMap *out, const void *base, int W, int H, int boxw, int boxh, int elem_bytes = 1);

// Launch facts of one kernel, per device: its dynamic shared-memory limit is
// set on each device once (a per-device attribute) and the SM count and
// resident CTAs per SM are kept.  Thread safe: the setup is idempotent and
// the results are atomics.
constexpr int kMaxDevices = 64;
struct KernelSlots {
    std::atomic<int> sms[kMaxDevices];
    std::atomic<int> per[kMaxDevices];
};

inline cudaError_t kernel_slots(KernelSlots &ks, const void *fn, int threads, size_t smem, int &sms, int &per) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int p = ks.per[dev].load(std::memory_order_acquire);
    if (p == 0) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int s = 0, q = 0;
        e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, fn, threads, smem);
        if (e != cudaSuccess) return e;
        ks.sms[dev].store(s, std::memory_order_relaxed);
        p = q > 0 ? q : 1;
        ks.per[dev].store(p, std::memory_order_release);
    }
    sms = ks.sms[dev].load(std::memory_order_relaxed);
    per = p;
    return cudaSuccess;
}

// Launch `kernel` as a programmatic dependent of the previous kernel on the
// stream (it must execute griddepcontrol.wait before touching anything that
// kernel wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Per-kernel timing of a plan run (fic_plan_run_timed): launchers call this
// after every kernel launch; it records an event only while a timed run is
// active on the calling thread.
void stage_mark(cudaStream_t st, const char *label);

// Launch mapping of the batched encoder and decoder (chosen by the
// autotuner; every choice produces the same output).
struct EncTune {
    int warps = 8;        // warps per CTA: 8 or 4 (one strip per warp at a time)
    int ctas_per_sm = 0;  // resident CTAs per SM; 0 = the occupancy limit
    int dynamic = 0;      // 1: strips from an atomic counter, 0: static grid stride
    int fused_pack = 0;   // 1: the warp finishing a chunk packs it; 0: a separate pack kernel
                          // (measured faster: the per-strip release fence costs more than the launch)
    int kernel32 = 0;     // set by the plan: 1 = mns_encode32_kernel (bmax 32, sub-blocks on their
                          // own centred domains), 0 = the general mns_encode_kernel
    int min2 = 0;         // set by the plan: a stream of the batch has 2 x 2 leaves
};
struct DecTune {
    int ctas_per_sm = 0;    // resident CTAs per SM of the iteration kernel; 0 = the occupancy limit
    int single_launch = 0;  // 2x2-sum path: 1 = iterations after the first in one cooperative launch
                            // with grid barriers, 0 = one launch per iteration (measured faster: the
                            // dependent launches overlap each iteration's ramp with the previous tail
                            // better than a grid barrier does)
};

// One image of a decode launch.
struct DecDesc {
    const fic_record *rec;
    const uint32_t *tile_off;
    uint8_t *buf[2];     // ping-pong iterates; the last iteration writes buf[0]
    int32_t W, H;
    int32_t tw, th, spr, strip_base, nstrips;
    int32_t mode, bmin, L, s_bits, o_bits;
    int32_t phase2_domain;  // as in fic_params
    // 2x2-sum iteration (centred streams): ping-pong (W/2) x (H/2) images of
    // 2x2 sums, their tensor maps, and the stream's info block for errors
    uint16_t *d4[2];
    const TmaMap *map[2];
    uint32_t *info;
};

// Fixed-point codebooks (Section 3.3): c = 128 s on 2^s_bits cell midpoints
// of [-1, 1); luminance levels round(255 q / (2^o_bits - 1)).
__host__ __device__ inline int contrast_code(int k, int s_bits) {
    const int K = 1 << s_bits;
    return (2 * k - (K - 1)) * (128 >> s_bits);  // 128 / K, K a power of two <= 128
}

// Phase-2 contrast sets of Section 3.2 in the c = round(128 s) fixed point:
// level 1 {.2, .5}, level 2 {.4, .65}, level 3 {.5, .9}.
__host__ __device__ inline int phase2_code(int level, int bit) {
    // level 1 (26, 64), level 2 (51, 83), level 3 (64, 115); selects, not a
    // table (an indexed local array would live in local memory)
    const int lo = level == 1 ? 26 : (level == 2 ? 51 : 64);
    const int hi = level == 1 ? 64 : (level == 2 ? 83 : 115);
    return bit ? hi : lo;
}

// Multiplier of the luminance level L(q) = floor((510 q + ko1) / (2 ko1))
// by a multiply-high, ko1 = 2^o_bits - 1: ceil(2^32 / (2 ko1)), exact for
// q <= ko1 <= 255.  A table over o_bits = 1..8 (the encoders and the decoder
// would otherwise do a 64-bit division per strip).
constexpr uint32_t lum_magic_of(int o_bits) {
    return (uint32_t)((0x100000000ULL + 2ULL * ((1ULL << o_bits) - 1) - 1) / (2ULL * ((1ULL << o_bits) - 1)));
}
constexpr bool lum_magic_exact(int o_bits) {
    const uint64_t ko1 = (1ULL << o_bits) - 1, m = lum_magic_of(o_bits);
    for (uint64_t q = 0; q <= ko1; ++q)
        if ((((510 * q + ko1) * m) >> 32) != (510 * q + ko1) / (2 * ko1)) return false;
    return true;
}
static_assert(lum_magic_exact(1) && lum_magic_exact(2) && lum_magic_exact(3) && lum_magic_exact(4) &&
                  lum_magic_exact(5) && lum_magic_exact(6) && lum_magic_exact(7) && lum_magic_exact(8),
              "multiply-high luminance levels are exact for every code");
__constant__ const uint32_t c_lum_magic[9] = {0u,              lum_magic_of(1), lum_magic_of(2),
                                              lum_magic_of(3), lum_magic_of(4), lum_magic_of(5),
                                              lum_magic_of(6), lum_magic_of(7), lum_magic_of(8)};
// ko1 / 255 for the encoders' float estimate of the luminance code.
__constant__ const float c_lum_qscale[9] = {0.f,          1.f / 255.f,  3.f / 255.f,  7.f / 255.f,  15.f / 255.f,
                                            31.f / 255.f, 63.f / 255.f, 127.f / 255.f, 255.f / 255.f};

__host__ __device__ inline int clampi(int v, int lo, int hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// Domain with the same centre as the range, moved inside the image.
__host__ __device__ inline int centred_origin(int x, int B, int W) {
    return clampi(x - B / 2, 0, W - 2 * B);
}

__device__ __forceinline__ unsigned dp2a_lo(unsigned a, unsigned b, unsigned c) {
    return __dp2a_lo(a, b, c);
}
__device__ __forceinline__ unsigned dp2a_hi(unsigned a, unsigned b, unsigned c) {
    return __dp2a_hi(a, b, c);
}

// Two 2x2 sums from two 4-pixel words of adjacent rows: returns the packed
// pair (p0+p1+q0+q1, p2+p3+q2+q3) as two 16-bit lanes.
__device__ __forceinline__ unsigned d4_pair(unsigned a, unsigned b) {
    unsigned lo = (a & 0x00FF00FFu) + (b & 0x00FF00FFu);
    unsigned hi = ((a >> 8) & 0x00FF00FFu) + ((b >> 8) & 0x00FF00FFu);
    return lo + hi;
}

// Accumulate sum and sum of squares of a packed pair of 10-bit values:
// v^2 = v * lo8(v) + 256 * v * hi8(v), both halves by dp2a.
__device__ __forceinline__ void acc_sq(unsigned p, unsigned &sq_lo, unsigned &sq_hi) {
    unsigned w = __byte_perm(p, 0, 0x3120);  // (v0.lo, v1.lo, v0.hi, v1.hi)
    sq_lo = dp2a_lo(p, w, sq_lo);
    sq_hi = dp2a_hi(p, w, sq_hi);
}

// Morton (Z-order) index of a cell (x, y), x, y < 8: bits of x at even and
// of y at odd positions.  Each 3-bit coordinate is spread by one byte
// permute from the table {0, 1, 4, 5, 16, 17, 20, 21} held in two words.
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y) {
    const uint32_t sx = __byte_perm(0x05040100u, 0x15141110u, x & 7u);
    const uint32_t sy = __byte_perm(0x05040100u, 0x15141110u, y & 7u);
    return sx | (sy << 1);
}

// Record the first device error bit of a stream.
__device__ __forceinline__ void raise_error(uint32_t *info, uint32_t bit) {
    atomicOr(info + FIC_INFO_ERROR, bit);
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}

// Which image of a launch owns global strip `g` (descs sorted by strip_base).
template <class D>
__device__ __forceinline__ int find_image(const D *descs, int count, int g) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (descs[mid].strip_base <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Stage the decimated window of a strip: rows ry0.. of the image, columns
// ax0..ax1 (16-aligned), as packed pairs of 2x2 sums, `upr` 16-pixel units
// per row (at most UPR).  Every lane issues its four loads before using them.
template <int BMAX, int UPR, int NP>
__device__ __forceinline__ void stage_window(const uint8_t *__restrict__ img, int W, int ry0, int ax0, int upr,
                                             uint32_t *d4e, int lane) {
    constexpr int ITER = BMAX * UPR / 32;
    uint4 a[ITER], b[ITER];
#pragma unroll
    for (int t = 0; t < ITER; ++t) {
        const int u = lane + 32 * t;
        const int r = u / UPR, cu = u % UPR;
        if (cu < upr) {
            const uint8_t *p = img + (size_t)(ry0 + 2 * r) * W + ax0 + 16 * cu;
            a[t] = __ldg(reinterpret_cast<const uint4 *>(p));
            b[t] = __ldg(reinterpret_cast<const uint4 *>(p + W));
        }
    }
#pragma unroll
    for (int t = 0; t < ITER; ++t) {
        const int u = lane + 32 * t;
        const int r = u / UPR, cu = u % UPR;
        if (cu < upr) {
            uint4 o;
            o.x = d4_pair(a[t].x, b[t].x);
            o.y = d4_pair(a[t].y, b[t].y);
            o.z = d4_pair(a[t].z, b[t].z);
            o.w = d4_pair(a[t].w, b[t].w);
            *reinterpret_cast<uint4 *>(d4e + r * NP + 4 * cu) = o;
        }
    }
}

// Same, from a window already copied into shared memory (row pitch `pitch`).
template <int BMAX, int UPR, int NP>
__device__ __forceinline__ void stage_window_smem(const uint8_t *raw, int pitch, int upr, uint32_t *d4e, int lane) {
    constexpr int ITER = BMAX * UPR / 32;
#pragma unroll
    for (int t = 0; t < ITER; ++t) {
        const int u = lane + 32 * t;
        const int r = u / UPR, cu = u % UPR;
        if (cu < upr) {
            const uint4 a = *reinterpret_cast<const uint4 *>(raw + (2 * r) * pitch + 16 * cu);
            const uint4 b = *reinterpret_cast<const uint4 *>(raw + (2 * r + 1) * pitch + 16 * cu);
            uint4 o;
            o.x = d4_pair(a.x, b.x);
            o.y = d4_pair(a.y, b.y);
            o.z = d4_pair(a.z, b.z);
            o.w = d4_pair(a.w, b.w);
            *reinterpret_cast<uint4 *>(d4e + r * NP + 4 * cu) = o;
        }
    }
}

constexpr int kImgTable = 1024;  // image strip bases kept in shared memory

template <class Desc>
__device__ __forceinline__ int find_image_s(const int *s_base, const Desc *descs, int count, int g) {
    if (count > kImgTable) return find_image(descs, count, g);
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace fic
