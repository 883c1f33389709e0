// exhaustive_tc.cu -- the exhaustive search on the 5th-generation tensor
// cores (tcgen05), with the screening epilogue fused.
//
// The contraction yields each candidate's screen value directly:
// Y[row, d] = sum_k A[row, k] W[d, k], A = range rows (range x isometry) with
// the range's mean removed, a_k = r_k - Sr / 64, W = the domain's screen
// operand w_k = (64 d4_k - Sd) 1024 / sqrt(nCdd), both rounded to fp16.  With
// x_k = 64 d4_k - Sd, sum_k x_k = 0 and sum_k x_k^2 = 64 nCdd, so exactly
// sum_k a_k w_k = sum_k r_k w_k = 1024 nCdr / sqrt(nCdd) = +-2 sqrt(L), L the
// largest improvement any contrast could give (exhaustive.cuh).  The error
// is bounded per row, independently of the domain: by Cauchy-Schwarz
// sum_k |a_k w_k| <= sqrt(nCrr / 64) 8192 = 1024 sqrt(nCrr); the two fp16
// roundings (2^-11 relative each) move Y by at most sqrt(nCrr), the fp32
// accumulation of 64 products by 0.03 sqrt(nCrr) (one unit in the last
// place per addition, taken four times over), and operand values too small
// to be normal fp16 by at most 1: |Y - 2 sqrt(L)| <= E_row = 1.1 sqrt(nCrr)
// + 4.  A candidate can beat the row's best exact error g only if sqrt(L) >=
// sqrt(-g), i.e. only if |Y| >= 2 sqrt(-g) - E_row; the epilogue screens a
// batch of 32 candidates with one maximum of |Y| per candidate.  While many
// of a batch's rows still pass (their thresholds are young: the first tiles
// of a sweep), each such lane first settles its batch's best-screened
// candidate at once, which raises its threshold before the rest of the
// batch is screened again.  Candidates that pass go to a per-warp queue; 32
// at a time, one per lane, they are settled exactly: sum r*d4 by dp2a from byte range rows and packed domain
// pairs, then the int64 contrast search, and each row's owner lane takes the
// best of its entries (the smaller domain index wins ties, so the order of
// evaluation does not change the result).
//
// One CTA owns 128 rows (16 ranges x 8 isometries) and streams every domain
// tile of 128 domains:
//   warp 0      TMA producer: the A tile once, W tiles through a 4-stage ring
//               (128-byte swizzle, mbarrier transaction counts);
//   warp 1      allocates 256 TMEM columns (two 128-column fp32
//               accumulators) and issues tcgen05.mma (M=128, N=128, K=16,
//               four per tile) from one lane, committing to mbarriers;
//   warps 2..9  epilogue: each warp reads one 32-lane quarter of an
//               accumulator (tcgen05.ld, 32x32b) for half of the columns.
// The accumulators alternate, so the epilogue of tile n overlaps the MMA of
// tile n+1.  Every mbarrier wait is bounded; a timeout sets an error flag,
// all roles leave their loops, and TMEM is freed before the CTA exits.
#include <cudaTypedefs.h>

#include "exhaustive.cuh"

namespace fic {

constexpr int kTcRows = 128;   // M
constexpr int kTcCols = 128;   // N per tile
constexpr int kTcStages = 4;
constexpr int kTcEpiWarps = 8;
constexpr int kTcThreads = (2 + kTcEpiWarps) * 32;
constexpr uint32_t kTileBytes = kTcCols * kExhK * 2;  // 16 KiB (also the A tile)
// a batch with this many passing rows settles their best candidates first
// (1, 2, 4, 8, 16 rows measured 2.08, 2.02, 2.10, 2.18, 2.27 ms at 1024 x 1024)
constexpr int kTcEagerRows = 2;

// Bounded wait whose polls each block in hardware for up to 1 us (a poll
// returns as soon as the phase completes), so that a waiting warp issues few
// instructions and leaves the issue slots to the working warps (measured:
// 1.995 -> 1.942 ms for the 1024 x 1024 search).  At most `limit` polls:
// about a second for kMbarLimit, then false.
__device__ __forceinline__ bool mbar_wait_hint(uint64_t *bar, uint32_t parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// K-major operand in shared memory with the 128-byte swizzle: rows of 128
// bytes (64 fp16), 8-row groups 1024 bytes apart.  Fields: start address
// >> 4 (bits 0-13), leading byte offset >> 4 (16-29, unused here: 1), stride
// byte offset >> 4 (32-45), descriptor version 1 (46-47), swizzle mode 2 =
// 128-byte (61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1),
// fp16 A and B (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Order in which a CTA visits its ntiles domain tiles: tile i, i + step,
// i + 2 step, ... (mod ntiles), with step near ntiles / phi and coprime with
// ntiles (a bijection).  The first tiles then sample the whole domain pool,
// so the rows' thresholds approach their final values early and fewer
// candidates pass the screen; the result does not depend on the order.
__device__ __forceinline__ int tc_tile_step(int ntiles) {
    int step = max(1, (int)(0.618034f * (float)ntiles));
    for (;; ++step) {
        int a = step, b = ntiles;
        while (b) {
            const int t = a % b;
            a = b;
            b = t;
        }
        if (a == 1) return step;
    }
}

// Largest of three floats (three-input max of sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Row state of the screening epilogue.
struct TcRow {
    long long g;  // best exact s-part error
    float thr;    // threshold on |Y| (tc_threshold)
    int d, k;
};

// Screen threshold of a row with best exact error g: exh_threshold(g) is a
// lower bound of sqrt(-g) (or -1 while g >= 0, when everything passes), and
// |Y| + E_row >= 2 sqrt(L) for every candidate.
__device__ __forceinline__ float tc_threshold(long long g, float er) {
    const float t = exh_threshold(g);
    return t > 0.f ? fmaf(2.f, t, -er) * (1.f - 1e-6f) - 1.f : -1.f;
}

// Exact sum r*d4 of one range row (64 bytes) and one domain (32 packed
// pairs), in four independent dp2a chains.
__device__ __forceinline__ int tc_sdr(const uint8_t *rb, const uint32_t *dp) {
    const uint4 *a4 = reinterpret_cast<const uint4 *>(rb);
    const uint4 *p4 = reinterpret_cast<const uint4 *>(dp);
    uint4 a[4], p[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = __ldg(a4 + i);  // range values 16i .. 16i+15
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = __ldg(p4 + i);
    unsigned acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        acc[i] = dp2a_lo(p[2 * i].x, a[i].x, acc[i]);
        acc[i] = dp2a_hi(p[2 * i].y, a[i].x, acc[i]);
        acc[i] = dp2a_lo(p[2 * i].z, a[i].y, acc[i]);
        acc[i] = dp2a_hi(p[2 * i].w, a[i].y, acc[i]);
        acc[i] = dp2a_lo(p[2 * i + 1].x, a[i].z, acc[i]);
        acc[i] = dp2a_hi(p[2 * i + 1].y, a[i].z, acc[i]);
        acc[i] = dp2a_lo(p[2 * i + 1].z, a[i].w, acc[i]);
        acc[i] = dp2a_hi(p[2 * i + 1].w, a[i].w, acc[i]);
    }
    return (int)(acc[0] + acc[1] + acc[2] + acc[3]);
}

// Best contrast code of a candidate and its exact s-part error.
__device__ __forceinline__ long long tc_eval(int sdr, int sr, int4 ds, int s_bits, int &k) {
    const int ncdr = 64 * sdr - ds.x * sr;
    const uint32_t ncdd = (uint32_t)ds.y;
    k = best_contrast<true>((long long)ncdr, (long long)ncdd, s_bits);
    const long long c = contrast_code(k, s_bits);
    return c * c * (long long)ncdd - 1024LL * c * ncdr;
}

__device__ __forceinline__ void tc_offer(TcRow &b, long long g, int d, int k, float er) {
    if (exh_better(g, d, b.g, b.d)) {
        b.g = g;
        b.thr = tc_threshold(g, er);
        b.d = d;
        b.k = k;
    }
}

// Settles entries 0 .. cnt-1 (cnt <= 32) of the warp's queue: lane i
// evaluates entry i (owner lane, domain) exactly; the entries that beat
// their owner's best as it stood (usually none) are then offered to their
// owners one at a time.  Called by the whole warp.
__device__ __forceinline__ void tc_flush(const ExhDesc &E, const uint2 *q, int cnt, int row_base, int sr, float er,
                                         TcRow &best, int lane) {
    const unsigned FULL = 0xffffffffu;
    const uint2 e = lane < cnt ? q[lane] : make_uint2(0u, 0u);
    const int o = (int)e.x, d = (int)e.y;
    const int sro = __shfl_sync(FULL, sr, o);
    const long long og = __shfl_sync(FULL, best.g, o);
    const int od = __shfl_sync(FULL, best.d, o);
    long long g = 0;
    int k = 0;
    bool cand = false;
    if (lane < cnt) {
        g = tc_eval(tc_sdr(E.rbytes + (size_t)(row_base + o) * kExhK, E.dpairs + (size_t)d * 32), sro,
                    __ldg(E.dstat + d), E.s_bits, k);
        cand = exh_better(g, d, og, od);
    }
    unsigned bal = __ballot_sync(FULL, cand);
    while (bal) {
        const int i = __ffs(bal) - 1;
        bal &= bal - 1u;
        const int oi = __shfl_sync(FULL, o, i), di = __shfl_sync(FULL, d, i), ki = __shfl_sync(FULL, k, i);
        const long long gi = __shfl_sync(FULL, g, i);
        if (lane == oi) tc_offer(best, gi, di, ki, er);
    }
}

// Settles the first 32 queued entries and moves the rest (at most 96) down.
__device__ __forceinline__ void tc_flush32(const ExhDesc &E, uint2 *q, int &qn, int row_base, int sr, float er,
                                           TcRow &best, int lane) {
    __syncwarp();
    tc_flush(E, q, 32, row_base, sr, er, best, lane);
    const int rest = qn - 32;
    uint2 mv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) mv[i] = 32 * i + lane < rest ? q[32 + 32 * i + lane] : make_uint2(0u, 0u);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (32 * i + lane < rest) q[32 * i + lane] = mv[i];
    __syncwarp();
    qn = rest;
}

__global__ void __launch_bounds__(kTcThreads, 2)
    exh_tc_kernel(ExhDesc E, const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  uint32_t *err) {
    extern __shared__ __align__(1024) uint8_t tsmem[];
    uint8_t *base = tsmem + ((1024u - (smem_u32(tsmem) & 1023u)) & 1023u);
    uint8_t *sA = base;
    uint8_t *sB = base + kTileBytes;
    __shared__ __align__(8) uint64_t bar_full[kTcStages], bar_empty[kTcStages], bar_acc_full[2], bar_acc_empty[2],
        bar_a;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ TcRow s_half[kTcRows];  // the second epilogue warp of each lane quarter hands its state over
    __shared__ uint2 s_q[kTcEpiWarps][128];  // per epilogue warp: candidates to settle (owner lane, domain)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * kTcRows;
    // this CTA's domain segment: tiles [t0, t0 + cnt)
    const int ntiles_all = E.nd_pad / kTcCols;
    const int t0 = (int)(((long long)blockIdx.y * ntiles_all) / gridDim.y);
    const int ntiles = (int)(((long long)(blockIdx.y + 1) * ntiles_all) / gridDim.y) - t0;
    const int tstep = ntiles > 0 ? tc_tile_step(ntiles) : 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&bar_acc_full[a], 1);
            mbar_init(&bar_acc_empty[a], kTcEpiWarps * 32);  // every epilogue thread reads every accumulator
        }
        mbar_init(&bar_a, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            mbar_arrive_expect_tx(&bar_a, kTileBytes);
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(smem_u32(sA)),
                "l"(reinterpret_cast<uint64_t>(&mapA)), "r"(0), "r"(row0), "r"(smem_u32(&bar_a))
                : "memory");
            int issued = 0, tix = 0;
            for (int n = 0; n < ntiles; ++n) {
                const int s = n % kTcStages;
                const uint32_t par = (uint32_t)((n / kTcStages) & 1) ^ 1u;
                if (!mbar_wait_hint(&bar_empty[s], par, kMbarLimit) || s_abort) {
                    s_abort = 1;
                    break;
                }
                issued = n + 1;
                mbar_arrive_expect_tx(&bar_full[s], kTileBytes);
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                    "%3}], [%4];" ::"r"(smem_u32(sB + s * kTileBytes)),
                    "l"(reinterpret_cast<uint64_t>(&mapB)), "r"(0), "r"((t0 + tix) * kTcCols), "r"(smem_u32(&bar_full[s]))
                    : "memory");
                tix += tstep;
                if (tix >= ntiles) tix -= ntiles;
            }
            // copies still in flight must land before the CTA may leave
            mbar_wait(&bar_a, 0u, kMbarLimit);
            for (int n = max(0, issued - kTcStages); n < issued; ++n)
                mbar_wait(&bar_full[n % kTcStages], (uint32_t)((n / kTcStages) & 1), kMbarLimit);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = f16_idesc(kTcRows, kTcCols);
            bool ok = mbar_wait(&bar_a, 0u, kMbarLimit);
            int last = -1;
            for (int n = 0; ok && n < ntiles; ++n) {
                const int s = n % kTcStages, acc = n & 1;
                if (!mbar_wait_hint(&bar_full[s], (uint32_t)((n / kTcStages) & 1), kMbarLimit) ||
                    !mbar_wait_hint(&bar_acc_empty[acc], (uint32_t)((n >> 1) & 1) ^ 1u, kMbarLimit) || s_abort) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * kTcCols);
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + s * kTileBytes);
#pragma unroll
                for (int kk = 0; kk < kExhK / 16; ++kk)
                    tc_mma(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, kk > 0);
                tc_commit(&bar_empty[s]);     // the B stage is free once these MMAs are done
                tc_commit(&bar_acc_full[acc]);
                last = n;
            }
            if (!ok) s_abort = 1;
            // every MMA issued must be complete before TMEM is freed
            if (last >= 0) mbar_wait(&bar_acc_full[last & 1], (uint32_t)((last >> 1) & 1), kMbarLimit);
        }
    } else {
        // ---------------- epilogue: warps 2..9; lane quarter q, column half h
        const int ew = warp - 2;
        const int q = warp & 3;              // TMEM lanes 32q .. 32q+31 belong to warps with warp % 4 == q
        const int h = ew >> 2;               // 0: columns 0..63, 1: columns 64..127
        const int rloc = 32 * q + lane;
        const int row = row0 + rloc;
        const int r = row >> 3, t = row & 7;
        const bool live = r < E.nr && t < E.isos;
        const int sr = live ? E.rstat[r].x : 0;
        // nCrr = 64 Srr - Sr^2 (exact in int64, then below 2^28)
        const float er = live ? fmaf(1.1f, sqrtf((float)(64LL * E.rstat[r].y - (long long)sr * sr)), 4.f) : 0.f;
        const int row_base = row0 + 32 * q;  // the warp's rows: lane i owns row_base + i
        TcRow best;
        best.g = 0x7fffffffffffffffLL;
        best.thr = live ? -1.f : __int_as_float(0x7f800000);  // everything passes / dead rows never pass
        best.d = -1;
        best.k = 0;
        if (live) {
            // seed with the grid domain nearest the range's centred domain: a
            // good candidate from the start raises the screen's threshold at
            // once (ties still go to the smaller domain index, so the result
            // does not depend on the seed)
            const int rx = (r % E.nrx) * kExhB, ry = (r / E.nrx) * kExhB;
            const int cx = clampi(rx - kExhB / 2, 0, E.W - 2 * kExhB), cy = clampi(ry - kExhB / 2, 0, E.H - 2 * kExhB);
            const int ix = min((cx + E.step / 2) / E.step, E.ndx - 1), iy = min((cy + E.step / 2) / E.step, E.ndy - 1);
            const int d0 = iy * E.ndx + ix;
            int k0;
            const long long g0 =
                tc_eval(tc_sdr(E.rbytes + (size_t)row * kExhK, E.dpairs + (size_t)d0 * 32), sr, __ldg(E.dstat + d0),
                        E.s_bits, k0);
            tc_offer(best, g0, d0, k0, er);
        }
        uint2 *qw = s_q[ew];
        int qn = 0;  // queued entries (warp-uniform)
        const unsigned lt = (1u << lane) - 1u;
        bool bad = false;
        for (int n = 0, tix = 0; n < ntiles; ++n, tix = tix + tstep >= ntiles ? tix + tstep - ntiles : tix + tstep) {
            const int acc = n & 1;
            const bool got = mbar_wait_hint(&bar_acc_full[acc], (uint32_t)((n >> 1) & 1), kMbarLimit);
            if (!__all_sync(0xffffffffu, got) || s_abort) {
                bad = true;
                break;
            }
            tc_fence_after();
#pragma unroll 1
            for (int c0 = 0; c0 < kTcCols / 2; c0 += 32) {
                const int col = h * (kTcCols / 2) + c0;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kTcCols + col), v);
                const int dbase = (t0 + tix) * kTcCols + col;
                // the batch's largest |Y| (32 independent maxima); the
                // threshold only rises as the row's best improves, so a batch
                // whose largest value is below it holds nothing to settle
                float mp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 32; j += 8)
#pragma unroll
                    for (int i = 0; i < 4; ++i) mp[i] = fmax3(mp[i], fabsf(v[j + 2 * i]), fabsf(v[j + 2 * i + 1]));
                const float m = fmax3(mp[0], mp[1], fmaxf(mp[2], mp[3]));
                const unsigned rows = __ballot_sync(0xffffffffu, m >= best.thr);
                if (rows) {
                    const int nvalid = E.nd - dbase;  // padding domains are never settled
                    unsigned done = 0;
                    if (__popc(rows) >= kTcEagerRows) {
                        // many rows still pass (their thresholds are young): each
                        // lane settles its batch's best-screened candidate at once,
                        // in parallel, which raises its threshold before the rest
                        // of the batch is screened again
                        int jm = 0;
#pragma unroll
                        for (int j = 31; j >= 0; --j) jm = fabsf(v[j]) == m ? j : jm;
                        if (m >= best.thr && jm < nvalid) {
                            int k;
                            const long long g = tc_eval(tc_sdr(E.rbytes + (size_t)(row_base + lane) * kExhK,
                                                               E.dpairs + (size_t)(dbase + jm) * 32),
                                                        sr, __ldg(E.dstat + dbase + jm), E.s_bits, k);
                            tc_offer(best, g, dbase + jm, k, er);
                            done = 1u << jm;
                        }
                    }
                    unsigned pm = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) pm |= (fabsf(v[j]) >= best.thr ? 1u : 0u) << j;
                    pm &= ~done;
                    if (nvalid < 32) pm &= nvalid > 0 ? (1u << nvalid) - 1u : 0u;
                    unsigned cols = __reduce_or_sync(0xffffffffu, pm);
                    while (cols) {
                        const int j = __ffs(cols) - 1;
                        cols &= cols - 1u;
                        const bool p = (pm >> j) & 1u;
                        const unsigned bal = __ballot_sync(0xffffffffu, p);
                        if (p) qw[qn + __popc(bal & lt)] = make_uint2((uint32_t)lane, (uint32_t)(dbase + j));
                        qn += __popc(bal);
                        // settling waits until the accumulator is released,
                        // unless the queue could overflow
                        if (qn > 96) tc_flush32(E, qw, qn, row_base, sr, er, best, lane);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&bar_acc_empty[acc]);
            while (qn >= 32) tc_flush32(E, qw, qn, row_base, sr, er, best, lane);
        }
        if (!bad && qn > 0) {
            __syncwarp();
            tc_flush(E, qw, qn, row_base, sr, er, best, lane);
        }
        if (bad) s_abort = 1;
        // merge the two column halves of each row (the lower domain half wins ties)
        if (h == 1) s_half[rloc] = best;
        asm volatile("bar.sync 1, %0;" ::"r"(kTcEpiWarps * 32));
        if (h == 0 && live) {
            const TcRow o = s_half[rloc];
            if (exh_better(o.g, o.d, best.g, best.d)) best = o;
            const size_t i = (size_t)blockIdx.y * E.nr * 8 + (size_t)r * 8 + t;
            E.row_g[i] = best.g;
            E.row_dk[i] = make_int2(best.d, best.k);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
    if (threadIdx.x == 0 && s_abort) atomicOr(err, FIC_DEVERR_TIMEOUT);
}

// Tensor maps of the two operands (fp16, 128-byte swizzle, 64 x 128 boxes).
static int make_f16_map(CUtensorMap *m, const void *base, int rows) {
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!encode) return -1;
    const cuuint64_t dims[2] = {(cuuint64_t)kExhK, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kExhK * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kExhK, (cuuint32_t)kTcRows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
               ? 0
               : -1;
}

size_t exh_tc_smem_bytes() { return (size_t)(1 + kTcStages) * kTileBytes + 1024; }

// The domain axis is split into up to kExhMaxSeg segments (one CTA per row
// tile and segment) so that small images still give every SM several CTAs;
// *nseg receives the count for exh_finalize.
cudaError_t launch_exh_tc(const ExhDesc &E, uint32_t *err, int *nseg, cudaStream_t st) {
    static KernelSlots ks;
    const size_t smem = exh_tc_smem_bytes();
    int sms = 0, per = 0;
    cudaError_t e = kernel_slots(ks, (const void *)exh_tc_kernel, kTcThreads, smem, sms, per);
    if (e != cudaSuccess) return e;
    const int slots = sms * per;
    CUtensorMap ma, mb;
    // rows past the end of A read as zeros (TMA out-of-bounds fill)
    if (make_f16_map(&ma, E.afp16, E.nr * 8) || make_f16_map(&mb, E.dsc, E.nd_pad)) return cudaErrorInvalidValue;
    const int ctas = (E.nr * 8 + kTcRows - 1) / kTcRows;
    const int ntiles = E.nd_pad / kTcCols;
    int seg = (4 * slots + ctas - 1) / ctas;  // about four waves of CTAs
    seg = seg < 1 ? 1 : (seg > kExhMaxSeg ? kExhMaxSeg : seg);
    seg = seg > ntiles ? ntiles : seg;
    *nseg = seg;
    exh_tc_kernel<<<dim3(ctas, seg), kTcThreads, smem, st>>>(E, ma, mb, err);
    stage_mark(st, "exh_tc_kernel");
    return cudaGetLastError();
}

}  // namespace fic
