/*
 * fic.h -- C ABI of the GB300 fractal image coder (libfic.so).
 *
 * The library implements the modified no-search (MNS) fractal encoder of
 * Salarian, Mohamadinia and Rasekhi, "A Modified No Search Algorithm for
 * Fractal Image Compression", the comparison modes it is measured against
 * and an iterated fixed-point decoder, as hand-written CUDA kernels for
 * sm_103a.  Every entry point is plain C: device or host pointers and sizes,
 * no framework types.  All GPU work is asynchronous on the cudaStream_t passed
 * as `stream` (NULL = legacy default stream); results are readable after the
 * stream is synchronised.
 *
 * Conventions
 *   image     8-bit greyscale, row-major, pitch = width bytes, on the device.
 *             The device pointer must be 16-byte aligned.
 *   range     B x B block of the image; B runs bmax, bmax/2, ..., bmin over
 *             the quadtree levels 1..L (L <= 4), Section 3 of the paper.
 *   domain    2B x 2B block, decimated 2:1 by the mean of each 2x2 group
 *             (Section 3, "mean filter to four neighbor pixels").
 *   transform rhat = O + s (d - mean d): contrast s coded on 2^s_bits cells of
 *             [-1, 1) (fixed point c = 128 s), luminance O on 2^o_bits levels
 *             of 0..255 (Section 3.3).
 *
 * Errors: every call returns FIC_OK (0) or a negative FIC_E* code.  Argument
 * errors are detected on the host before anything is enqueued.  Errors found
 * on the device (a bounded wait that ran out, a record buffer too small) are
 * written to the stream's info block (FIC_INFO_ERROR) and reported by
 * fic_stream_info().
 */
#ifndef FIC_H
#define FIC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FIC_API __attribute__((visibility("default")))
#else
#define FIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Search modes. */
#define FIC_NOSEARCH 0   /* one centred domain per range, Section 3 */
#define FIC_MNS 1        /* no-search + phase 2 (Technique 1), Sections 3.1-3.2 */
#define FIC_LOCAL 2      /* domains around the centred one, Section 2 */
#define FIC_EXHAUSTIVE 3 /* every domain on a grid, every isometry, Section 1 */

/* Return codes. */
#define FIC_OK 0
#define FIC_EBADSIZE -1   /* width/height not supported for these params */
#define FIC_EBADPARAM -2  /* invalid fic_params or pointer */
#define FIC_ENOMEM -3     /* workspace or buffer too small / allocation failed */
#define FIC_ECAPACITY -4  /* record buffer too small */
#define FIC_ECUDA -5      /* a CUDA call failed */
#define FIC_ETIMEOUT -6   /* a bounded device wait ran out */
#define FIC_EBUDGET -7    /* serving: request can never fit the memory budget */
#define FIC_EBUSY -8      /* serving: queue full / not finished yet */
#define FIC_ECANCELLED -9 /* serving: request cancelled or server stopped */

/* Encoder parameters (one set per image). */
typedef struct fic_params {
    int32_t mode;         /* FIC_NOSEARCH .. FIC_EXHAUSTIVE */
    int32_t bmax, bmin;   /* range sides, powers of two, 4 <= bmin <= bmax <= 32, L <= 4;
                             FIC_NOSEARCH / FIC_MNS also bmin = 2 (bmax 8 or 16: the
                             paper's 16 -> 2 quadtree of Sections 3.3-3.4);
                             FIC_EXHAUSTIVE: a flat partition, bmax = bmin = 8 */
    double thr_rms[4];    /* RMS error threshold E_j per level j=1..4 (Section 3);
                             compared as SSE < round(256 T^2)/256 * n */
    int32_t s_bits;       /* contrast code bits, 1..7 (5: 32 cells) */
    int32_t o_bits;       /* luminance code bits, 1..8 (7: 128 levels) */
    int32_t phase2;       /* MNS only: 1 = try phase 2 before splitting */
    int32_t local_radius; /* FIC_LOCAL: search radius in pixels (16) */
    int32_t local_step;   /* FIC_LOCAL: offset step, even (4) */
    int32_t dom_step;     /* FIC_EXHAUSTIVE: domain grid step in pixels (4) */
    int32_t isometries;   /* FIC_EXHAUSTIVE: the first 1..8 isometries are tried */
    int32_t engine;       /* FIC_EXHAUSTIVE: 0 tensor cores (tcgen05), 1 CUDA cores */
    int32_t phase2_domain; /* MNS phase 2: the domain of each sub-block (the paper does not
                              say): 0 its own centred domain, 1 the matching quadrant of
                              the parent block's centred domain */
} fic_params;

/* One stored transform = one quadtree leaf (16 bytes).
 * phase 1: k = contrast code, q = luminance code.
 * phase 2 (MNS, Section 3.3): the block is coded as four sub-blocks TL, TR,
 *   BL, BR; q = code of the block mean O_i, delta[0..2] = O_k - O_i for the
 *   first three sub-blocks (O_4 follows from eq. (1)), bit b of k = contrast
 *   choice of sub-block b from the level's two-element set (Section 3.2).
 * dx, dy, iso: domain position and isometry (centred domain for
 *   no-search/MNS). */
typedef struct fic_record {
    uint16_t x, y;
    uint8_t level;
    uint8_t phase;
    uint8_t k;
    uint8_t q;
    int8_t delta[3];
    uint8_t iso;
    uint16_t dx, dy;
} fic_record;

/* Info block words (uint32) written by the encoder. */
#define FIC_INFO_RECORDS 0  /* number of records */
#define FIC_INFO_ERROR 1    /* 0 or a positive device error bit set */
#define FIC_INFO_FITS_LO 2  /* range-domain fits evaluated (64-bit, low word) */
#define FIC_INFO_FITS_HI 3
#define FIC_INFO_WORDS 16

/* Device error bits in FIC_INFO_ERROR. */
#define FIC_DEVERR_TIMEOUT 1u
#define FIC_DEVERR_CAPACITY 2u
#define FIC_DEVERR_FORMAT 4u   /* fic_parse: the bitstream does not tile the image */

/* A transform stream in device memory.  The caller allocates every buffer
 * (sizes from fic_stream_sizes) and keeps ownership.
 *   records      capacity entries; leaves in canonical order: top-level
 *                blocks in raster order, inside each the quadtree in
 *                depth-first order TL, TR, BL, BR.
 *   tile_offsets ntop + 1 entries: index of the first record of each
 *                top-level block; the last entry is the record count.
 *   split        ntop entries: bit 0 = the top-level block was split,
 *                bits 1..4 = its children, bits 5..20 = grandchildren
 *                (each group in depth-first order).
 *   info         FIC_INFO_WORDS uint32 (record count, error bits, fits). */
typedef struct fic_stream {
    int32_t width, height;
    fic_params params;
    int32_t ntop;
    int32_t capacity;
    fic_record *records;
    uint32_t *tile_offsets;
    uint32_t *split;
    uint32_t *info;
} fic_stream;

/* Library version (major * 10000 + minor * 100 + patch). */
FIC_API int fic_version(void);

/* Check width/height/params for the GPU encoder.  Returns FIC_OK or the
 * error code the encoder would return.  Requirements: width and height
 * multiples of bmax and of 16, at least 2*bmax, at most 65535. */
FIC_API int fic_validate(int width, int height, const fic_params *p);
/* The checks a stream that already exists must pass to be decoded,
 * serialised or rescaled: the geometry and codebooks of fic_validate without
 * the encoder's mode-specific limits (an exhaustive-search stream rescaled
 * by 2 has 16 x 16 ranges). */
FIC_API int fic_validate_stream(int width, int height, const fic_params *p);

/* Sizes of the buffers of a stream for this image: number of top-level
 * blocks and the largest possible record count (every range at bmin). */
FIC_API int fic_stream_sizes(int width, int height, const fic_params *p, int32_t *ntop,
                     int32_t *max_records);

/* Device workspace (bytes) fic_encode_batch needs for these images (fic_encode
 * is a batch of one).  The workspace holds the image descriptors and the
 * look-back state of the stream packer; it is overwritten by every call. */
FIC_API size_t fic_encode_workspace_bytes(int count, const int *widths, const int *heights,
                                  const fic_params *params);

/* Encode one image (MNS quadtree, Section 3; or the mode in p).
 * d_img: device image; out: stream whose buffers the caller allocated (its
 * width/height/params/ntop/capacity are filled in).  d_workspace: device
 * buffer of at least fic_encode_workspace_bytes(1, ...) bytes.
 * One persistent kernel launch does the whole encode: moments, phase 1,
 * phase 2, split and stream packing of every level. */
FIC_API int fic_encode(const uint8_t *d_img, int width, int height, const fic_params *p, fic_stream *out,
               void *d_workspace, size_t workspace_bytes, void *stream);

/* Encode `count` images of any sizes in one persistent launch.  d_imgs,
 * widths, heights, params, outs are host arrays of `count` entries (params
 * may differ per image but all must share one bmax and one mode family). */
FIC_API int fic_encode_batch(const uint8_t *const *d_imgs, const int *widths, const int *heights,
                     int count, const fic_params *params, fic_stream *outs, void *d_workspace,
                     size_t workspace_bytes, void *stream);

/* Device workspace (bytes) fic_decode_batch needs: one image-sized scratch
 * buffer per image (the Jacobi iterate) plus the descriptor table. */
FIC_API size_t fic_decode_workspace_bytes(int count, const int *widths, const int *heights);

/* Decode a stream: start from mid-grey (128) and apply every transform to
 * the previous iterate `iters` times (Jacobi); the result (uint8, width x
 * height) is written to d_out.  The paper leaves the decoder unspecified
 * beyond its iterated-function-system basis (Section 1). */
FIC_API int fic_decode(const fic_stream *st, int iters, uint8_t *d_out, void *d_workspace,
               size_t workspace_bytes, void *stream);

/* Decode `count` streams, one kernel launch per iteration for all of them. */
FIC_API int fic_decode_batch(const fic_stream *sts, int count, int iters, uint8_t *const *d_outs,
                     void *d_workspace, size_t workspace_bytes, void *stream);

/* Copy a stream's info block to the host (synchronises `stream`) and return
 * FIC_OK, FIC_ETIMEOUT or FIC_ECAPACITY according to its error bits.
 * records/fits may be NULL. */
FIC_API int fic_stream_info(const fic_stream *st, int64_t *records, int64_t *fits, void *stream);

/* ---- Plans: prepare once, launch many times (e.g. inside a CUDA graph) ----
 * A plan uploads the image descriptors of a batch into the caller's
 * workspace (one synchronous-staging host-to-device copy) and records the
 * launch geometry on the host.  fic_*_plan_run only enqueues kernels on
 * `stream`, so it may be captured into a CUDA graph and replayed; the
 * workspace, images and streams named at creation must stay allocated and
 * must not be reused by another plan while the plan is in use. */
typedef struct fic_plan fic_plan;

/* Same arguments as fic_encode_batch; *plan receives a host object that
 * fic_plan_destroy frees. */
FIC_API int fic_encode_plan_create(const uint8_t *const *d_imgs, const int *widths, const int *heights,
                           int count, const fic_params *params, fic_stream *outs, void *d_workspace,
                           size_t workspace_bytes, void *stream, fic_plan **plan);
/* Enqueue the encode of every image of the plan.  No-search, MNS and local
 * search: one persistent encoder kernel over all images and one pack kernel.
 * Exhaustive search: four kernels per image (domain and range preparation,
 * the search, the record writer). */
FIC_API int fic_encode_plan_run(const fic_plan *plan, void *stream);

/* Same arguments as fic_decode_batch, without the iteration count. */
FIC_API int fic_decode_plan_create(const fic_stream *sts, int count, uint8_t *const *d_outs,
                           void *d_workspace, size_t workspace_bytes, void *stream, fic_plan **plan);
/* Enqueue `iters` decoder iterations (one kernel launch each). */
FIC_API int fic_decode_plan_run(const fic_plan *plan, int iters, void *stream);

FIC_API void fic_plan_destroy(fic_plan *plan);

/* Run a plan once (as fic_*_plan_run; `iters` is ignored for encode plans)
 * with a CUDA event after every kernel launch, wait for it and return each
 * kernel's duration in ms[i] (from the previous kernel's end, so the first
 * includes any queueing on `stream`) and its name in labels[i] (static
 * strings; labels may be NULL); *n = number of kernels (at most `cap`;
 * later kernels still run, untimed).  Synchronous; not for graph capture. */
FIC_API int fic_plan_run_timed(const fic_plan *plan, int iters, void *stream, float *ms, const char **labels,
                               int cap, int *n);

/* ---- Launch mapping and its autotuner ----
 * How the batched kernels map onto the GPU; no choice changes any output
 * (strips write their records to fixed slots and are packed afterwards).
 * Applies to no-search / MNS encode plans and to decode plans. */
typedef struct fic_tuning {
    int32_t enc_warps;       /* encoder warps per CTA (one strip per warp at a time): 8 or 4 */
    int32_t enc_ctas_per_sm; /* encoder CTAs per SM; 0 = as many as fit */
    int32_t enc_dynamic;     /* 1: strips taken from an atomic counter; 0: static grid stride */
    int32_t dec_ctas_per_sm; /* decoder iteration kernel CTAs per SM; 0 = as many as fit */
    int32_t enc_fused_pack;  /* 1: the encoder warp that finishes a 32-strip chunk packs it into
                                the stream (no pack launch); 0: a separate pack kernel */
    int32_t dec_single_launch; /* decoders of centred streams (2x2-sum iteration): 1 = every
                                  iteration after the first in one cooperative launch, a grid
                                  barrier between iterations; 0 = one launch per iteration, each
                                  a programmatic dependent of the previous one (default).  A
                                  barrier wait is bounded: if another launch keeps some CTAs
                                  from being resident it gives up and the streams report
                                  FIC_DEVERR_TIMEOUT -- keep 0 for decodes that share the GPU
                                  with concurrent kernels. */
} fic_tuning;

FIC_API int fic_plan_get_tuning(const fic_plan *plan, fic_tuning *t);
/* FIC_EBADPARAM for values outside the ranges above. */
FIC_API int fic_plan_set_tuning(fic_plan *plan, const fic_tuning *t);
/* Time every candidate mapping on the plan's own batch and keep the fastest.
 * Encode plans try warps {8, 4} x CTAs per SM {1, 2, ..., max} x schedule
 * {static, dynamic} x packing {fused, separate}; decode plans try CTAs per SM {1, 2, 3, 4} x
 * {single launch, one launch per iteration} with `iters` iterations.  Each candidate runs once untimed, then `reps` times between
 * CUDA events on `stream`; the score is the median.  Synchronous: returns
 * after the last run with the plan's outputs written (identical for every
 * candidate).  *best and *best_ms (either may be NULL) receive the choice
 * and its median time; `trace` (may be NULL) receives up to `trace_cap`
 * (candidate, ms) rows as 7 floats each: enc_warps, enc_ctas_per_sm,
 * enc_dynamic, dec_ctas_per_sm, enc_fused_pack, dec_single_launch, ms, and
 * *ntrace their number.
 * Other encode families return FIC_EBADPARAM. */
FIC_API int fic_plan_autotune(fic_plan *plan, int iters, int reps, void *stream, fic_tuning *best,
                              float *best_ms, float *trace, int trace_cap, int *ntrace);

/* ---- Allocation-free encode ----
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory -- code inside a host application that owns
 * the whole device heap and offers no allocator, or code on a latency-
 * critical path where a device allocation (which may synchronise the
 * device) is not allowed.  It encodes one image exactly like fic_encode,
 * but keeps the encoder's scratch (image descriptor, look-back status of the
 * stream packer, ticket) in a static device array of the library instead of
 * a caller workspace; the caller still passes the image and the stream's
 * buffers.  It calls no cudaMalloc/cudaFree.
 *   - Limit: at most FIC_NOALLOC_MAX_STRIPS strips of 1024 pixels, i.e. 64 Mi
 *     pixels (e.g. 8192 x 8192); larger images return FIC_EBADSIZE.
 *   - Every GPU that loads the library holds the array (about 256 KiB) until
 *     the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, once per device, with that device current).
 *   - It must not be called while `stream` is being captured into a CUDA
 *     graph: it stages the image descriptor and tensor map from its own host
 *     memory with cudaMemcpyAsync, which a graph could not replay, so it
 *     returns FIC_EBADPARAM before enqueuing anything.  These copies are from
 *     pageable memory, so the call may wait for them on the host.
 *   - Modes FIC_NOSEARCH and FIC_MNS with bmin >= 4 only (FIC_EBADPARAM
 *     otherwise).
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (e.g. on two streams without ordering) race and corrupt each other's
 *     streams.  Each call clears the parts that must start at zero.  */
#define FIC_NOALLOC_MAX_STRIPS 65536
FIC_API int fic_encode_noalloc(const uint8_t *d_img, int width, int height, const fic_params *p,
                               fic_stream *out, void *stream);

/* ---- Records to host memory ----
 * Copy each stream's records -- as many as its info block counts, at most
 * its capacity -- and, when h_info is not NULL, its info block
 * (FIC_INFO_WORDS words) to host memory, without a round trip to the host:
 * the count is read on the device, so only the records the stream holds
 * cross the bus (a plain device-to-host copy would have to move the whole
 * capacity, or wait for the count).  h_records[i] (16-byte aligned, room
 * for stream i's capacity) and h_info[i] must be host memory the device
 * can address: page-locked (cudaHostAlloc / cudaMallocHost, or
 * cudaHostRegister), or any host memory where the device reads the host's
 * page tables (a coherent CPU-GPU link); other pointers, and misaligned
 * ones, give FIC_EBADPARAM before anything is enqueued.  One kernel launch per 64 streams, asynchronous on `stream`:
 * the host may read the buffers once the stream has passed this point. */
FIC_API int fic_records_to_host(const fic_stream *sts, int count, fic_record *const *h_records,
                                uint32_t *const *h_info, void *stream);

/* ---- Bitstream of the stored parameters (Sections 3.3 and 3.4) ----
 * Layout: bits appended least-significant first into uint32 words; leaves
 * in the stream's canonical order; per leaf: level - 1 in ceil(log2 L)
 * bits (with technique2 != 0, omitted for a last-level leaf that is not the
 * top-left of its group of four: Technique 2, Section 3.4); 1 phase bit at
 * levels < L when MNS phase 2 is on; phase 1: k (s_bits), q (o_bits), and
 * for local search the offset index ((oy/step + R/step) * per + ox/step +
 * R/step, per = 2R/step + 1) in ceil(log2 per^2) bits, for exhaustive search
 * the domain's raster index on the step grid (ceil(log2 #domains) bits) and
 * the isometry (ceil(log2 isometries) bits); phase 2: q_i (o_bits), the
 * three differences O_k - O_i (M bits two's complement, M = 5 at level 1,
 * 6 below, Section 3.3), the four contrast bits.  Positions and centred
 * domains are implied by the order.  tile_bits[t] (uint64, ntop + 1 entries)
 * is the first bit of top-level block t and tile_bits[ntop] the total: an
 * index that lets every block be read independently.  The paper fixes the
 * fields and widths; their order is this library's.  Device pointers,
 * asynchronous on `stream`; the workspace holds the scans. */
FIC_API int64_t fic_bitstream_max_words(int width, int height, const fic_params *p);
FIC_API size_t fic_bitstream_workspace_bytes(int width, int height, const fic_params *p);
/* Write the bitstream of `st` (records, tile offsets and record count as an
 * encode left them) into d_words (at least fic_bitstream_max_words words;
 * zeroed first) and its index into d_tile_bits. */
FIC_API int fic_serialize(const fic_stream *st, int technique2, uint32_t *d_words, int64_t nwords,
                          uint64_t *d_tile_bits, void *d_workspace, size_t workspace_bytes, void *stream);
/* Read a bitstream back into `out` (width, height and params set by the
 * caller, buffers from fic_stream_sizes): records, tile offsets, split masks
 * and the record count (fits 0).  A stream that does not tile the image
 * sets FIC_DEVERR_FORMAT in out->info (fic_stream_info returns FIC_EBADPARAM
 * for it). */
FIC_API int fic_parse(const uint32_t *d_words, int64_t nwords, const uint64_t *d_tile_bits, int technique2,
                      fic_stream *out, void *d_workspace, size_t workspace_bytes, void *stream);
/* The same for `count` streams at once (Sections 3.3-3.4): three kernel
 * launches for every 48 streams instead of three per stream.  Stream i uses
 * d_words[i] (nwords[i] words, at least fic_bitstream_max_words; zeroed by
 * the writer) and d_tile_bits[i]; one workspace of
 * fic_bitstream_batch_workspace_bytes holds every stream's scans.  Results
 * are those of fic_serialize / fic_parse on each stream.  Errors as there;
 * the first bad argument of any stream fails the whole call before anything
 * is enqueued for the streams after it. */
FIC_API size_t fic_bitstream_batch_workspace_bytes(const fic_stream *sts, int count);
FIC_API int fic_serialize_batch(const fic_stream *sts, int count, int technique2, uint32_t *const *d_words,
                                const int64_t *nwords, uint64_t *const *d_tile_bits, void *d_workspace,
                                size_t workspace_bytes, void *stream);
FIC_API int fic_parse_batch(const uint32_t *const *d_words, const int64_t *nwords, const uint64_t *const *d_tile_bits,
                            int technique2, fic_stream *outs, int count, void *d_workspace, size_t workspace_bytes,
                            void *stream);

/* ---- Resolution-independent decoding (Section 1) ----
 * The stored transforms describe the image at no particular resolution.
 * fic_rescale_params gives the geometry of a stream rescaled by 2^shift
 * (shift +1: twice the resolution, -1: half): sides, block sides, local
 * search radius/step and domain step times 2^shift.  FIC_EBADPARAM when a
 * rescaled quantity is not an integer or leaves fic_validate_stream's
 * limits.  fic_stream_rescale writes the rescaled records (positions and
 * domains times 2^shift, codes unchanged), tile offsets, split masks and
 * info into `out`, whose width/height/params must be the rescaled ones and
 * whose buffers come from fic_stream_sizes; decoding `out` renders the
 * attractor on the rescaled grid.  Asynchronous on `stream`. */
FIC_API int fic_rescale_params(int width, int height, const fic_params *p, int shift, int *width_out,
                               int *height_out, fic_params *p_out);
FIC_API int fic_stream_rescale(const fic_stream *in, int shift, fic_stream *out, void *stream);

/* ---- Self-test of the bounded device waits ----
 * Every wait in the library's kernels (look-back spins, mbarrier waits for
 * TMA and tensor-core completions) gives up after an iteration limit and
 * reports FIC_DEVERR_TIMEOUT instead of hanging.  This runs the same two
 * helpers on a word that nothing writes (d_never: device memory holding 0)
 * and on an mbarrier whose announced transfer never comes; d_out (3 uint32)
 * receives 1, 1 when both gave up, and the spin's iteration count.  Takes
 * about a second; the context stays usable. */
FIC_API int fic_selftest_waits(const uint32_t *d_never, uint32_t *d_out, void *stream);

/* ---- Position statistics (Section 2, Figs. 2 and 3) ----
 * Histograms of x_d - x_r and y_d - y_r over the stream's records: the
 * offset between each range block and its domain block.  hx has 2*width
 * bins (bin (x_d - x_r) + width), hy 2*height bins (bin (y_d - y_r) +
 * height), uint32 device arrays; counts are ADDED (zero them first).  The
 * record count is read on the device from the stream's info block.  For
 * no-search / MNS streams the domain is the centred one (phase-2 records:
 * the block's).  Asynchronous on `stream`; FIC_EBADPARAM for null pointers. */
FIC_API int fic_offset_histogram(const fic_stream *st, uint32_t *d_hx, uint32_t *d_hy, void *stream);

/* ---- Serving: continuous batching of encode and decode requests ----
 * The paper has a single encoder; the server runs many of them at once on
 * one GPU.  It owns one device allocation of `hbm_budget_bytes` (sub-
 * allocated per job: image, stream buffers, workspace) and a pinned host
 * staging area.  fic_submit queues a job and returns at once; a worker
 * thread admits queued jobs in arrival order as soon as their memory fits
 * in the budget, forms batches of the admitted jobs (encode jobs sharing
 * bmax and search family go into one persistent launch, decode jobs into
 * one decode launch), and runs batches on `streams` CUDA streams so that
 * work of different batches overlaps on the device.  Jobs that arrive while
 * others run are admitted as memory frees.  A job whose footprint exceeds
 * the whole budget is rejected at submit with FIC_EBUDGET. */
#define FIC_JOB_ENCODE 0
#define FIC_JOB_DECODE 1

typedef struct fic_server fic_server;

typedef struct fic_server_config {
    int32_t device;           /* CUDA device ordinal */
    int32_t streams;          /* concurrent CUDA streams, >= 1 */
    int32_t max_batch;        /* jobs per batched launch, >= 1 */
    int32_t queue_capacity;   /* queued + running jobs; fic_submit returns FIC_EBUSY beyond */
    int64_t hbm_budget_bytes; /* device memory of the server (one allocation at creation) */
    int64_t host_staging_bytes; /* pinned host memory for inputs/outputs (one allocation) */
} fic_server_config;

/* A job.  Host buffers stay owned by the caller and must stay valid until
 * the job completes.  encode: image (width x height, uint8, pitch width) in,
 * out_records (capacity (width/bmin)*(height/bmin)) and optionally out_split
 * ((width/bmax)*(height/bmax)) out.  decode: records (canonical order,
 * nrecords, as an encode produced them) in, out_image (width x height) out,
 * `iters` decoder iterations. */
typedef struct fic_job {
    int32_t kind;
    int32_t width, height;
    fic_params params;
    int32_t iters;
    int32_t nrecords;
    const uint8_t *image;
    const fic_record *records;
    uint8_t *out_image;
    fic_record *out_records;
    uint32_t *out_split;
} fic_job;

typedef struct fic_job_result {
    int32_t status;     /* FIC_OK or an error code */
    int32_t nrecords;   /* encode: records written */
    int64_t fits;       /* encode: range-domain fits */
    double latency_ms;  /* submit -> completion */
    double queue_ms;    /* submit -> launch */
} fic_job_result;

typedef struct fic_server_stats {
    int64_t submitted, completed, rejected, batches;
    int64_t peak_device_bytes;
    double p50_ms, p99_ms, mean_ms, max_ms; /* latency of completed jobs */
    double mean_batch;                      /* jobs per batch */
} fic_server_stats;

FIC_API int fic_server_create(const fic_server_config *cfg, fic_server **out);
/* Queue a job; *ticket identifies it.  Never blocks on the GPU. */
FIC_API int fic_submit(fic_server *srv, const fic_job *job, int64_t *ticket);
/* FIC_EBUSY while the job is queued or running; otherwise the job's
 * status, with *res filled (the ticket is then released). */
FIC_API int fic_poll(fic_server *srv, int64_t ticket, fic_job_result *res);
/* Wait up to timeout_ms (< 0: no limit) for the job; FIC_ETIMEOUT if not done. */
FIC_API int fic_wait(fic_server *srv, int64_t ticket, int32_t timeout_ms, fic_job_result *res);
FIC_API int fic_server_get_stats(fic_server *srv, fic_server_stats *st);
/* Finish every accepted job, stop the worker and free the server. */
FIC_API int fic_server_destroy(fic_server *srv);

/* Human-readable name of a return code. */
FIC_API const char *fic_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* FIC_H */
