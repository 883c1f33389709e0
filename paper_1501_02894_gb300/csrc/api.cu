// api.cu -- the C ABI of libfic.so: argument checks, descriptor tables,
// workspace layout and kernel launches.  No allocation happens here: every
// device buffer (streams, outputs, workspace) belongs to the caller.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "exhaustive.cuh"
#include "trace.cuh"

namespace fic {
cudaError_t launch_exhaustive(const ExhDesc &E, int engine, cudaStream_t st);

// Event recorder of fic_plan_run_timed (active on one thread at a time).
struct StageMarks {
    std::vector<cudaEvent_t> ev;
    std::vector<const char *> label;
    size_t used = 0;
};
thread_local StageMarks *t_marks = nullptr;

void stage_mark(cudaStream_t st, const char *label) {
    StageMarks *m = t_marks;
    if (!m || m->used >= m->ev.size()) return;
    if (cudaEventRecord(m->ev[m->used], st) == cudaSuccess) m->label[m->used++] = label;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); the static is initialised once, thread safe.
void *tensor_map_encoder() {
    static void *const fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return f;
    }();
    return fn;
}

int make_tma_map(TmaMap *out, const void *base, int W, int H, int boxw, int boxh, int elem_bytes) {
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!encode) return FIC_ECUDA;
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)W * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)boxw, (cuuint32_t)boxh};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = encode(&m, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return FIC_ECUDA;
    memcpy(out, &m, sizeof(TmaMap));
    return FIC_OK;
}

int box_width(int bmax, int W) {
    const int bw = bmax == 32 ? WinBox<32>::W : (bmax == 16 ? WinBox<16>::W : WinBox<8>::W);
    return bw < W ? bw : W;
}

cudaError_t launch_mns_encode(int bmax, const EncDesc *d_descs, int count, int total_strips, uint32_t *status,
                              uint32_t *ticket, cudaStream_t st);
cudaError_t launch_mns_encode_slots(int bmax, const EncDesc *d_descs, int count, int total_strips, int total_chunks,
                                    uint32_t *pack_status, uint32_t *ticket, const EncTune &tune, cudaStream_t st);
cudaError_t launch_local_encode(int bmax, const EncDesc *d_descs, int count, int total_strips, int total_chunks,
                                uint32_t *pack_status, cudaStream_t st);
cudaError_t launch_decode(int bmax, const DecDesc *d_descs, int count, int total_strips, void *tables, int iters,
                          bool d4, const DecTune &tune, cudaStream_t st);
cudaError_t launch_decode_leaves(const DecDesc *d_descs, const DecDesc *hdec, int count, int max_recs, int iters,
                                 cudaStream_t st);
int decode_d4_box(int bmax);
size_t decode_table_bytes_per_strip();
int mns_strip_width(int bmax);
}  // namespace fic

using namespace fic;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

inline bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int levels_of(const fic_params *p) {
    int L = 1;
    for (int b = p->bmax; b > p->bmin; b >>= 1) ++L;
    return L;
}

int check_params(const fic_params *p) {
    if (!p) return FIC_EBADPARAM;
    if (p->mode < FIC_NOSEARCH || p->mode > FIC_EXHAUSTIVE) return FIC_EBADPARAM;
    if (p->mode == FIC_EXHAUSTIVE &&
        (p->bmax != kExhB || p->bmin != kExhB || p->isometries < 1 || p->isometries > 8 || p->dom_step < 1 ||
         p->engine < 0 || p->engine > 1))
        return FIC_EBADPARAM;
    if (p->mode == FIC_LOCAL &&
        (p->local_radius < 0 || p->local_radius > 16 || (p->local_radius & 1) || p->local_step < 2 ||
         (p->local_step & 1)))
        return FIC_EBADPARAM;
    if (!(p->bmax == 8 || p->bmax == 16 || p->bmax == 32)) return FIC_EBADPARAM;
    // 2 x 2 leaves (the paper's 16 -> 2 quadtree) for the centred-domain modes
    const int min_b = (p->mode == FIC_NOSEARCH || p->mode == FIC_MNS) ? 2 : 4;
    if (!is_pow2(p->bmin) || p->bmin < min_b || p->bmin > p->bmax) return FIC_EBADPARAM;
    if (levels_of(p) > 4) return FIC_EBADPARAM;
    if (p->s_bits < 1 || p->s_bits > 7 || p->o_bits < 1 || p->o_bits > 8) return FIC_EBADPARAM;
    if (p->phase2_domain != 0 && p->phase2_domain != 1) return FIC_EBADPARAM;
    const int L = levels_of(p);
    for (int j = 0; j < L; ++j)
        if (!(p->thr_rms[j] >= 0.0) || !(p->thr_rms[j] < 256.0)) return FIC_EBADPARAM;
    return FIC_OK;
}

int check_size(int W, int H, const fic_params *p) {
    if (W <= 0 || H <= 0 || W > 65535 || H > 65535) return FIC_EBADSIZE;
    if (W % p->bmax || H % p->bmax || W % 16 || H % 16) return FIC_EBADSIZE;
    if (W < 2 * p->bmax || H < 2 * p->bmax) return FIC_EBADSIZE;
    return FIC_OK;
}

// Geometry and codebooks a stream must have to be stored, decoded,
// serialised or rescaled (the encoder's mode-specific limits -- the
// exhaustive search's 8x8 ranges, the local search's radius -- do not
// apply to a stream that already exists, e.g. one rescaled by 2).
int check_stream(int W, int H, const fic_params *p) {
    if (!p) return FIC_EBADPARAM;
    if (p->mode < FIC_NOSEARCH || p->mode > FIC_EXHAUSTIVE) return FIC_EBADPARAM;
    if (!(p->bmax == 8 || p->bmax == 16 || p->bmax == 32)) return FIC_EBADPARAM;
    if (!is_pow2(p->bmin) || p->bmin < 2 || p->bmin > p->bmax) return FIC_EBADPARAM;
    if (levels_of(p) > 4) return FIC_EBADPARAM;
    if (p->mode == FIC_EXHAUSTIVE && (p->bmin != p->bmax || p->isometries < 1 || p->isometries > 8 || p->dom_step < 1))
        return FIC_EBADPARAM;
    if (p->mode == FIC_LOCAL && (p->local_radius < 0 || p->local_step < 2 || (p->local_step & 1)))
        return FIC_EBADPARAM;
    if (p->s_bits < 1 || p->s_bits > 7 || p->o_bits < 1 || p->o_bits > 8) return FIC_EBADPARAM;
    if (p->phase2_domain != 0 && p->phase2_domain != 1) return FIC_EBADPARAM;
    return check_size(W, H, p);
}

inline int64_t t2q_of(double t) { return (int64_t)(t * t * 256.0 + 0.5); }

int strips_per_row(int W, int bmax) {
    const int tops = fic::mns_strip_width(bmax) / bmax;
    const int tw = W / bmax;
    return (tw + tops - 1) / tops;
}

int nstrips_of(int W, int H, int bmax) { return strips_per_row(W, bmax) * (H / bmax); }

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? FIC_OK : FIC_ECUDA; }

}  // namespace

// Host-side plan of an encode launch: the uploaded descriptor table and the
// look-back state live in the caller's workspace.
struct fic_plan {
    int kind;  // 0 encode, 1 decode
    int family;  // encode: 0 no-search / MNS, 1 local search, 2 exhaustive search
    int count;
    int bmax;
    int total_strips;
    int total_chunks;
    void *ws;
    size_t ws_bytes;
    EncDesc *d_enc;
    DecDesc *d_dec;
    uint32_t *status;
    uint32_t *ticket;
    std::vector<DecDesc> hdec;  // decode: host copy (buffers per image)
    std::vector<ExhDesc> hexh;  // exhaustive search: one descriptor per image (launched in turn)
    std::vector<int> engines;
    void *dec_tables;           // decode: per-strip transform tables
    std::vector<uint8_t *> outs;
    std::vector<size_t> out_bytes;
    EncTune etune;  // launch mapping (fic_plan_set_tuning / fic_plan_autotune)
    DecTune dtune;
    bool d4 = false;  // decode: iterate on 2x2-sum images (every stream centred)
    bool leaves = false;  // decode: a stream with 2 x 2 leaves (transform-per-thread iteration)
    int max_recs = 0;     // decode: the largest record capacity of the batch
};

// Exhaustive search: per image, decimated domains (packed) and the tensor
// path's screen operand, domain and range statistics, permuted range rows
// (fp16 and bytes) and per-row results.
struct ExhLayout {
    size_t dpairs, dsc, dstat, dscr, afp16, rbytes, rstat, row_g, row_dk, total;
};

static ExhLayout exh_layout(int W, int H, const fic_params *p, int *nd_out, int *nd_pad_out, int *ndx_out,
                            int *ndy_out) {
    const int ndx = (W - 2 * kExhB) / p->dom_step + 1, ndy = (H - 2 * kExhB) / p->dom_step + 1;
    const int nd = ndx * ndy, nd_pad = ((nd + kExhNTile - 1) / kExhNTile) * kExhNTile;
    const size_t nr = (size_t)(W / kExhB) * (H / kExhB);
    ExhLayout L;
    L.dpairs = 0;
    L.dsc = L.dpairs + align_up((size_t)nd * 128);
    L.dstat = L.dsc + align_up((size_t)nd_pad * 128);
    L.dscr = L.dstat + align_up((size_t)nd_pad * 16);
    L.afp16 = L.dscr + align_up((size_t)nd_pad * 16);
    L.rbytes = L.afp16 + align_up(nr * 8 * 128);
    L.rstat = L.rbytes + align_up(nr * 8 * 64);
    L.row_g = L.rstat + align_up(nr * 16);
    L.row_dk = L.row_g + align_up(nr * 8 * 8 * kExhMaxSeg);
    L.total = L.row_dk + align_up(nr * 8 * 8 * kExhMaxSeg);
    if (nd_out) *nd_out = nd;
    if (nd_pad_out) *nd_pad_out = nd_pad;
    if (ndx_out) *ndx_out = ndx;
    if (ndy_out) *ndy_out = ndy;
    return L;
}

// Plan of a batch of exhaustive searches: each image gets its own workspace
// slice and kernel sequence (prep, search, finalize).
static int exh_plan_create(const uint8_t *const *d_imgs, const int *widths, const int *heights, int count,
                           const fic_params *params, fic_stream *outs, void *d_workspace, size_t ws_bytes,
                           fic_plan **plan_out) {
    if ((reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1))) return FIC_ENOMEM;
    fic_plan *pl = new (std::nothrow) fic_plan();
    if (!pl) return FIC_ENOMEM;
    uint8_t *w = static_cast<uint8_t *>(d_workspace);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        const fic_params *p = &params[i];
        int rc = fic_validate(widths[i], heights[i], p);
        if (rc == FIC_OK && p->mode != FIC_EXHAUSTIVE) rc = FIC_EBADPARAM;
        fic_stream *o = &outs[i];
        if (rc == FIC_OK && (!d_imgs[i] || !o->records || !o->tile_offsets || !o->split || !o->info ||
                             (reinterpret_cast<uintptr_t>(o->records) & 15)))
            rc = FIC_EBADPARAM;
        const int W = widths[i], H = heights[i];
        if (rc == FIC_OK && o->capacity < (W / kExhB) * (H / kExhB)) rc = FIC_ECAPACITY;
        int nd = 0, nd_pad = 0, ndx = 0, ndy = 0;
        const ExhLayout L = exh_layout(W, H, p, &nd, &nd_pad, &ndx, &ndy);
        if (rc == FIC_OK && off + L.total > ws_bytes) rc = FIC_ENOMEM;
        if (rc) {
            delete pl;
            return rc;
        }
        o->width = W;
        o->height = H;
        o->params = *p;
        o->ntop = (W / kExhB) * (H / kExhB);
        ExhDesc E;
        std::memset(&E, 0, sizeof(E));
        E.img = d_imgs[i];
        E.W = W;
        E.H = H;
        E.nrx = W / kExhB;
        E.nry = H / kExhB;
        E.nr = E.nrx * E.nry;
        E.ndx = ndx;
        E.ndy = ndy;
        E.nd = nd;
        E.nd_pad = nd_pad;
        E.step = p->dom_step;
        E.isos = p->isometries;
        E.s_bits = p->s_bits;
        E.o_bits = p->o_bits;
        E.dpairs = reinterpret_cast<uint32_t *>(w + off + L.dpairs);
        E.dsc = reinterpret_cast<__half *>(w + off + L.dsc);
        E.dstat = reinterpret_cast<int4 *>(w + off + L.dstat);
        E.dscr = reinterpret_cast<float4 *>(w + off + L.dscr);
        E.nseg = 1;
        E.afp16 = reinterpret_cast<__half *>(w + off + L.afp16);
        E.rbytes = w + off + L.rbytes;
        E.rstat = reinterpret_cast<int4 *>(w + off + L.rstat);
        E.row_g = reinterpret_cast<long long *>(w + off + L.row_g);
        E.row_dk = reinterpret_cast<int2 *>(w + off + L.row_dk);
        E.rec = o->records;
        E.tile_off = o->tile_offsets;
        E.split = o->split;
        E.info = o->info;
        off += L.total;
        pl->hexh.push_back(E);
        pl->engines.push_back(p->engine);
    }
    pl->kind = 0;
    pl->family = 2;
    pl->count = count;
    pl->bmax = kExhB;
    pl->ws = d_workspace;
    pl->ws_bytes = ws_bytes;
    *plan_out = pl;
    return FIC_OK;
}

extern "C" {

int fic_version(void) { return 100; }

const char *fic_strerror(int code) {
    switch (code) {
    case FIC_OK: return "ok";
    case FIC_EBADSIZE: return "unsupported image size";
    case FIC_EBADPARAM: return "invalid parameter";
    case FIC_ENOMEM: return "buffer or workspace too small";
    case FIC_ECAPACITY: return "record buffer too small";
    case FIC_ECUDA: return "CUDA error";
    case FIC_ETIMEOUT: return "device wait timed out";
    case FIC_EBUDGET: return "request exceeds the memory budget";
    case FIC_EBUSY: return "busy";
    case FIC_ECANCELLED: return "cancelled";
    default: return "unknown error";
    }
}

int fic_validate_stream(int width, int height, const fic_params *p) { return check_stream(width, height, p); }

int fic_validate(int width, int height, const fic_params *p) {
    int rc = check_params(p);
    if (rc) return rc;
    return check_size(width, height, p);
}

int fic_stream_sizes(int width, int height, const fic_params *p, int32_t *ntop, int32_t *max_records) {
    int rc = check_stream(width, height, p);
    if (rc) return rc;
    if (ntop) *ntop = (width / p->bmax) * (height / p->bmax);
    if (max_records) *max_records = (width / p->bmin) * (height / p->bmin);
    return FIC_OK;
}

// Encoder workspace layout (each part 256-byte aligned): tensor maps, image
// descriptors, per-strip (count, fits), pack look-back status (one word per
// 32-strip chunk + 1), per-strip record slots (64 records = 1 KiB per strip).
struct EncLayout {
    size_t maps, descs, stats, pstatus, slots, total;
};

static EncLayout enc_layout(int count, size_t strips, size_t chunks, size_t slot_records) {
    EncLayout L;
    L.maps = 0;
    L.descs = L.maps + align_up(sizeof(TmaMap) * (size_t)count);
    L.stats = L.descs + align_up(sizeof(EncDesc) * (size_t)count);
    L.pstatus = L.stats + align_up(8 * strips);
    L.slots = L.pstatus + align_up(4 * (2 * chunks + 1));  // status, strip counter, chunk counters
    L.total = L.slots + align_up(sizeof(fic_record) * slot_records);
    return L;
}

// Records one strip of 1024 pixels can emit: a 4 x 4 leaf each 16 pixels,
// a 2 x 2 leaf each 4.
static int slot_records_of(const fic_params *p) { return p->bmin < 4 ? 256 : 64; }

size_t fic_encode_workspace_bytes(int count, const int *widths, const int *heights, const fic_params *params) {
    if (count <= 0 || !widths || !heights || !params) return 0;
    size_t strips = 0, chunks = 0, exh = 0, slot_recs = 0;
    for (int i = 0; i < count; ++i) {
        if (fic_validate(widths[i], heights[i], &params[i])) return 0;
        if (params[i].mode == FIC_EXHAUSTIVE) {
            exh += exh_layout(widths[i], heights[i], &params[i], nullptr, nullptr, nullptr, nullptr).total;
            continue;
        }
        const size_t n = (size_t)nstrips_of(widths[i], heights[i], params[i].bmax);
        strips += n;
        chunks += (n + 31) / 32;
        slot_recs += n * (size_t)slot_records_of(&params[i]);
    }
    return enc_layout(count, strips, chunks, slot_recs).total + exh;
}

}  // extern "C"

namespace fic {

size_t encode_plan_staging_bytes(int count) {
    return align_up(sizeof(TmaMap) * (size_t)count) + align_up(sizeof(EncDesc) * (size_t)count);
}

size_t decode_plan_staging_bytes(int count) {
    return align_up(sizeof(DecDesc) * (size_t)count) + align_up(2 * sizeof(TmaMap) * (size_t)count);
}

// `staging`, when given, is pinned host memory of encode_plan_staging_bytes
// that must stay untouched until the plan's work on `stream` has run: the
// descriptor upload is then a true asynchronous copy.
int encode_plan_create_staged(const uint8_t *const *d_imgs, const int *widths, const int *heights, int count,
                              const fic_params *params, fic_stream *outs, void *d_workspace, size_t ws_bytes,
                              void *stream, uint8_t *staging, fic_plan **plan_out) {
    if (!plan_out || count <= 0 || !d_imgs || !widths || !heights || !params || !outs || !d_workspace)
        return FIC_EBADPARAM;
    *plan_out = nullptr;
    if (params[0].mode == FIC_EXHAUSTIVE)
        return exh_plan_create(d_imgs, widths, heights, count, params, outs, d_workspace, ws_bytes, plan_out);
    const int bmax = params[0].bmax;
    std::vector<EncDesc> h((size_t)count);
    std::vector<TmaMap> maps((size_t)count);
    const TmaMap *d_maps = static_cast<const TmaMap *>(d_workspace);
    int strips = 0, chunks = 0;
    size_t slot_recs = 0;
    std::vector<size_t> slot_base((size_t)count);
    bool min2 = false;  // a stream with 2 x 2 leaves
    for (int i = 0; i < count; ++i) {
        const fic_params *p = &params[i];
        int rc = fic_validate(widths[i], heights[i], p);
        if (rc) return rc;
        if (p->bmax != bmax) return FIC_EBADPARAM;
        if ((p->mode == FIC_LOCAL) != (params[0].mode == FIC_LOCAL) || p->mode == FIC_EXHAUSTIVE)
            return FIC_EBADPARAM;  // one kernel family per launch
        if (!d_imgs[i] || (reinterpret_cast<uintptr_t>(d_imgs[i]) & 15)) return FIC_EBADPARAM;
        fic_stream *o = &outs[i];
        if (!o->records || !o->tile_offsets || !o->split || !o->info || o->capacity <= 0) return FIC_EBADPARAM;
        if (reinterpret_cast<uintptr_t>(o->records) & 15) return FIC_EBADPARAM;
        if (reinterpret_cast<uintptr_t>(o->info) & 7) return FIC_EBADPARAM;
        const int W = widths[i], H = heights[i];
        o->width = W;
        o->height = H;
        o->params = *p;
        o->ntop = (W / bmax) * (H / bmax);
        EncDesc &d = h[(size_t)i];
        std::memset(&d, 0, sizeof(d));
        d.img = d_imgs[i];
        d.rec = o->records;
        d.tile_off = o->tile_offsets;
        d.split = o->split;
        d.info = o->info;
        const int L = levels_of(p);
        for (int j = 0; j < 4; ++j) d.t2q[j] = t2q_of(p->thr_rms[j < L ? j : L - 1]);
        d.W = W;
        d.H = H;
        d.tw = W / bmax;
        d.th = H / bmax;
        d.spr = strips_per_row(W, bmax);
        d.strip_base = strips;
        d.nstrips = nstrips_of(W, H, bmax);
        d.capacity = o->capacity;
        d.mode = p->mode;
        d.bmin = p->bmin;
        d.L = L;
        d.phase2 = p->phase2 ? 1 : 0;
        d.phase2_domain = p->phase2_domain ? 1 : 0;
        d.s_bits = p->s_bits;
        d.o_bits = p->o_bits;
        d.local_radius = p->local_radius;
        d.local_step = p->local_step;
        d.boxw = box_width(bmax, W);
        d.bmax = bmax;
        d.map = d_maps + i;
        rc = make_tma_map(&maps[(size_t)i], d_imgs[i], W, H, d.boxw, 2 * bmax);
        if (rc) return rc;
        d.chunk_base = chunks;
        d.nchunks = (d.nstrips + 31) / 32;
        d.slot_recs = slot_records_of(p);
        slot_base[(size_t)i] = slot_recs;
        slot_recs += (size_t)d.nstrips * (size_t)d.slot_recs;
        min2 = min2 || p->bmin < 4;
        strips += d.nstrips;
        chunks += d.nchunks;
    }
    const EncLayout lay = enc_layout(count, (size_t)strips, (size_t)chunks, slot_recs);
    const size_t need = lay.total;
    if (ws_bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1))) return FIC_ENOMEM;
    fic_plan *pl = new (std::nothrow) fic_plan();
    if (!pl) return FIC_ENOMEM;
    uint8_t *w = static_cast<uint8_t *>(d_workspace);
    pl->kind = 0;
    pl->family = params[0].mode == FIC_LOCAL ? 1 : 0;
    pl->count = count;
    pl->bmax = bmax;
    pl->total_strips = strips;
    pl->ws = d_workspace;
    pl->ws_bytes = ws_bytes;
    pl->d_enc = reinterpret_cast<EncDesc *>(w + lay.descs);
    pl->status = reinterpret_cast<uint32_t *>(w + lay.pstatus);
    pl->ticket = pl->status + chunks;  // the strip counter of the dynamic schedule
    pl->total_chunks = chunks;
    pl->d_dec = nullptr;
    {
        bool own_domains = true;  // every image's phase-2 sub-blocks use their own centred domains
        for (int i = 0; i < count; ++i) own_domains = own_domains && !params[i].phase2_domain;
        pl->etune.kernel32 = (bmax == 32 && own_domains) ? 1 : 0;
        pl->etune.min2 = min2 ? 1 : 0;
    }
    {
        fic_record *slots = reinterpret_cast<fic_record *>(w + lay.slots);
        uint2 *stats = reinterpret_cast<uint2 *>(w + lay.stats);
        for (int i = 0; i < count; ++i) {
            h[(size_t)i].slots = slots + slot_base[(size_t)i];
            h[(size_t)i].stats = stats + h[(size_t)i].strip_base;
        }
    }
    const void *src_maps = maps.data(), *src_descs = h.data();
    if (staging) {
        memcpy(staging, maps.data(), sizeof(TmaMap) * (size_t)count);
        memcpy(staging + align_up(sizeof(TmaMap) * (size_t)count), h.data(), sizeof(EncDesc) * (size_t)count);
        src_maps = staging;
        src_descs = staging + align_up(sizeof(TmaMap) * (size_t)count);
    }
    cudaError_t e = cudaMemcpyAsync(w, src_maps, sizeof(TmaMap) * (size_t)count, cudaMemcpyHostToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->ticket, 0, sizeof(uint32_t), static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pl->d_enc, src_descs, sizeof(EncDesc) * (size_t)count, cudaMemcpyHostToDevice,
                            static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        delete pl;
        return FIC_ECUDA;
    }
    *plan_out = pl;
    return FIC_OK;
}

}  // namespace fic

extern "C" {

int fic_encode_plan_create(const uint8_t *const *d_imgs, const int *widths, const int *heights, int count,
                           const fic_params *params, fic_stream *outs, void *d_workspace, size_t ws_bytes,
                           void *stream, fic_plan **plan_out) {
    return encode_plan_create_staged(d_imgs, widths, heights, count, params, outs, d_workspace, ws_bytes, stream,
                                     nullptr, plan_out);
}

int fic_encode_plan_run(const fic_plan *pl, void *stream) {
    if (!pl || pl->kind != 0) return FIC_EBADPARAM;
    fic::TraceRange tr("fic encode");
    if (pl->family == 2) {
        for (size_t i = 0; i < pl->hexh.size(); ++i) {
            const cudaError_t e = launch_exhaustive(pl->hexh[i], pl->engines[i], static_cast<cudaStream_t>(stream));
            if (e != cudaSuccess) return FIC_ECUDA;
        }
        return FIC_OK;
    }
    if (pl->family == 1)
        return cuda_rc(launch_local_encode(pl->bmax, pl->d_enc, pl->count, pl->total_strips, pl->total_chunks,
                                           pl->status, static_cast<cudaStream_t>(stream)));
    return cuda_rc(launch_mns_encode_slots(pl->bmax, pl->d_enc, pl->count, pl->total_strips, pl->total_chunks,
                                           pl->status, pl->ticket, pl->etune, static_cast<cudaStream_t>(stream)));
}

void fic_plan_destroy(fic_plan *pl) { delete pl; }

int fic_plan_run_timed(const fic_plan *pl, int iters, void *stream, float *ms, const char **labels, int cap,
                       int *n) {
    if (!pl || !ms || !n || cap < 1 || cap > 4096 || (pl->kind == 1 && iters < 0)) return FIC_EBADPARAM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StageMarks m;
    m.ev.resize((size_t)cap + 1, nullptr);
    m.label.resize((size_t)cap + 1, nullptr);
    int rc = FIC_OK;
    for (auto &e : m.ev)
        if (cudaEventCreate(&e) != cudaSuccess) rc = FIC_ECUDA;
    cudaEvent_t start = m.ev.back();
    m.ev.pop_back();
    if (rc == FIC_OK && cudaEventRecord(start, st) != cudaSuccess) rc = FIC_ECUDA;
    if (rc == FIC_OK) {
        t_marks = &m;
        rc = pl->kind == 0 ? fic_encode_plan_run(pl, stream) : fic_decode_plan_run(pl, iters, stream);
        t_marks = nullptr;
    }
    if (rc == FIC_OK && m.used > 0 && cudaEventSynchronize(m.ev[m.used - 1]) != cudaSuccess) rc = FIC_ECUDA;
    for (size_t i = 0; rc == FIC_OK && i < m.used; ++i) {
        if (cudaEventElapsedTime(&ms[i], i ? m.ev[i - 1] : start, m.ev[i]) != cudaSuccess) rc = FIC_ECUDA;
        if (labels) labels[i] = m.label[i];
    }
    *n = rc == FIC_OK ? (int)m.used : 0;
    for (auto e : m.ev)
        if (e) cudaEventDestroy(e);
    if (start) cudaEventDestroy(start);
    return rc;
}

int fic_plan_get_tuning(const fic_plan *pl, fic_tuning *t) {
    if (!pl || !t) return FIC_EBADPARAM;
    t->enc_warps = pl->etune.warps;
    t->enc_ctas_per_sm = pl->etune.ctas_per_sm;
    t->enc_dynamic = pl->etune.dynamic;
    t->dec_ctas_per_sm = pl->dtune.ctas_per_sm;
    t->enc_fused_pack = pl->etune.fused_pack;
    t->dec_single_launch = pl->dtune.single_launch;
    return FIC_OK;
}

int fic_plan_set_tuning(fic_plan *pl, const fic_tuning *t) {
    if (!pl || !t) return FIC_EBADPARAM;
    if ((t->enc_warps != 8 && t->enc_warps != 4) || t->enc_ctas_per_sm < 0 || t->enc_ctas_per_sm > 64 ||
        (t->enc_dynamic != 0 && t->enc_dynamic != 1) || t->dec_ctas_per_sm < 0 || t->dec_ctas_per_sm > 64 ||
        (t->enc_fused_pack != 0 && t->enc_fused_pack != 1) ||
        (t->dec_single_launch != 0 && t->dec_single_launch != 1))
        return FIC_EBADPARAM;
    pl->etune.warps = t->enc_warps;
    pl->etune.ctas_per_sm = t->enc_ctas_per_sm;
    pl->etune.dynamic = t->enc_dynamic;
    pl->dtune.ctas_per_sm = t->dec_ctas_per_sm;
    pl->etune.fused_pack = t->enc_fused_pack;
    pl->dtune.single_launch = t->dec_single_launch;
    return FIC_OK;
}

int fic_plan_autotune(fic_plan *pl, int iters, int reps, void *stream, fic_tuning *best, float *best_ms,
                      float *trace, int trace_cap, int *ntrace) {
    if (!pl || reps < 1 || reps > 1000 || (pl->kind == 0 && pl->family != 0) || (pl->kind == 1 && iters < 1))
        return FIC_EBADPARAM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // candidate list; CTAs per SM beyond what fits is clamped by the
    // launcher, so every count up to the register limit is tried
    std::vector<fic_tuning> cands;
    fic_tuning cur;
    fic_plan_get_tuning(pl, &cur);
    if (pl->kind == 0) {
        for (int w : {8, 4})
            for (int k = 1; k <= (w == 8 ? 3 : 4); ++k)
                for (int dyn = 0; dyn <= 1; ++dyn)
                    for (int fp = 1; fp >= 0; --fp)
                        cands.push_back(fic_tuning{w, k, dyn, cur.dec_ctas_per_sm, fp, cur.dec_single_launch});
    } else {
        // the iteration kernels are built for 4 resident CTAs of 8 warps (a
        // 48-register build for 5 measured slower: 113 vs 105 us per decode)
        for (int one = 1; one >= 0; --one)
            for (int k = 1; k <= 4; ++k)
                cands.push_back(
                    fic_tuning{cur.enc_warps, cur.enc_ctas_per_sm, cur.enc_dynamic, k, cur.enc_fused_pack, one});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FIC_ECUDA;
    }
    auto run = [&]() { return pl->kind == 0 ? fic_encode_plan_run(pl, stream) : fic_decode_plan_run(pl, iters, stream); };
    int rc = FIC_OK, nt = 0, bi = -1;
    float bms = 0.f;
    std::vector<float> times((size_t)reps);
    for (size_t c = 0; c < cands.size() && rc == FIC_OK; ++c) {
        fic_plan_set_tuning(pl, &cands[c]);
        rc = run();  // untimed
        for (int r = 0; r < reps && rc == FIC_OK; ++r) {
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = FIC_ECUDA;
            if (rc == FIC_OK) rc = run();
            if (rc == FIC_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = FIC_ECUDA;
            if (rc == FIC_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = FIC_ECUDA;
            if (rc == FIC_OK && cudaEventElapsedTime(&times[(size_t)r], e0, e1) != cudaSuccess) rc = FIC_ECUDA;
        }
        if (rc != FIC_OK) break;
        std::sort(times.begin(), times.end());
        const float med = times[(size_t)reps / 2];
        if (trace && nt < trace_cap) {
            float *row = trace + 7 * nt;
            row[0] = (float)cands[c].enc_warps;
            row[1] = (float)cands[c].enc_ctas_per_sm;
            row[2] = (float)cands[c].enc_dynamic;
            row[3] = (float)cands[c].dec_ctas_per_sm;
            row[4] = (float)cands[c].enc_fused_pack;
            row[5] = (float)cands[c].dec_single_launch;
            row[6] = med;
            ++nt;
        }
        if (bi < 0 || med < bms) {
            bi = (int)c;
            bms = med;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FIC_OK) {
        fic_plan_set_tuning(pl, &cur);
        return rc;
    }
    fic_plan_set_tuning(pl, &cands[(size_t)bi]);
    if (best) *best = cands[(size_t)bi];
    if (best_ms) *best_ms = bms;
    if (ntrace) *ntrace = nt;
    return FIC_OK;
}

int fic_encode_batch(const uint8_t *const *d_imgs, const int *widths, const int *heights, int count,
                     const fic_params *params, fic_stream *outs, void *d_workspace, size_t workspace_bytes,
                     void *stream) {
    fic_plan *pl = nullptr;
    int rc = fic_encode_plan_create(d_imgs, widths, heights, count, params, outs, d_workspace, workspace_bytes,
                                    stream, &pl);
    if (rc) return rc;
    rc = fic_encode_plan_run(pl, stream);
    fic_plan_destroy(pl);
    return rc;
}

int fic_encode(const uint8_t *d_img, int width, int height, const fic_params *p, fic_stream *out,
               void *d_workspace, size_t workspace_bytes, void *stream) {
    return fic_encode_batch(&d_img, &width, &height, 1, p, out, d_workspace, workspace_bytes, stream);
}

// Decoder workspace layout (each part 256-byte aligned): image descriptors,
// one scratch iterate per image, per-strip transform tables.
// Decoder workspace head: descriptors, then two tensor maps per image (the
// 2x2-sum ping-pong images of centred streams).
static size_t dec_head_bytes(int count) {
    return align_up(sizeof(DecDesc) * (size_t)count) + align_up(2 * sizeof(TmaMap) * (size_t)count);
}

size_t fic_decode_workspace_bytes(int count, const int *widths, const int *heights) {
    if (count <= 0 || !widths || !heights) return 0;
    size_t b = dec_head_bytes(count);
    size_t strips = 0;
    for (int i = 0; i < count; ++i) {
        if (widths[i] <= 0 || heights[i] <= 0) return 0;
        b += align_up((size_t)widths[i] * (size_t)heights[i]);
        // strip count for the bmax that needs the most (the plan knows bmax)
        size_t most = 0;
        for (int bm = 8; bm <= 32; bm *= 2) {
            const size_t n = (size_t)strips_per_row(widths[i], bm) * (size_t)(heights[i] / bm);
            if (n > most) most = n;
        }
        strips += most;
    }
    return b + align_up(strips * decode_table_bytes_per_strip());
}

}  // extern "C"

namespace fic {

int decode_plan_create_staged(const fic_stream *sts, int count, uint8_t *const *d_outs, void *d_workspace,
                              size_t ws_bytes, void *stream, uint8_t *staging, fic_plan **plan_out) {
    if (!plan_out || count <= 0 || !sts || !d_outs || !d_workspace) return FIC_EBADPARAM;
    *plan_out = nullptr;
    const int bmax = sts[0].params.bmax;
    std::vector<int> ws((size_t)count), hs((size_t)count);
    for (int i = 0; i < count; ++i) {
        ws[(size_t)i] = sts[i].width;
        hs[(size_t)i] = sts[i].height;
    }
    const size_t need = fic_decode_workspace_bytes(count, ws.data(), hs.data());
    if (need == 0) return FIC_EBADPARAM;
    if (ws_bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1))) return FIC_ENOMEM;
    fic_plan *pl = new (std::nothrow) fic_plan();
    if (!pl) return FIC_ENOMEM;
    pl->hdec.resize((size_t)count);
    uint8_t *w = static_cast<uint8_t *>(d_workspace);
    uint8_t *scratch = w + dec_head_bytes(count);
    TmaMap *d_maps = reinterpret_cast<TmaMap *>(w + align_up(sizeof(DecDesc) * (size_t)count));
    std::vector<TmaMap> maps(2 * (size_t)count);
    // 2x2-sum iteration when every stream uses centred domains and is wide
    // enough for the window box
    bool d4 = true, leaves = false;
    int max_recs = 0;
    for (int i = 0; i < count; ++i) {
        d4 = d4 && (sts[i].params.mode == FIC_NOSEARCH || sts[i].params.mode == FIC_MNS) &&
             sts[i].width / 2 >= decode_d4_box(bmax);
        leaves = leaves || sts[i].params.bmin < 4;
        if (sts[i].params.bmin > 0)
            max_recs = std::max(max_recs, (sts[i].width / sts[i].params.bmin) * (sts[i].height / sts[i].params.bmin));
    }
    if (leaves) d4 = false;
    int strips = 0;
    for (int i = 0; i < count; ++i) {
        const fic_stream *s = &sts[i];
        int rc = check_stream(s->width, s->height, &s->params);
        if (rc == FIC_OK && s->params.bmax != bmax) rc = FIC_EBADPARAM;
        if (rc == FIC_OK && (!s->records || !s->tile_offsets || !d_outs[i] ||
                             (reinterpret_cast<uintptr_t>(d_outs[i]) & 15)))
            rc = FIC_EBADPARAM;
        if (rc) {
            delete pl;
            return rc;
        }
        DecDesc &d = pl->hdec[(size_t)i];
        std::memset(&d, 0, sizeof(d));
        d.rec = s->records;
        d.tile_off = s->tile_offsets;
        d.buf[0] = d_outs[i];
        d.buf[1] = scratch;
        if (d4) {
            const size_t half = (size_t)s->width * (size_t)s->height / 2;  // one (W/2) x (H/2) uint16 image
            d.d4[0] = reinterpret_cast<uint16_t *>(scratch);
            d.d4[1] = reinterpret_cast<uint16_t *>(scratch + half);
            for (int k = 0; k < 2; ++k) {
                rc = make_tma_map(&maps[2 * (size_t)i + k], d.d4[k], s->width / 2, s->height / 2, decode_d4_box(bmax),
                                  bmax, 2);
                if (rc) {
                    delete pl;
                    return rc;
                }
                d.map[k] = d_maps + 2 * i + k;
            }
            d.info = s->info;
        }
        scratch += align_up((size_t)s->width * (size_t)s->height);
        d.W = s->width;
        d.H = s->height;
        d.tw = s->width / bmax;
        d.th = s->height / bmax;
        d.spr = strips_per_row(s->width, bmax);
        d.strip_base = strips;
        d.nstrips = nstrips_of(s->width, s->height, bmax);
        d.mode = s->params.mode;
        d.bmin = s->params.bmin;
        d.L = levels_of(&s->params);
        d.s_bits = s->params.s_bits;
        d.o_bits = s->params.o_bits;
        d.phase2_domain = s->params.phase2_domain ? 1 : 0;
        strips += d.nstrips;
        pl->outs.push_back(d_outs[i]);
        pl->out_bytes.push_back((size_t)s->width * (size_t)s->height);
    }
    pl->kind = 1;
    pl->count = count;
    pl->bmax = bmax;
    pl->d4 = d4;
    pl->leaves = leaves;
    pl->max_recs = max_recs;
    pl->total_strips = strips;
    pl->dec_tables = scratch;  // after the per-image iterate buffers
    pl->ws = d_workspace;
    pl->ws_bytes = ws_bytes;
    pl->d_dec = reinterpret_cast<DecDesc *>(w);
    pl->d_enc = nullptr;
    const void *src = pl->hdec.data(), *src_maps = maps.data();
    if (staging) {
        memcpy(staging, pl->hdec.data(), sizeof(DecDesc) * (size_t)count);
        memcpy(staging + align_up(sizeof(DecDesc) * (size_t)count), maps.data(), 2 * sizeof(TmaMap) * (size_t)count);
        src = staging;
        src_maps = staging + align_up(sizeof(DecDesc) * (size_t)count);
    }
    cudaError_t e = cudaMemcpyAsync(pl->d_dec, src, sizeof(DecDesc) * (size_t)count, cudaMemcpyHostToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e == cudaSuccess && d4)
        e = cudaMemcpyAsync(d_maps, src_maps, 2 * sizeof(TmaMap) * (size_t)count, cudaMemcpyHostToDevice,
                            static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        delete pl;
        return FIC_ECUDA;
    }
    *plan_out = pl;
    return FIC_OK;
}

}  // namespace fic

extern "C" {

int fic_decode_plan_create(const fic_stream *sts, int count, uint8_t *const *d_outs, void *d_workspace,
                           size_t ws_bytes, void *stream, fic_plan **plan_out) {
    return decode_plan_create_staged(sts, count, d_outs, d_workspace, ws_bytes, stream, nullptr, plan_out);
}

int fic_decode_plan_run(const fic_plan *pl, int iters, void *stream) {
    if (!pl || pl->kind != 1 || iters < 0) return FIC_EBADPARAM;
    fic::TraceRange tr("fic decode");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (iters == 0) {
        for (size_t i = 0; i < pl->outs.size(); ++i) {
            cudaError_t e = cudaMemsetAsync(pl->outs[i], 128, pl->out_bytes[i], st);
            if (e != cudaSuccess) return FIC_ECUDA;
        }
        return FIC_OK;
    }
    if (pl->leaves)
        return cuda_rc(launch_decode_leaves(pl->d_dec, pl->hdec.data(), pl->count, pl->max_recs, iters, st));
    return cuda_rc(launch_decode(pl->bmax, pl->d_dec, pl->count, pl->total_strips, pl->dec_tables, iters, pl->d4,
                                 pl->dtune, st));
}

int fic_decode_batch(const fic_stream *sts, int count, int iters, uint8_t *const *d_outs, void *d_workspace,
                     size_t workspace_bytes, void *stream) {
    fic_plan *pl = nullptr;
    int rc = fic_decode_plan_create(sts, count, d_outs, d_workspace, workspace_bytes, stream, &pl);
    if (rc) return rc;
    rc = fic_decode_plan_run(pl, iters, stream);
    fic_plan_destroy(pl);
    return rc;
}

int fic_decode(const fic_stream *st, int iters, uint8_t *d_out, void *d_workspace, size_t workspace_bytes,
               void *stream) {
    return fic_decode_batch(st, 1, iters, &d_out, d_workspace, workspace_bytes, stream);
}

int fic_stream_info(const fic_stream *st, int64_t *records, int64_t *fits, void *stream) {
    if (!st || !st->info) return FIC_EBADPARAM;
    uint32_t h[FIC_INFO_WORDS];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h, st->info, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return FIC_ECUDA;
    if (records) *records = (int64_t)h[FIC_INFO_RECORDS];
    if (fits) *fits = (int64_t)h[FIC_INFO_FITS_LO] | ((int64_t)h[FIC_INFO_FITS_HI] << 32);
    if (h[FIC_INFO_ERROR] & FIC_DEVERR_TIMEOUT) return FIC_ETIMEOUT;
    if (h[FIC_INFO_ERROR] & FIC_DEVERR_CAPACITY) return FIC_ECAPACITY;
    if (h[FIC_INFO_ERROR] & FIC_DEVERR_FORMAT) return FIC_EBADPARAM;
    return FIC_OK;
}

}  // extern "C"
