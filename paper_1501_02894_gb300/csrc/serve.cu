// serve.cu -- request server with continuous batching (fic_submit & co).
//
// Host-side runtime around the encoder and decoder kernels: one device
// arena (the HBM budget) and one pinned host arena are allocated when the
// server is created and sub-allocated per job and per batch; a worker thread
// admits queued jobs in arrival order as their memory fits, groups admitted
// jobs into batches (encode: same bmax and search family; decode: same
// bmax), launches each batch as one batched plan on one of several CUDA
// streams, and completes jobs when their batch's event fires.  Jobs that
// arrive while batches run are admitted as soon as memory frees, so batches
// of different arrival times overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fic_internal.cuh"
#include "trace.cuh"

namespace fic {
size_t encode_plan_staging_bytes(int count);
size_t decode_plan_staging_bytes(int count);
int encode_plan_create_staged(const uint8_t *const *d_imgs, const int *widths, const int *heights, int count,
                              const fic_params *params, fic_stream *outs, void *d_workspace, size_t ws_bytes,
                              void *stream, uint8_t *staging, fic_plan **plan_out);
int decode_plan_create_staged(const fic_stream *sts, int count, uint8_t *const *d_outs, void *d_workspace,
                              size_t ws_bytes, void *stream, uint8_t *staging, fic_plan **plan_out);
}  // namespace fic

namespace {

using Clock = std::chrono::steady_clock;

inline size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// First-fit sub-allocator over one block (256-byte granules, coalescing).
class Arena {
  public:
    void init(uint8_t *base, size_t size) {
        base_ = base;
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
    }
    uint8_t *alloc(size_t n) {
        n = a256(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            used_ += n;
            peak_ = std::max(peak_, used_);
            return base_ + off;
        }
        return nullptr;
    }
    void release(uint8_t *p, size_t n) {
        if (!p) return;
        n = a256(n ? n : 1);
        size_t off = (size_t)(p - base_);
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    size_t size() const { return size_; }
    size_t peak() const { return peak_; }

  private:
    uint8_t *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Alloc {
    uint8_t *p = nullptr;
    size_t n = 0;
};

// Host copies between the caller's buffers and pinned staging.  Large ones
// are split over a few helper threads: one thread's memcpy bandwidth would
// otherwise bound the server on big images.
class CopyPool {
  public:
    explicit CopyPool(int helpers) {
        for (int i = 0; i < helpers; ++i) threads_.emplace_back([this] { run(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : threads_) t.join();
    }
    void copy(void *dst, const void *src, size_t n) {
        const size_t parts = std::min(threads_.size() + 1, n / kChunk);
        if (parts <= 1) {
            memcpy(dst, src, n);
            return;
        }
        const size_t per = (n / parts + 63) & ~(size_t)63;
        std::atomic<int> left((int)parts - 1);
        {
            std::lock_guard<std::mutex> g(mu_);
            for (size_t k = 1; k < parts; ++k) {
                const size_t off = k * per, len = std::min(per, n - std::min(n, off));
                tasks_.push_back(Task{static_cast<uint8_t *>(dst) + off, static_cast<const uint8_t *>(src) + off, len,
                                      &left});
            }
        }
        cv_.notify_all();
        memcpy(dst, src, std::min(per, n));
        while (left.load(std::memory_order_acquire) > 0) std::this_thread::yield();
    }

  private:
    static constexpr size_t kChunk = 256 << 10;  // copies of 512 KiB and more are split
    struct Task {
        uint8_t *dst;
        const uint8_t *src;
        size_t n;
        std::atomic<int> *left;
    };
    void run() {
        for (;;) {
            Task t;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [this] { return stop_ || !tasks_.empty(); });
                if (stop_ && tasks_.empty()) return;
                t = tasks_.front();
                tasks_.pop_front();
            }
            if (t.n) memcpy(t.dst, t.src, t.n);
            t.left->fetch_sub(1, std::memory_order_release);
        }
    }
    std::vector<std::thread> threads_;
    std::deque<Task> tasks_;
    std::mutex mu_;
    std::condition_variable cv_;
    bool stop_ = false;
};

struct Job {
    int64_t ticket = 0;
    fic_job job{};
    Clock::time_point t_submit, t_launch;
    size_t footprint = 0;  // device bytes accounted for admission
    int ntop = 0, cap = 0;
    // device buffers
    Alloc d_img, d_rec, d_meta, d_out;
    // pinned staging: inputs then outputs
    Alloc h_stage;
    fic_stream st{};
    fic_job_result res{};
    bool done = false;
};

struct Batch {
    std::vector<Job *> jobs;
    int stream = 0;
    cudaEvent_t ev = nullptr;
    Alloc d_ws, h_desc;
};

}  // namespace

struct fic_server {
    fic_server_config cfg{};
    std::vector<cudaStream_t> streams;
    std::vector<int> inflight_per_stream;
    uint8_t *d_base = nullptr, *h_base = nullptr;
    Arena dev, host;
    size_t dev_accounted = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;                       // submitted, not admitted
    std::deque<Job *> admitted;                    // admitted, not launched
    std::vector<Batch *> inflight;
    std::unordered_map<int64_t, Job *> jobs;      // all live tickets
    int64_t next_ticket = 1;
    bool stopping = false;
    std::thread worker;
    CopyPool copies{6};  // helpers: host copies of big images and results at high request rates

    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched_jobs = 0;
    std::vector<double> latencies;
};

namespace {

// Device bytes of a job alone: its buffers plus its part of a batch workspace.
size_t job_footprint(const fic_job &j, int *ntop, int *cap) {
    const fic_params &p = j.params;
    int32_t nt = 0, mr = 0;
    if (fic_stream_sizes(j.width, j.height, &p, &nt, &mr)) return 0;
    *ntop = nt;
    *cap = mr;
    const size_t meta = a256(4 * ((size_t)nt + 1)) + a256(4 * (size_t)nt) + 256;
    const size_t img = (size_t)j.width * j.height;
    if (j.kind == FIC_JOB_ENCODE) {
        const size_t ws = fic_encode_workspace_bytes(1, &j.width, &j.height, &p);
        return a256(img) + a256((size_t)mr * 16) + meta + ws + 4096;
    }
    const size_t ws = fic_decode_workspace_bytes(1, &j.width, &j.height);
    return a256((size_t)std::max(j.nrecords, 1) * 16) + meta + a256(img) + ws + 4096;
}

size_t job_staging(const Job &J) {
    const size_t img = (size_t)J.job.width * J.job.height;
    if (J.job.kind == FIC_JOB_ENCODE)
        return a256(img) + a256((size_t)J.cap * 16) + a256(4 * (size_t)J.ntop) + 256;
    return a256((size_t)std::max(J.job.nrecords, 1) * 16) + a256(4 * ((size_t)J.ntop + 1)) + a256(img);
}

void free_job(fic_server *S, Job *J) {
    S->dev.release(J->d_img.p, J->d_img.n);
    S->dev.release(J->d_rec.p, J->d_rec.n);
    S->dev.release(J->d_meta.p, J->d_meta.n);
    S->dev.release(J->d_out.p, J->d_out.n);
    S->host.release(J->h_stage.p, J->h_stage.n);
    J->d_img = J->d_rec = J->d_meta = J->d_out = J->h_stage = Alloc{};
    std::lock_guard<std::mutex> g(S->mu);
    S->dev_accounted -= J->footprint;
}

// Allocate a job's buffers and stage its inputs (worker thread).
bool prepare_job(fic_server *S, Job *J) {
    fic::TraceRange tr("fic server: admit job");
    const fic_job &j = J->job;
    const size_t img = (size_t)j.width * j.height;
    auto dget = [&](Alloc &a, size_t n) {
        a.n = n;
        a.p = S->dev.alloc(n);
        return a.p != nullptr;
    };
    J->h_stage.n = job_staging(*J);
    J->h_stage.p = S->host.alloc(J->h_stage.n);
    bool ok = J->h_stage.p != nullptr;
    const size_t meta = a256(4 * ((size_t)J->ntop + 1)) + a256(4 * (size_t)J->ntop) + 256;
    if (j.kind == FIC_JOB_ENCODE) {
        ok = ok && dget(J->d_img, img) && dget(J->d_rec, (size_t)J->cap * 16) && dget(J->d_meta, meta);
        if (ok) S->copies.copy(J->h_stage.p, j.image, img);
    } else {
        ok = ok && dget(J->d_rec, (size_t)std::max(j.nrecords, 1) * 16) && dget(J->d_meta, meta) &&
             dget(J->d_out, img);
        if (ok) {
            // records and the tile offsets of the canonical order
            S->copies.copy(J->h_stage.p, j.records, (size_t)j.nrecords * 16);
            uint32_t *offs = reinterpret_cast<uint32_t *>(J->h_stage.p + a256((size_t)std::max(j.nrecords, 1) * 16));
            const int bmax = j.params.bmax, tw = j.width / bmax;
            int r = 0;
            for (int t = 0; t <= J->ntop; ++t) {
                while (r < j.nrecords && (int)(j.records[r].y / bmax) * tw + (int)(j.records[r].x / bmax) < t) ++r;
                offs[t] = (uint32_t)r;
            }
            offs[J->ntop] = (uint32_t)j.nrecords;
        }
    }
    if (!ok) {
        S->dev.release(J->d_img.p, J->d_img.n);
        S->dev.release(J->d_rec.p, J->d_rec.n);
        S->dev.release(J->d_meta.p, J->d_meta.n);
        S->dev.release(J->d_out.p, J->d_out.n);
        S->host.release(J->h_stage.p, J->h_stage.n);
        J->d_img = J->d_rec = J->d_meta = J->d_out = J->h_stage = Alloc{};
        return false;
    }
    fic_stream &st = J->st;
    memset(&st, 0, sizeof(st));
    st.width = j.width;
    st.height = j.height;
    st.params = j.params;
    st.ntop = J->ntop;
    st.capacity = j.kind == FIC_JOB_ENCODE ? J->cap : std::max(j.nrecords, 1);
    st.records = reinterpret_cast<fic_record *>(J->d_rec.p);
    st.tile_offsets = reinterpret_cast<uint32_t *>(J->d_meta.p);
    st.split = reinterpret_cast<uint32_t *>(J->d_meta.p + a256(4 * ((size_t)J->ntop + 1)));
    st.info = reinterpret_cast<uint32_t *>(J->d_meta.p + a256(4 * ((size_t)J->ntop + 1)) + a256(4 * (size_t)J->ntop));
    return true;
}

// Jobs in one batch share kind, search family and bmax (one launch
// configuration) and, for decoding, the iteration count.
int64_t batch_key(const fic_job &j) {
    const int64_t fam = j.params.mode == FIC_LOCAL ? 1 : (j.params.mode == FIC_EXHAUSTIVE ? 2 : 0);
    const int64_t iters = j.kind == FIC_JOB_DECODE ? j.iters : 0;
    return (iters << 24) | ((int64_t)j.kind << 16) | (fam << 8) | j.params.bmax;
}

// Morton index of cell (cx, cy) of a top-level block: TL, TR, BL, BR order.
int morton(int cx, int cy) {
    int m = 0;
    for (int b = 0; b < 4; ++b) m |= (((cx >> b) & 1) << (2 * b)) | (((cy >> b) & 1) << (2 * b + 1));
    return m;
}

// Records of a decode job come from the caller's host memory: check that
// they form a stream the decoder can read (every leaf inside the image, the
// leaves of each top-level block an exact quadtree partition in depth-first
// order, codes within their codebooks, domains inside the image).
bool records_valid(const fic_job &j) {
    const fic_params &p = j.params;
    int L = 1;
    for (int b = p.bmax; b > p.bmin; b >>= 1) ++L;
    const int tw = j.width / p.bmax, ntop = tw * (j.height / p.bmax);
    const int cells = p.bmax / p.bmin;
    int tile = 0, cursor = 0;
    for (int i = 0; i < j.nrecords; ++i) {
        const fic_record &r = j.records[i];
        if (r.level < 1 || r.level > L) return false;
        const int b = p.bmax >> (r.level - 1);
        if (r.x % b || r.y % b || r.x + b > j.width || r.y + b > j.height) return false;
        const int t = (r.y / p.bmax) * tw + r.x / p.bmax;
        if (t != tile) {
            if (t < tile || cursor != cells * cells) return false;  // previous tile incomplete
            if (t != tile + 1) return false;                          // a tile with no leaf
            tile = t;
            cursor = 0;
        }
        if (morton((r.x % p.bmax) / p.bmin, (r.y % p.bmax) / p.bmin) != cursor) return false;
        cursor += (b / p.bmin) * (b / p.bmin);
        if (r.q >= (1 << p.o_bits)) return false;
        if (r.phase == 1) {
            if (r.k >= (1 << p.s_bits)) return false;
        } else if (r.phase == 2) {
            if (p.mode != FIC_MNS || r.level >= L || r.level > 3 || r.k >= 16) return false;
        } else {
            return false;
        }
        if (p.mode == FIC_LOCAL || p.mode == FIC_EXHAUSTIVE) {
            if (r.iso > 7 || r.dx + 2 * b > j.width || r.dy + 2 * b > j.height) return false;
        }
    }
    return j.nrecords > 0 && tile == ntop - 1 && cursor == cells * cells;
}

// Enqueue one batch on its stream: inputs in, one batched launch, outputs out.
int launch_batch(fic_server *S, Batch *B) {
    fic::TraceRange tr(B->jobs[0]->job.kind == FIC_JOB_ENCODE ? "fic server: encode batch" : "fic server: decode batch");
    cudaStream_t s = S->streams[(size_t)B->stream];
    const int n = (int)B->jobs.size();
    const fic_job &j0 = B->jobs[0]->job;
    std::vector<const uint8_t *> imgs;
    std::vector<int> W, H;
    std::vector<fic_params> P;
    std::vector<fic_stream> sts;
    std::vector<uint8_t *> outs;
    for (Job *J : B->jobs) {
        const fic_job &j = J->job;
        const size_t img = (size_t)j.width * j.height;
        if (j.kind == FIC_JOB_ENCODE) {
            if (cudaMemcpyAsync(J->d_img.p, J->h_stage.p, img, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return FIC_ECUDA;
            imgs.push_back(J->d_img.p);
        } else {
            const size_t rb = (size_t)std::max(j.nrecords, 1) * 16;
            if (cudaMemcpyAsync(J->d_rec.p, J->h_stage.p, (size_t)j.nrecords * 16, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess ||
                cudaMemcpyAsync(J->st.tile_offsets, J->h_stage.p + a256(rb), 4 * ((size_t)J->ntop + 1),
                                cudaMemcpyHostToDevice, s) != cudaSuccess)
                return FIC_ECUDA;
            outs.push_back(J->d_out.p);
        }
        W.push_back(j.width);
        H.push_back(j.height);
        P.push_back(j.params);
        sts.push_back(J->st);
    }
    fic_plan *plan = nullptr;
    int rc;
    if (j0.kind == FIC_JOB_ENCODE) {
        rc = fic::encode_plan_create_staged(imgs.data(), W.data(), H.data(), n, P.data(), sts.data(), B->d_ws.p,
                                            B->d_ws.n, s, B->h_desc.p, &plan);
        if (rc == FIC_OK) rc = fic_encode_plan_run(plan, s);
    } else {
        rc = fic::decode_plan_create_staged(sts.data(), n, outs.data(), B->d_ws.p, B->d_ws.n, s, B->h_desc.p, &plan);
        if (rc == FIC_OK && S->streams.size() > 1) {
            // batches on other streams run beside this one: no grid barriers
            fic_tuning t;
            fic_plan_get_tuning(plan, &t);
            t.dec_single_launch = 0;
            rc = fic_plan_set_tuning(plan, &t);
        }
        if (rc == FIC_OK) rc = fic_decode_plan_run(plan, j0.iters, s);
    }
    if (plan) fic_plan_destroy(plan);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        Job *J = B->jobs[(size_t)i];
        const fic_job &j = J->job;
        const size_t img = (size_t)j.width * j.height;
        cudaError_t e;
        if (j.kind == FIC_JOB_ENCODE) {
            J->st = sts[(size_t)i];
            uint8_t *h = J->h_stage.p + a256(img);
            e = cudaMemcpyAsync(h, J->st.records, (size_t)J->cap * 16, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h + a256((size_t)J->cap * 16), J->st.split, 4 * (size_t)J->ntop,
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h + a256((size_t)J->cap * 16) + a256(4 * (size_t)J->ntop), J->st.info, 64,
                                    cudaMemcpyDeviceToHost, s);
        } else {
            const size_t rb = (size_t)std::max(j.nrecords, 1) * 16;
            e = cudaMemcpyAsync(J->h_stage.p + a256(rb) + a256(4 * ((size_t)J->ntop + 1)), J->d_out.p, img,
                                cudaMemcpyDeviceToHost, s);
        }
        if (e != cudaSuccess) return FIC_ECUDA;
    }
    return cudaEventRecord(B->ev, s) == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

// Copy a finished job's outputs to the caller and fill its result.
void finish_job(fic_server *S, Job *J, int status, Clock::time_point now) {
    fic::TraceRange tr("fic server: complete job");
    const fic_job &j = J->job;
    const size_t img = (size_t)j.width * j.height;
    fic_job_result &r = J->res;
    r.status = status;
    if (status == FIC_OK && j.kind == FIC_JOB_ENCODE) {
        const uint8_t *h = J->h_stage.p + a256(img);
        const uint32_t *info =
            reinterpret_cast<const uint32_t *>(h + a256((size_t)J->cap * 16) + a256(4 * (size_t)J->ntop));
        if (info[FIC_INFO_ERROR] & FIC_DEVERR_TIMEOUT) r.status = FIC_ETIMEOUT;
        else if (info[FIC_INFO_ERROR] & FIC_DEVERR_CAPACITY) r.status = FIC_ECAPACITY;
        r.nrecords = (int32_t)info[FIC_INFO_RECORDS];
        r.fits = (int64_t)info[FIC_INFO_FITS_LO] | ((int64_t)info[FIC_INFO_FITS_HI] << 32);
        if (j.out_records) S->copies.copy(j.out_records, h, (size_t)std::min(r.nrecords, J->cap) * 16);
        if (j.out_split) memcpy(j.out_split, h + a256((size_t)J->cap * 16), 4 * (size_t)J->ntop);
    } else if (status == FIC_OK) {
        const size_t rb = (size_t)std::max(j.nrecords, 1) * 16;
        if (j.out_image) S->copies.copy(j.out_image, J->h_stage.p + a256(rb) + a256(4 * ((size_t)J->ntop + 1)), img);
    }
    r.latency_ms = std::chrono::duration<double, std::milli>(now - J->t_submit).count();
    r.queue_ms = std::chrono::duration<double, std::milli>(J->t_launch - J->t_submit).count();
    free_job(S, J);
}

// The worker.  Queues shared with fic_submit / fic_poll are touched under
// the mutex only; the arenas, the admitted list and the in-flight batches
// belong to the worker alone, so copies and launches run without the lock.
void worker_main(fic_server *S) {
    cudaSetDevice(S->cfg.device);
    int rr = 0;
    for (;;) {
        bool progress = false;
        // 1. admission in arrival order while the budget allows
        for (;;) {
            Job *J = nullptr;
            {
                std::lock_guard<std::mutex> g(S->mu);
                if (!S->queue.empty() && S->dev_accounted + S->queue.front()->footprint <= (size_t)S->cfg.hbm_budget_bytes) {
                    J = S->queue.front();
                    S->queue.pop_front();
                    S->dev_accounted += J->footprint;
                }
            }
            if (!J) break;
            if (!prepare_job(S, J)) {  // fragmentation: retry when memory frees
                std::lock_guard<std::mutex> g(S->mu);
                S->dev_accounted -= J->footprint;
                if (S->inflight.empty() && S->admitted.empty()) {
                    // both arenas are wholly free and the job still cannot be
                    // placed: no later release can help, so it fails now
                    J->res.status = FIC_ENOMEM;
                    J->res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - J->t_submit).count();
                    J->done = true;
                    S->completed += 1;
                    S->cv_done.notify_all();
                    progress = true;
                    continue;
                }
                S->queue.push_front(J);
                break;
            }
            S->admitted.push_back(J);
            progress = true;
        }
        // 2. batches of admitted jobs, on streams with room
        while (!S->admitted.empty()) {
            int sidx = -1;
            for (int k = 0; k < (int)S->streams.size(); ++k) {
                const int c = (rr + k) % (int)S->streams.size();
                if (S->inflight_per_stream[(size_t)c] < 2) {
                    sidx = c;
                    break;
                }
            }
            if (sidx < 0) break;
            rr = (sidx + 1) % (int)S->streams.size();
            Batch *B = new Batch();
            B->stream = sidx;
            const int64_t key = batch_key(S->admitted.front()->job);
            for (auto it = S->admitted.begin(); it != S->admitted.end() && (int)B->jobs.size() < S->cfg.max_batch;) {
                if (batch_key((*it)->job) == key) {
                    B->jobs.push_back(*it);
                    it = S->admitted.erase(it);
                } else {
                    ++it;
                }
            }
            // The batch workspace; when it does not fit, the batch is halved
            // (each job's footprint already counts a workspace of its own).
            const bool enc = B->jobs[0]->job.kind == FIC_JOB_ENCODE;
            for (;;) {
                const int n = (int)B->jobs.size();
                std::vector<int> W, H;
                std::vector<fic_params> P;
                for (Job *J : B->jobs) {
                    W.push_back(J->job.width);
                    H.push_back(J->job.height);
                    P.push_back(J->job.params);
                }
                B->d_ws.n = enc ? fic_encode_workspace_bytes(n, W.data(), H.data(), P.data())
                                : fic_decode_workspace_bytes(n, W.data(), H.data());
                B->d_ws.p = S->dev.alloc(B->d_ws.n);
                B->h_desc.n = enc ? fic::encode_plan_staging_bytes(n) : fic::decode_plan_staging_bytes(n);
                B->h_desc.p = S->host.alloc(B->h_desc.n);
                if ((B->d_ws.p && B->h_desc.p) || n == 1) break;
                S->dev.release(B->d_ws.p, B->d_ws.n);
                S->host.release(B->h_desc.p, B->h_desc.n);
                B->d_ws = B->h_desc = Alloc{};
                for (int k = n - 1; k >= n / 2; --k) S->admitted.push_front(B->jobs[(size_t)k]);
                B->jobs.resize((size_t)(n / 2));
            }
            const int n = (int)B->jobs.size();
            if (!B->d_ws.p || !B->h_desc.p) {
                S->dev.release(B->d_ws.p, B->d_ws.n);
                S->host.release(B->h_desc.p, B->h_desc.n);
                if (!S->inflight.empty()) {
                    // room comes back when a running batch completes
                    S->admitted.push_front(B->jobs[0]);
                    delete B;
                    break;
                }
                // nothing running to wait for: the arena is fragmented past use
                for (Job *J : B->jobs) finish_job(S, J, FIC_ENOMEM, Clock::now());
                {
                    std::lock_guard<std::mutex> g(S->mu);
                    for (Job *J : B->jobs) {
                        J->done = true;
                        S->completed += 1;
                    }
                }
                delete B;
                S->cv_done.notify_all();
                continue;
            }
            cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
            const auto now = Clock::now();
            for (Job *J : B->jobs) J->t_launch = now;
            const int rc = launch_batch(S, B);
            S->batches += 1;
            S->batched_jobs += n;
            if (rc != FIC_OK) {
                cudaStreamSynchronize(S->streams[(size_t)sidx]);
                for (Job *J : B->jobs) finish_job(S, J, rc, Clock::now());
                S->dev.release(B->d_ws.p, B->d_ws.n);
                S->host.release(B->h_desc.p, B->h_desc.n);
                cudaEventDestroy(B->ev);
                {
                    std::lock_guard<std::mutex> g(S->mu);
                    for (Job *J : B->jobs) {
                        J->done = true;
                        S->completed += 1;
                    }
                }
                delete B;
                S->cv_done.notify_all();
                continue;
            }
            S->inflight_per_stream[(size_t)sidx] += 1;
            S->inflight.push_back(B);
            progress = true;
        }
        // 3. completions
        for (size_t i = 0; i < S->inflight.size();) {
            Batch *B = S->inflight[i];
            const cudaError_t q = cudaEventQuery(B->ev);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const auto now = Clock::now();
            for (Job *J : B->jobs) finish_job(S, J, q == cudaSuccess ? FIC_OK : FIC_ECUDA, now);
            S->dev.release(B->d_ws.p, B->d_ws.n);
            S->host.release(B->h_desc.p, B->h_desc.n);
            cudaEventDestroy(B->ev);
            S->inflight_per_stream[(size_t)B->stream] -= 1;
            {
                std::lock_guard<std::mutex> g(S->mu);
                for (Job *J : B->jobs) {
                    J->done = true;
                    S->completed += 1;
                    S->latencies.push_back(J->res.latency_ms);
                }
            }
            delete B;
            S->inflight.erase(S->inflight.begin() + (long)i);
            progress = true;
            S->cv_done.notify_all();
        }
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stopping && S->queue.empty() && S->admitted.empty() && S->inflight.empty()) break;
        if (!progress) {
            // batches in flight are polled every 20 us; with none, only a
            // submit or the shutdown (both signal cv_work) can change anything
            if (!S->inflight.empty() || !S->admitted.empty())
                S->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
    }
}

}  // namespace

extern "C" {

int fic_server_create(const fic_server_config *cfg, fic_server **out) {
    if (!cfg || !out || cfg->streams < 1 || cfg->max_batch < 1 || cfg->queue_capacity < 1 ||
        cfg->hbm_budget_bytes <= 0 || cfg->host_staging_bytes <= 0)
        return FIC_EBADPARAM;
    *out = nullptr;
    fic_server *S = new (std::nothrow) fic_server();
    if (!S) return FIC_ENOMEM;
    S->cfg = *cfg;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete S;
        return FIC_ECUDA;
    }
    if (cudaMalloc(&S->d_base, (size_t)cfg->hbm_budget_bytes) != cudaSuccess) {
        delete S;
        return FIC_ENOMEM;
    }
    if (cudaHostAlloc(&S->h_base, (size_t)cfg->host_staging_bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaFree(S->d_base);
        delete S;
        return FIC_ENOMEM;
    }
    S->dev.init(S->d_base, (size_t)cfg->hbm_budget_bytes);
    S->host.init(S->h_base, (size_t)cfg->host_staging_bytes);
    for (int i = 0; i < cfg->streams; ++i) {
        cudaStream_t s;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        S->streams.push_back(s);
        S->inflight_per_stream.push_back(0);
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return FIC_OK;
}

int fic_submit(fic_server *S, const fic_job *job, int64_t *ticket) {
    if (!S || !job || !ticket) return FIC_EBADPARAM;
    if (job->kind != FIC_JOB_ENCODE && job->kind != FIC_JOB_DECODE) return FIC_EBADPARAM;
    if (job->kind == FIC_JOB_ENCODE && (!job->image || !job->out_records)) return FIC_EBADPARAM;
    if (job->kind == FIC_JOB_DECODE && (!job->records || job->nrecords <= 0 || !job->out_image || job->iters < 0))
        return FIC_EBADPARAM;
    const int rc = job->kind == FIC_JOB_ENCODE ? fic_validate(job->width, job->height, &job->params)
                                               : fic_validate_stream(job->width, job->height, &job->params);
    if (rc) return rc;
    if (job->kind == FIC_JOB_DECODE && !records_valid(*job)) return FIC_EBADPARAM;
    Job *J = new (std::nothrow) Job();
    if (!J) return FIC_ENOMEM;
    J->job = *job;
    J->footprint = job_footprint(*job, &J->ntop, &J->cap);
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stopping) {
        delete J;
        return FIC_ECANCELLED;
    }
    if (J->footprint == 0 || J->footprint > (size_t)S->cfg.hbm_budget_bytes ||
        job_staging(*J) > (size_t)S->cfg.host_staging_bytes) {
        S->rejected += 1;
        delete J;
        return FIC_EBUDGET;
    }
    if ((int64_t)S->jobs.size() >= S->cfg.queue_capacity) {
        delete J;
        return FIC_EBUSY;
    }
    J->ticket = S->next_ticket++;
    J->t_submit = Clock::now();
    S->jobs[J->ticket] = J;
    S->queue.push_back(J);
    S->submitted += 1;
    *ticket = J->ticket;
    S->cv_work.notify_one();
    return FIC_OK;
}

int fic_poll(fic_server *S, int64_t ticket, fic_job_result *res) {
    if (!S) return FIC_EBADPARAM;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return FIC_EBADPARAM;
    Job *J = it->second;
    if (!J->done) return FIC_EBUSY;
    if (res) *res = J->res;
    const int st = J->res.status;
    S->jobs.erase(it);
    delete J;
    return st;
}

int fic_wait(fic_server *S, int64_t ticket, int32_t timeout_ms, fic_job_result *res) {
    if (!S) return FIC_EBADPARAM;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return FIC_EBADPARAM;
    Job *J = it->second;
    auto pred = [&] { return J->done; };
    if (timeout_ms < 0) S->cv_done.wait(lk, pred);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return FIC_ETIMEOUT;
    if (res) *res = J->res;
    const int st = J->res.status;
    S->jobs.erase(ticket);
    delete J;
    return st;
}

int fic_server_get_stats(fic_server *S, fic_server_stats *st) {
    if (!S || !st) return FIC_EBADPARAM;
    std::lock_guard<std::mutex> g(S->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->rejected = S->rejected;
    st->batches = S->batches;
    st->peak_device_bytes = (int64_t)S->dev.peak();
    st->mean_batch = S->batches ? (double)S->batched_jobs / (double)S->batches : 0.0;
    if (!S->latencies.empty()) {
        std::vector<double> v = S->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
            return v[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / (double)v.size();
    }
    return FIC_OK;
}

int fic_server_destroy(fic_server *S) {
    if (!S) return FIC_EBADPARAM;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->jobs) delete kv.second;
    for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
    cudaFreeHost(S->h_base);
    cudaFree(S->d_base);
    delete S;
    return FIC_OK;
}

}  // extern "C"
