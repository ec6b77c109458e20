// serve.cpp -- continuous batching of smearing jobs (tls_serve_* in include/tls.h).
//
// The pattern the paper builds towards (Sec. 3, Sec. 6): one two-link field W
// per gauge configuration stays resident and is reused by every source and
// sink smeared on it.  Here jobs arrive at any time; a scheduler thread packs
// the vectors of compatible jobs (same gauge, storage precision and slice
// selection) into the slots of one multi-right-hand-side batch and advances
// all active slots together, `steps_per_launch` smearing steps per round.
// Between rounds it retires finished jobs and admits waiting ones into free
// slots, so new work joins a running batch instead of waiting for it.
//
// Per-slot state lives in device tables: alpha[j][s] = width/(4N) of the job
// in slot s for step j of the round, and active[j][s] = 1 while that job has
// steps left.  Inactive slots are skipped by the kernel, so a finished slot
// keeps its result in the buffer its last step wrote.  The per-vector
// arithmetic is that of the multi-RHS step kernel (interleaved layout, one
// record per slot), so a job's result is
// bitwise the same alone and in any mix.  A round's launches are captured
// once per (batch, starting buffer) in a CUDA graph and replayed; batches
// run on their own streams and overlap on the device.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>

#include "api_internal.h"

namespace tls {

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t id = 0;
    tls_job d{};
    tls_status status = TLS_OK;
    bool done = false;
    double submit_ms = 0, start_ms = -1, done_ms = -1;
    int slot0 = -1;
    int parity = -1;            // buffer holding the result once finished
    void *staging = nullptr;    // device copy of host vectors
    size_t staging_bytes = 0;
};

struct BatchKey {
    int64_t gauge;
    int storage, timeslice;
    bool operator<(const BatchKey &o) const
    {
        if (gauge != o.gauge) return gauge < o.gauge;
        if (storage != o.storage) return storage < o.storage;
        return timeslice < o.timeslice;
    }
};

struct Batch {
    BatchKey key{};
    int S = 0, K = 1, vb = 8;
    int nsl = 0, t_first = 0, nblk = 0;
    int64_t vs = 0;
    char *buf[2] = {nullptr, nullptr};
    size_t buf_bytes = 0;
    double *d_alpha = nullptr;
    int *d_active = nullptr;
    double *h_alpha = nullptr;
    int *h_active = nullptr;
    size_t tab_bytes = 0;    // one K x S table of 8-byte entries
    size_t alpha_bytes = 0;  // the alpha table: FP64 entries, then the same rounded to FP32
    int cur = 0;
    std::vector<Job *> slot_job;
    std::vector<int> slot_left;
    std::vector<double> slot_alpha;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool launched = false;
    int *d_err = nullptr;    // device error word of this batch's kernels (bounded waits)
    int *h_err = nullptr;    // pinned copy, read after each round

    int active_slots() const
    {
        int n = 0;
        for (int s = 0; s < S; ++s) n += slot_left[s] > 0;
        return n;
    }
    int used_slots() const
    {
        int n = 0;
        for (int s = 0; s < S; ++s) n += slot_job[s] != nullptr;
        return n;
    }
};

}  // namespace

struct Server {
    tls_serve_opts opts{};
    std::thread th;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<Job *> pending;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    uint64_t next_id = 1;
    std::map<BatchKey, std::unique_ptr<Batch>> batches;
    Clock::time_point t0;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

size_t io_elem(int io_prec) { return io_prec == TLS_F64 ? 8 : 4; }

void destroy_batch(tls_ctx *ctx, Batch *b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    dev_free(ctx, b->buf[0], b->buf_bytes);
    dev_free(ctx, b->buf[1], b->buf_bytes);
    dev_free(ctx, b->d_alpha, b->alpha_bytes);
    dev_free(ctx, b->d_active, b->tab_bytes);
    if (b->h_alpha) cudaFreeHost(b->h_alpha);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->stream) cudaStreamDestroy(b->stream);
    dev_free(ctx, b->d_err, 256);
    if (b->h_err) cudaFreeHost(b->h_err);
}

// Slots of a batch: FP32 and 16-bit record groups hold an even number of vectors.
int batch_slots(int storage, int max_slots) { return storage != TLS_F64 ? (max_slots + 1) & ~1 : max_slots; }

size_t batch_bytes(const Gauge &gg, int storage, int timeslice, int S, int K)
{
    S = batch_slots(storage, S);
    const int nsl = timeslice < 0 ? gg.L[3] : 1;
    const int64_t vs = (int64_t)nsl * 8 * gg.g.Ps * vfmt_bytes(storage);
    return 2 * (size_t)vs * S + 2 * (size_t)K * S * 8 + (size_t)K * S * 4 + 256;
}

tls_status make_batch(tls_ctx *ctx, Server *sv, const BatchKey &key, const Gauge &gg, Batch **out)
{
    std::unique_ptr<Batch> b(new Batch());
    b->key = key;
    b->S = batch_slots(key.storage, sv->opts.max_slots);
    b->K = sv->opts.steps_per_launch;
    b->vb = default_il_vb(key.storage, b->S);
    b->nsl = key.timeslice < 0 ? gg.L[3] : 1;
    b->t_first = key.timeslice < 0 ? 0 : key.timeslice;
    b->nblk = b->nsl * 8;
    b->vs = (int64_t)b->nblk * gg.g.Ps * vfmt_bytes(key.storage);
    b->buf_bytes = (size_t)b->vs * b->S;
    b->tab_bytes = (size_t)b->K * b->S * 8;
    b->alpha_bytes = b->tab_bytes + (size_t)b->K * b->S * 4;
    tls_status s = dev_alloc(ctx, (void **)&b->buf[0], b->buf_bytes, "serve: batch buffer A");
    if (s == TLS_OK) s = dev_alloc(ctx, (void **)&b->buf[1], b->buf_bytes, "serve: batch buffer B");
    if (s == TLS_OK) s = dev_alloc(ctx, (void **)&b->d_alpha, b->alpha_bytes, "serve: alpha table");
    if (s == TLS_OK) s = dev_alloc(ctx, (void **)&b->d_active, b->tab_bytes, "serve: active table");
    if (s == TLS_OK) s = dev_alloc(ctx, (void **)&b->d_err, 256, "serve: error word");
    if (s == TLS_OK && cudaMallocHost(&b->h_err, sizeof(int)) != cudaSuccess) s = fail(TLS_ERR_NOMEM, "serve: pinned word");
    if (s == TLS_OK && cudaMallocHost(&b->h_alpha, b->alpha_bytes) != cudaSuccess) s = fail(TLS_ERR_NOMEM, "serve: pinned table");
    if (s == TLS_OK && cudaMallocHost(&b->h_active, b->tab_bytes) != cudaSuccess) s = fail(TLS_ERR_NOMEM, "serve: pinned table");
    if (s == TLS_OK && cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        s = fail(TLS_ERR_CUDA, "serve: stream");
    if (s != TLS_OK) {
        destroy_batch(ctx, b.get());
        return s;
    }
    cudaMemsetAsync(b->d_err, 0, 256, b->stream);
    *b->h_err = 0;
    cudaMemsetAsync(b->buf[0], 0, b->buf_bytes, b->stream);
    cudaMemsetAsync(b->buf[1], 0, b->buf_bytes, b->stream);
    b->slot_job.assign(b->S, nullptr);
    b->slot_left.assign(b->S, 0);
    b->slot_alpha.assign(b->S, 0.0);
    *out = b.get();
    sv->batches[key] = std::move(b);
    return TLS_OK;
}

int find_slots(const Batch &b, int n)
{
    for (int s0 = 0; s0 + n <= b.S; ++s0) {
        bool free = true;
        for (int s = s0; s < s0 + n && free; ++s) free = b.slot_job[s] == nullptr;
        if (free) return s0;
    }
    return -1;
}

void finish(Server *sv, Job *j, tls_status st)
{
    std::lock_guard<std::mutex> lk(sv->m);
    j->status = st;
    j->done = true;
    j->done_ms = sv->now_ms();
    sv->cv_done.notify_all();
}

// Frees batches with no slot in use (except `keep`).  Returns true if any was freed.
bool drop_idle_batches(tls_ctx *ctx, Server *sv, const Batch *keep)
{
    bool any = false;
    for (auto it = sv->batches.begin(); it != sv->batches.end();) {
        Batch *b = it->second.get();
        if (b != keep && b->used_slots() == 0) {
            destroy_batch(ctx, b);
            it = sv->batches.erase(it);
            any = true;
        } else {
            ++it;
        }
    }
    return any;
}

bool any_busy(const Server *sv)
{
    for (auto &kv : sv->batches)
        if (kv.second->used_slots() > 0) return true;
    return false;
}

// 0: admitted (or finished with an error), 1: must wait for resources.
int try_admit(tls_ctx *ctx, Server *sv, Job *j)
{
    auto git = ctx->gauges.find(j->d.gauge);
    if (git == ctx->gauges.end() || !git->second.built) {
        finish(sv, j, fail(TLS_ERR_NOT_BUILT, "serve: gauge %lld is gone or not built", (long long)j->d.gauge));
        return 0;
    }
    const Gauge &gg = git->second;
    BatchKey key{j->d.gauge, j->d.storage, j->d.timeslice};
    Batch *b = nullptr;
    auto bit = sv->batches.find(key);
    if (bit != sv->batches.end()) {
        b = bit->second.get();
    } else {
        tls_status s = make_batch(ctx, sv, key, gg, &b);
        if (s == TLS_ERR_ADMIT || s == TLS_ERR_NOMEM) {
            if (drop_idle_batches(ctx, sv, nullptr)) s = make_batch(ctx, sv, key, gg, &b);
        }
        if (s != TLS_OK) {
            if (!any_busy(sv)) {
                finish(sv, j, s);
                return 0;
            }
            return 1;
        }
    }
    const int s0 = find_slots(*b, j->d.nvec);
    if (s0 < 0) return 1;
    const int64_t Vslice = (int64_t)gg.L[0] * gg.L[1] * gg.L[2];
    const int64_t V = Vslice * gg.L[3];
    const size_t slice_b = (size_t)Vslice * 6 * io_elem(j->d.io_prec);
    const char *src = (const char *)j->d.vecs;
    int64_t svs = V;
    int t_rel = b->t_first;
    if (!j->d.vecs_on_device) {
        j->staging_bytes = slice_b * b->nsl * j->d.nvec;
        tls_status s = dev_alloc(ctx, &j->staging, j->staging_bytes, "serve: host staging");
        if (s != TLS_OK) {
            j->staging = nullptr;
            if (!any_busy(sv)) {
                finish(sv, j, s);
                return 0;
            }
            return 1;
        }
        const size_t width = slice_b * b->nsl, pitch = (size_t)V * 6 * io_elem(j->d.io_prec);
        cudaError_t e = cudaMemcpy2DAsync(j->staging, width, src + (size_t)b->t_first * slice_b, pitch, width,
                                          j->d.nvec, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) {
            dev_free(ctx, j->staging, j->staging_bytes);
            j->staging = nullptr;
            finish(sv, j, cuda_fail(e, "serve: host to device"));
            return 0;
        }
        src = (const char *)j->staging;
        svs = Vslice * b->nsl;
        t_rel = 0;
    }
    cudaError_t e = launch_pack_il(src, j->d.io_prec, svs, b->buf[b->cur], j->d.storage, gg.g, gg.L, t_rel, b->nsl,
                                   j->d.nvec, b->S, s0, b->stream);
    if (e != cudaSuccess) {
        finish(sv, j, cuda_fail(e, "serve: pack"));
        return 0;
    }
    const double a = j->d.N > 0 ? j->d.width / (4.0 * j->d.N) : 0.0;
    for (int s = s0; s < s0 + j->d.nvec; ++s) {
        b->slot_job[s] = j;
        b->slot_left[s] = j->d.N;
        b->slot_alpha[s] = a;
    }
    j->slot0 = s0;
    j->parity = j->d.N == 0 ? b->cur : -1;
    {
        std::lock_guard<std::mutex> lk(sv->m);
        j->start_ms = sv->now_ms();
    }
    return 0;
}

cudaError_t launch_round(tls_ctx *ctx, Server *sv, Batch *b)
{
    const Gauge &gg = ctx->gauges.at(b->key.gauge);
    for (int j = 0; j < b->K; ++j)
        for (int s = 0; s < b->S; ++s) {
            const bool on = b->slot_left[s] > j;
            b->h_active[j * b->S + s] = on ? 1 : 0;
            b->h_alpha[j * b->S + s] = on ? b->slot_alpha[s] : 0.0;
        }
    float *h_alphaf = reinterpret_cast<float *>(b->h_alpha + (size_t)b->K * b->S);
    for (size_t k = 0; k < (size_t)b->K * b->S; ++k) h_alphaf[k] = (float)b->h_alpha[k];  // round to nearest
    cudaError_t e = cudaMemcpyAsync(b->d_alpha, b->h_alpha, b->alpha_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_active, b->h_active, b->tab_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return e;
    StepArgs sa{};
    sa.W = gg.W + (size_t)b->t_first * 8 * 3 * gg.g.Ps * wfmt_bytes(gg.wfmt);
    sa.g = gg.g;
    sa.nblk = b->nblk;
    sa.nvec = b->S;
    sa.vstride_in = sa.vstride_out = b->vs;
    sa.wfmt = gg.wfmt;
    sa.prec_in = sa.prec_out = b->key.storage;
    sa.vb = b->vb;
    sa.threads = 128;
    // FP32 and 16-bit batches: whole-row CTAs with the W rows staged by TMA and
    // vector-pair arithmetic (the packed kernel where the row shape does not
    // allow it); FP64 batches use the plain interleaved kernel
    if (b->key.storage != TLS_F64) sa.tile[1] = 6;
    sa.err = b->d_err;
    const float *d_alphaf = reinterpret_cast<const float *>(b->d_alpha + (size_t)b->K * b->S);
    sa.stream = b->stream;
    auto issue = [&]() -> cudaError_t {
        for (int j = 0; j < b->K; ++j) {
            sa.in = b->buf[(b->cur + j) & 1];
            sa.out = b->buf[(b->cur + j + 1) & 1];
            sa.alpha = b->d_alpha + (size_t)j * b->S;
            sa.alphaf = d_alphaf + (size_t)j * b->S;
            sa.active = b->d_active + (size_t)j * b->S;
            cudaError_t r = launch_step_il(sa);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    if (sv->opts.use_graphs) {
        cudaGraphExec_t &ge = b->graph[b->cur];
        if (!ge) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return e;
            cudaError_t r = issue();
            e = cudaStreamEndCapture(b->stream, &graph);
            if (r != cudaSuccess) e = r;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                ge = nullptr;
                return e;
            }
        }
        e = cudaGraphLaunch(ge, b->stream);
    } else {
        e = issue();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < b->S; ++s) {
        if (b->slot_left[s] <= 0) continue;
        if (b->slot_left[s] <= b->K) {
            Job *j = b->slot_job[s];
            j->parity = (b->cur + b->slot_left[s]) & 1;
            b->slot_left[s] = 0;
        } else {
            b->slot_left[s] -= b->K;
        }
    }
    b->cur = (b->cur + b->K) & 1;
    b->launched = true;
    return cudaSuccess;
}

void retire(tls_ctx *ctx, Server *sv, Batch *b)
{
    const Gauge &gg = ctx->gauges.at(b->key.gauge);
    for (int s = 0; s < b->S; ++s) {
        Job *j = b->slot_job[s];
        if (!j || s != j->slot0) continue;
        bool fin = true;
        for (int k = s; k < s + j->d.nvec; ++k) fin = fin && b->slot_left[k] == 0;
        if (!fin || j->parity < 0) continue;
        const int64_t Vslice = (int64_t)gg.L[0] * gg.L[1] * gg.L[2];
        const int64_t V = Vslice * gg.L[3];
        const size_t slice_b = (size_t)Vslice * 6 * io_elem(j->d.io_prec);
        cudaError_t e;
        if (j->d.vecs_on_device) {
            e = launch_unpack_il(b->buf[j->parity], b->key.storage, j->d.vecs, j->d.io_prec, V, gg.g, gg.L, b->t_first,
                                 b->nsl, j->d.nvec, b->S, s, b->stream);
        } else {
            e = launch_unpack_il(b->buf[j->parity], b->key.storage, j->staging, j->d.io_prec, Vslice * b->nsl, gg.g,
                                 gg.L, 0, b->nsl, j->d.nvec, b->S, s, b->stream);
            const size_t width = slice_b * b->nsl, pitch = (size_t)V * 6 * io_elem(j->d.io_prec);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync((char *)j->d.vecs + (size_t)b->t_first * slice_b, pitch, j->staging, width,
                                      width, j->d.nvec, cudaMemcpyDeviceToHost, b->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (j->staging) {
            dev_free(ctx, j->staging, j->staging_bytes);
            j->staging = nullptr;
        }
        for (int k = s; k < s + j->d.nvec; ++k) {
            b->slot_job[k] = nullptr;
            b->slot_left[k] = 0;
        }
        finish(sv, j, e == cudaSuccess ? TLS_OK : cuda_fail(e, "serve: unpack"));
    }
}

void fail_batch(tls_ctx *ctx, Server *sv, Batch *b, tls_status st)
{
    for (int s = 0; s < b->S; ++s) {
        Job *j = b->slot_job[s];
        if (j && s == j->slot0) {
            if (j->staging) dev_free(ctx, j->staging, j->staging_bytes);
            j->staging = nullptr;
            finish(sv, j, st);
        }
        b->slot_job[s] = nullptr;
        b->slot_left[s] = 0;
    }
}

void scheduler(tls_ctx *ctx, Server *sv)
{
    cudaSetDevice(ctx->device);
    for (;;) {
        std::vector<Job *> waiting;
        {
            std::unique_lock<std::mutex> lk(sv->m);
            if (!sv->stop && sv->pending.empty() && !any_busy(sv))
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            if (sv->stop) break;
            waiting.assign(sv->pending.begin(), sv->pending.end());
            sv->pending.clear();
        }
        std::vector<Batch *> running;
        {
            std::lock_guard<FairMutex> g(ctx->mu);
            std::vector<Job *> keep;
            for (Job *j : waiting)
                if (try_admit(ctx, sv, j)) keep.push_back(j);
            if (!keep.empty()) {
                std::lock_guard<std::mutex> lk(sv->m);
                sv->pending.insert(sv->pending.begin(), keep.begin(), keep.end());
            }
            for (auto &kv : sv->batches) {
                Batch *b = kv.second.get();
                if (b->used_slots() == 0) continue;
                if (b->active_slots() > 0) {
                    cudaError_t e = launch_round(ctx, sv, b);
                    if (e != cudaSuccess) {
                        fail_batch(ctx, sv, b, cuda_fail(e, "serve: round"));
                        continue;
                    }
                }
                running.push_back(b);
            }
        }
        // Wait for the device without holding the context lock: other host
        // threads may call into the library meanwhile.  Batches with slots in
        // use are never destroyed outside this thread.
        std::vector<cudaError_t> status(running.size());
        for (size_t k = 0; k < running.size(); ++k) status[k] = cudaStreamSynchronize(running[k]->stream);
        {
            std::lock_guard<FairMutex> g(ctx->mu);
            for (size_t k = 0; k < running.size(); ++k) {
                if (status[k] != cudaSuccess) {
                    fail_batch(ctx, sv, running[k], cuda_fail(status[k], "serve: round"));
                    continue;
                }
                if (*running[k]->h_err) {  // a bounded device wait ran out: the batch's results are void
                    const int herr = *running[k]->h_err;
                    *running[k]->h_err = 0;
                    cudaMemsetAsync(running[k]->d_err, 0, sizeof(int), running[k]->stream);
                    fail_batch(ctx, sv, running[k],
                               fail((herr & DERR_TIMEOUT) ? TLS_ERR_TIMEOUT : TLS_ERR_DEVICE,
                                    "serve: device error word 0x%x", herr));
                    continue;
                }
                retire(ctx, sv, running[k]);
            }
        }
    }
}

}  // namespace

void serve_shutdown(tls_ctx *ctx)
{
    Server *sv = ctx->server;
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->m);
        sv->stop = true;
        sv->cv_work.notify_all();
    }
    if (sv->th.joinable()) sv->th.join();
    std::lock_guard<FairMutex> g(ctx->mu);
    for (auto &kv : sv->batches) {
        fail_batch(ctx, sv, kv.second.get(), fail(TLS_ERR_STATE, "serve: stopped"));
        destroy_batch(ctx, kv.second.get());
    }
    sv->batches.clear();
    for (Job *j : sv->pending) finish(sv, j, fail(TLS_ERR_STATE, "serve: stopped before admission"));
    sv->pending.clear();
    delete sv;
    ctx->server = nullptr;
}

bool serve_gauge_busy(tls_ctx *ctx, int64_t id)
{
    Server *sv = ctx->server;
    if (!sv) return false;
    // The caller holds ctx->mu, so the scheduler is not admitting or launching;
    // sv->m keeps its idle check (any_busy) off the map while it changes.
    std::lock_guard<std::mutex> lk(sv->m);
    for (Job *j : sv->pending)
        if (j->d.gauge == id) return true;
    for (auto it = sv->batches.begin(); it != sv->batches.end();) {
        Batch *b = it->second.get();
        if (b->key.gauge == id) {
            if (b->used_slots() > 0) return true;
            destroy_batch(ctx, b);
            it = sv->batches.erase(it);
        } else {
            ++it;
        }
    }
    return false;
}

}  // namespace tls

using namespace tls;

extern "C" {

tls_status tls_serve_start(tls_ctx *ctx, const tls_serve_opts *opts)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_serve_start: ctx is NULL");
    std::lock_guard<FairMutex> g(ctx->mu);
    if (ctx->server) return fail(TLS_ERR_STATE, "tls_serve_start: already serving");
    std::unique_ptr<Server> sv(new Server());
    sv->opts.max_slots = 64;
    sv->opts.steps_per_launch = 1;
    sv->opts.use_graphs = 1;
    if (opts) sv->opts = *opts;
    if (sv->opts.max_slots < 1 || sv->opts.max_slots > 256)
        return fail(TLS_ERR_ARG, "tls_serve_start: max_slots %d outside [1, 256]", sv->opts.max_slots);
    if (sv->opts.steps_per_launch < 1 || sv->opts.steps_per_launch > 1024)
        return fail(TLS_ERR_ARG, "tls_serve_start: steps_per_launch %d", sv->opts.steps_per_launch);
    sv->t0 = Clock::now();
    Server *raw = sv.release();
    ctx->server = raw;
    raw->th = std::thread(scheduler, ctx, raw);
    return ok();
}

tls_status tls_serve_stop(tls_ctx *ctx)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_serve_stop: ctx is NULL");
    if (!ctx->server) return fail(TLS_ERR_STATE, "tls_serve_stop: not serving");
    serve_shutdown(ctx);
    return ok();
}

tls_status tls_serve_submit(tls_ctx *ctx, const tls_job *job, uint64_t *job_id)
{
    if (!ctx || !job || !job_id) return fail(TLS_ERR_ARG, "tls_serve_submit: NULL argument");
    Server *sv = ctx->server;
    if (!sv) return fail(TLS_ERR_STATE, "tls_serve_submit: not serving");
    if (!job->vecs || job->nvec < 1 || job->N < 0 || (job->io_prec != TLS_F64 && job->io_prec != TLS_F32))
        return fail(TLS_ERR_ARG, "tls_serve_submit: bad job (vecs, nvec, N or io_prec)");
    if (job->storage != TLS_F32 && job->storage != TLS_F16 && job->storage != TLS_BF16 && job->storage != TLS_F64)
        return fail(TLS_ERR_ARG, "tls_serve_submit: storage %d", job->storage);
    if (job->nvec > sv->opts.max_slots)
        return fail(TLS_ERR_ARG, "tls_serve_submit: nvec %d exceeds max_slots %d", job->nvec, sv->opts.max_slots);
    {
        std::lock_guard<FairMutex> g(ctx->mu);
        auto it = ctx->gauges.find(job->gauge);
        if (it == ctx->gauges.end()) return fail(TLS_ERR_NOT_FOUND, "tls_serve_submit: unknown gauge");
        const Gauge &gg = it->second;
        if (!gg.built) return fail(TLS_ERR_NOT_BUILT, "tls_serve_submit: W not built");
        if (job->timeslice < TLS_ALL_T || job->timeslice >= gg.L[3])
            return fail(TLS_ERR_ARG, "tls_serve_submit: timeslice %d", job->timeslice);
        tls_status s = check_smear_combo(gg, job->storage);
        if (s != TLS_OK) return s;
        if (ctx->cap) {
            size_t need = batch_bytes(gg, job->storage, job->timeslice, sv->opts.max_slots, sv->opts.steps_per_launch);
            if (!job->vecs_on_device) {
                const int nsl = job->timeslice < 0 ? gg.L[3] : 1;
                need += (size_t)gg.L[0] * gg.L[1] * gg.L[2] * nsl * 6 * io_elem(job->io_prec) * job->nvec;
            }
            size_t resident = 0;
            for (auto &kv : ctx->gauges) resident += kv.second.W_bytes + kv.second.Up_bytes;
            if (resident + need > ctx->cap)
                return fail(TLS_ERR_ADMIT, "tls_serve_submit: the job needs %zu bytes beside %zu resident; cap %llu",
                            need, resident, (unsigned long long)ctx->cap);
        }
    }
    std::unique_ptr<Job> j(new Job());
    j->d = *job;
    {
        std::lock_guard<std::mutex> lk(sv->m);
        j->id = sv->next_id++;
        j->submit_ms = sv->now_ms();
        *job_id = j->id;
        sv->pending.push_back(j.get());
        sv->jobs[j->id] = std::move(j);
        sv->cv_work.notify_all();
    }
    return ok();
}

tls_status tls_serve_poll(tls_ctx *ctx, uint64_t job_id, int *done)
{
    if (!ctx || !done) return fail(TLS_ERR_ARG, "tls_serve_poll: NULL argument");
    Server *sv = ctx->server;
    if (!sv) return fail(TLS_ERR_STATE, "tls_serve_poll: not serving");
    std::lock_guard<std::mutex> lk(sv->m);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) return fail(TLS_ERR_NOT_FOUND, "tls_serve_poll: unknown job %llu", (unsigned long long)job_id);
    *done = it->second->done ? 1 : 0;
    return ok();
}

tls_status tls_serve_wait(tls_ctx *ctx, uint64_t job_id, double timeout_s, tls_job_result *result)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_serve_wait: ctx is NULL");
    Server *sv = ctx->server;
    if (!sv) return fail(TLS_ERR_STATE, "tls_serve_wait: not serving");
    std::unique_lock<std::mutex> lk(sv->m);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) return fail(TLS_ERR_NOT_FOUND, "tls_serve_wait: unknown job %llu", (unsigned long long)job_id);
    Job *j = it->second.get();
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (!j->done) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !j->done)
            return fail(TLS_ERR_TIMEOUT, "tls_serve_wait: job %llu not finished after %.3f s",
                        (unsigned long long)job_id, timeout_s);
    }
    if (result) {
        result->status = j->status;
        result->submit_ms = j->submit_ms;
        result->start_ms = j->start_ms;
        result->done_ms = j->done_ms;
    }
    const tls_status st = j->status;
    sv->jobs.erase(it);
    if (st != TLS_OK) return fail(st, "tls_serve_wait: job %llu failed with status %d", (unsigned long long)job_id, st);
    return ok();
}

}  // extern "C"
