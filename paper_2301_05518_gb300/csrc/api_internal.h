// api_internal.h -- the context object behind the C ABI (shared by api.cu and serve.cpp).
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tls.h"
#include "tls_internal.h"

namespace tls {

struct Server;

// Recursive mutex that grants the lock in arrival order (ticket lock), so a
// host thread calling into the library is not starved by the serving
// scheduler re-taking the lock round after round.
class FairMutex {
  public:
    void lock()
    {
        std::unique_lock<std::mutex> lk(m_);
        if (depth_ > 0 && owner_ == std::this_thread::get_id()) {
            ++depth_;
            return;
        }
        const uint64_t ticket = next_++;
        cv_.wait(lk, [&] { return serving_ == ticket && depth_ == 0; });
        owner_ = std::this_thread::get_id();
        depth_ = 1;
    }
    void unlock()
    {
        std::unique_lock<std::mutex> lk(m_);
        if (--depth_ == 0) {
            owner_ = std::thread::id();
            ++serving_;
            cv_.notify_all();
        }
    }

  private:
    std::mutex m_;
    std::condition_variable cv_;
    uint64_t next_ = 0, serving_ = 0;
    std::thread::id owner_;
    int depth_ = 0;
};

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
};

struct Gauge {
    int L[4] = {0, 0, 0, 0};
    SubGeom g{};
    double *Up = nullptr;  // packed spatial links, FP64
    size_t Up_bytes = 0;
    char *W = nullptr;     // packed two-link field
    size_t W_bytes = 0;
    int wfmt = -1;
    bool built = false;
    char *L1 = nullptr;    // one-link field (Eq. 2 links, rounded), W planes
    size_t L1_bytes = 0;
    int l1fmt = -1;
};

// Best kernel per problem shape, filled by tls_autotune-style measurement.
struct TuneKey {
    int L[4];
    int nsl, nvec, storage, wfmt;
    bool operator<(const TuneKey &o) const
    {
        const int a[] = {L[0], L[1], L[2], L[3], nsl, nvec, storage, wfmt};
        const int b[] = {o.L[0], o.L[1], o.L[2], o.L[3], o.nsl, o.nvec, o.storage, o.wfmt};
        for (int k = 0; k < 8; ++k)
            if (a[k] != b[k]) return a[k] < b[k];
        return false;
    }
};
struct TuneVal {
    int kernel, vb, threads;
    int tile[3];
    double ms;
};

}  // namespace tls

struct tls_ctx {
    int device = 0;
    int num_sms = 0;
    int max_smem = 0;                       // opt-in shared memory per CTA (bytes)
    uint64_t cap = 0;                       // 0 = no cap
    std::atomic<uint64_t> used{0};
    tls::FairMutex mu;                      // serialises device work on this context
    std::map<int64_t, tls::Gauge> gauges;
    int64_t next_id = 1;

    // smear workspace (grown on demand)
    tls::DevBuf A, B, S0, S1, staging, alpha, partials, norms;
    double *h_alpha = nullptr;              // pinned
    size_t h_alpha_n = 0;
    double *h_norms = nullptr;              // pinned
    int *h_err = nullptr;                   // pinned copy of the error word
    size_t h_norms_n = 0;
    int *d_err = nullptr;                   // device error word
    unsigned *d_bar = nullptr;              // barrier words (count, generation)
    long long barrier_budget = 0;           // 0 = default

    bool profiling = false;
    tls_profile prof{};
    cudaEvent_t ev[8] = {};
    std::vector<cudaEvent_t> evp;           // timing events of one smear call (grown on demand)

    // host-buffer pipeline: copies in / out on their own streams, ordered by events
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t e_in[3] = {}, e_done[3] = {}, e_out[3] = {}, e_sync[2] = {};

    std::map<tls::TuneKey, tls::TuneVal> tune;

    tls::Server *server = nullptr;
};

namespace tls {

// Thread-local error message and status helpers.
tls_status fail(tls_status code, const char *fmt, ...);
tls_status ok();
tls_status cuda_fail(cudaError_t e, const char *what);

// Device memory under the context's cap.
tls_status dev_alloc(tls_ctx *ctx, void **p, size_t bytes, const char *what);
void dev_free(tls_ctx *ctx, void *p, size_t bytes);
tls_status ensure(tls_ctx *ctx, DevBuf &b, size_t bytes, const char *what);
void release(tls_ctx *ctx, DevBuf &b);

// Shared argument checks for smearing (tls_smear and serving).
tls_status check_smear_combo(const Gauge &gg, int storage);
int default_vb(int storage, int nvec);
// Vectors per thread of the interleaved multi-RHS kernel (a divisor of nvec).
int default_il_vb(int storage, int nvec);

// tls_smear with an optional forced vectors-per-thread / threads / tile (0 = planner's choice).
// op = 0: two-link smearing (Eq. tlSmear, width = sigma); op = 1: one-link Gaussian
// smearing (Eq. 3 with C = 1, width = alpha) on the link field.
tls_status smear_impl(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int vecs_on_device, int nvec, int N,
                      double width, int timeslice, int storage, int kernel, int force_vb, int force_threads,
                      const int *force_tile, void *stream, double *norms_out, int op = 0);

// The serving subsystem (serve.cpp).
void serve_shutdown(tls_ctx *ctx);
// True if serving still holds jobs on gauge `id`; otherwise drops its idle batches.
bool serve_gauge_busy(tls_ctx *ctx, int64_t id);

}  // namespace tls
