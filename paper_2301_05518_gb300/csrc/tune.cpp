// tune.cpp -- autotuner for the smearing kernels (tls_autotune, tls_tune_set).
//
// For one problem shape (lattice, slice selection, vector count, storage and
// W format) it times each candidate kernel over a few steps with CUDA events
// on the context's launch stream and records the fastest; TLS_KERNEL_AUTO
// then uses it.  Candidates: the one-vector-per-launch kernel (up to four
// vectors) and the multi-right-hand-side kernels that won at some measured
// shape, at several vectors per thread and CTA shapes.
#include <algorithm>
#include <cstring>

#include "api_internal.h"

namespace tls {

namespace {

struct Cand {
    int kernel, vb, threads;
    int tile[3];
};

std::vector<Cand> candidates(int nvec, int storage)
{
    // The kernels that won at some measured shape.  Measured and dropped (they
    // never won at any benchmarked shape): the register-capped and W-staged
    // interleaved variants, explicit strip lengths, eight vectors per thread in
    // the packed kernel, the TMA row kernel, the z-marching kernel and both
    // persistent forms (tls_smear still runs any of them when asked for).
    std::vector<Cand> c;
    if (nvec <= 4) {
        c.push_back({TLS_KERNEL_SINGLE, 1, 128, {0, 0, 0}});
        c.push_back({TLS_KERNEL_SINGLE, 1, 256, {0, 0, 0}});
    }
    const int G = std::min(nvec, 256);
    const int G2 = storage != TLS_F64 ? (G + 1) & ~1 : G;  // FP32 and 16-bit records come in vector pairs
    for (int vb : {1, 2, 4}) {
        if (G2 % vb != 0 || (storage == TLS_F64 && vb > 2)) continue;
        if (storage == TLS_F64) {
            for (int t : {128, 256}) c.push_back({TLS_KERNEL_MRHS, vb, t, {0, 0, 0}});
            c.push_back({TLS_KERNEL_MRHS, vb, 128, {0, 1, 0}});  // W of the strip staged in shared memory
            continue;
        }
        if (vb == 1 && G2 >= 8) continue;
        // whole rows with the W rows staged by TMA: all vectors or half of them per CTA
        c.push_back({TLS_KERNEL_MRHS, vb, 0, {0, 6, 0}});
        c.push_back({TLS_KERNEL_MRHS, vb, 0, {0, 6, -1}});  // rows ahead requested into L2
        c.push_back({TLS_KERNEL_MRHS, vb, 0, {0, 7, 0}});
        if (vb % 2 == 0) c.push_back({TLS_KERNEL_MRHS, vb, 0, {0, 8, 0}});  // the row's records staged too
        // fewer vectors per CTA: smaller CTAs, W staged once per group (each
        // distinct count once)
        int tried[3], ntried = 0;
        for (int ng : {G2 / 2, 24, 12}) {
            if (ng >= G2 || ng < 2 * vb || ng % vb != 0 || G2 % ng != 0) continue;
            if (std::find(tried, tried + ntried, ng) != tried + ntried) continue;
            tried[ntried++] = ng;
            c.push_back({TLS_KERNEL_MRHS, vb, 0, {ng, 6, 0}});
        }
        // packed FP32 pairs with the W broadcasts staged by the threads (any row length)
        c.push_back({TLS_KERNEL_MRHS, vb, 128, {0, 2, 0}});
    }
    if (storage == TLS_F32 && G2 % 8 == 0) {  // eight FP32 vectors per thread, one colour at a time
        c.push_back({TLS_KERNEL_MRHS, 8, 0, {0, 6, 0}});
        c.push_back({TLS_KERNEL_MRHS, 8, 0, {0, 7, 0}});
        c.push_back({TLS_KERNEL_MRHS, 8, 0, {0, 7, -1}});
    }
    return c;
}

}  // namespace

}  // namespace tls

using namespace tls;

extern "C" {

tls_status tls_tune_set(tls_ctx *ctx, tls_gauge_id id, int nvec, int storage, int timeslice,
                        const tls_tune_entry *entry)
{
    if (!ctx || !entry) return fail(TLS_ERR_ARG, "tls_tune_set: NULL argument");
    if (entry->kernel < TLS_KERNEL_SINGLE || entry->kernel > TLS_KERNEL_MRHS_ZM)
        return fail(TLS_ERR_ARG, "tls_tune_set: kernel %d", entry->kernel);
    std::lock_guard<FairMutex> lk(ctx->mu);
    auto it = ctx->gauges.find(id);
    if (it == ctx->gauges.end()) return fail(TLS_ERR_NOT_FOUND, "tls_tune_set: unknown gauge");
    const Gauge &gg = it->second;
    if (!gg.built) return fail(TLS_ERR_NOT_BUILT, "tls_tune_set: W not built");
    const int nsl = timeslice < 0 ? gg.L[3] : 1;
    TuneKey key{{gg.L[0], gg.L[1], gg.L[2], gg.L[3]}, nsl, nvec, storage, gg.wfmt};
    ctx->tune[key] = TuneVal{entry->kernel, entry->vecs_per_thread, entry->threads,
                             {entry->tile[0], entry->tile[1], entry->tile[2]}, entry->ms_per_step};
    return ok();
}

tls_status tls_autotune(tls_ctx *ctx, tls_gauge_id id, int nvec, int storage, int timeslice, int steps,
                        tls_tune_entry *best, tls_tune_entry *all, int max_all, int *n_all)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_autotune: ctx is NULL");
    if (nvec < 1 || steps < 1) return fail(TLS_ERR_ARG, "tls_autotune: nvec %d, steps %d", nvec, steps);
    std::lock_guard<FairMutex> lk(ctx->mu);
    auto it = ctx->gauges.find(id);
    if (it == ctx->gauges.end()) return fail(TLS_ERR_NOT_FOUND, "tls_autotune: unknown gauge");
    const Gauge gg = it->second;
    if (!gg.built) return fail(TLS_ERR_NOT_BUILT, "tls_autotune: W not built");
    tls_status s = check_smear_combo(gg, storage);
    if (s != TLS_OK) return s;
    cudaSetDevice(ctx->device);
    const int nsl = timeslice < 0 ? gg.L[3] : 1;
    const int64_t Vslice = (int64_t)gg.L[0] * gg.L[1] * gg.L[2];
    const int io = storage == TLS_F64 ? TLS_F64 : TLS_F32;
    const size_t bytes = (size_t)nvec * gg.L[3] * Vslice * 6 * (io == TLS_F64 ? 8 : 4);
    void *tmp = nullptr;
    s = dev_alloc(ctx, &tmp, bytes, "tls_autotune: scratch vectors");
    if (s != TLS_OK) return s;
    cudaMemset(tmp, 0, bytes);
    const bool was = ctx->profiling;
    ctx->profiling = true;
    TuneVal win{0, 0, 0, {0, 0, 0}, 1e300};
    int n = 0;
    for (const Cand &c : candidates(nvec, storage)) {
        // one warm-up call, then the timed one
        s = smear_impl(ctx, id, tmp, io, 1, nvec, 1, 0.5, timeslice, storage, c.kernel, c.vb, c.threads, c.tile,
                       nullptr, nullptr);
        if (s == TLS_OK)
            s = smear_impl(ctx, id, tmp, io, 1, nvec, steps, 0.5 * steps, timeslice, storage, c.kernel, c.vb,
                           c.threads, c.tile, nullptr, nullptr);
        if (s != TLS_OK) {
            if (s == TLS_ERR_UNSUPPORTED) continue;
            break;
        }
        const double ms = ctx->prof.ms_iter / steps;
        if (all && n < max_all) all[n] = tls_tune_entry{c.kernel, c.vb, c.threads, {c.tile[0], c.tile[1], c.tile[2]}, ms};
        ++n;
        if (ms < win.ms) win = TuneVal{c.kernel, c.vb, c.threads, {c.tile[0], c.tile[1], c.tile[2]}, ms};
    }
    ctx->profiling = was;
    dev_free(ctx, tmp, bytes);
    if (s != TLS_OK && s != TLS_ERR_UNSUPPORTED) return s;
    if (win.kernel == 0) return fail(TLS_ERR_UNSUPPORTED, "tls_autotune: no candidate ran");
    TuneKey key{{gg.L[0], gg.L[1], gg.L[2], gg.L[3]}, nsl, nvec, storage, gg.wfmt};
    ctx->tune[key] = win;
    if (best) *best = tls_tune_entry{win.kernel, win.vb, win.threads, {win.tile[0], win.tile[1], win.tile[2]}, win.ms};
    if (n_all) *n_all = n;
    return ok();
}

}  // extern "C"
