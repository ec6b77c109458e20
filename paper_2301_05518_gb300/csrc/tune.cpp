// tune.cpp -- autotuner for the smearing kernels (tls_autotune, tls_tune_set).
//
// For one problem shape (lattice, slice selection, vector count, storage and
// W format) it times each candidate kernel over a few steps with CUDA events
// on the context's launch stream and records the fastest; TLS_KERNEL_AUTO
// then uses it.  Candidates: the one-vector-per-launch kernel, the
// interleaved multi-RHS kernel at several CTA sizes, and the persistent
// kernel at several vectors-per-thread.
#include <algorithm>
#include <cstring>

#include "api_internal.h"

namespace tls {

namespace {

struct Cand {
    int kernel, vb, threads;
    int tile[3];
};

std::vector<Cand> candidates(int nvec, int storage, bool rows, bool onchip)
{
    std::vector<Cand> c;
    if (nvec <= 4) {
        c.push_back({TLS_KERNEL_SINGLE, 1, 128, {0, 0, 0}});
        c.push_back({TLS_KERNEL_SINGLE, 1, 256, {0, 0, 0}});
    }
    const int G = std::min(nvec, 256);
    for (int vb : {1, 2, 4}) {
        if (G % vb != 0 || (storage == TLS_F64 && vb > 2)) continue;
        const int tx = G / vb;
        for (int t : {64, 128, 256})
            if (t >= tx || t == 256) c.push_back({TLS_KERNEL_MRHS, vb, t, {0, 0, 0}});
        if (tx <= 128) c.push_back({TLS_KERNEL_MRHS, vb, -128, {0, 0, 0}});
        for (int t : {128, 256})  // W of the strip staged in shared memory
            if (t >= tx) c.push_back({TLS_KERNEL_MRHS, vb, t, {0, 1, 0}});
        if (storage != TLS_F64)  // packed FP32 pairs with broadcast W in shared memory
            for (int t : {128, 256})
                if (t >= tx) {
                    c.push_back({TLS_KERNEL_MRHS, vb, t, {0, 2, 0}});
                    c.push_back({TLS_KERNEL_MRHS, vb, t, {0, 4, 0}});  // W as stored, packed FMAs
                }
        if (storage != TLS_F64 && tx <= 96)  // packed kernel, register-capped CTAs of <= 96 threads
            c.push_back({TLS_KERNEL_MRHS, vb, 96, {0, 5, 0}});
        if (storage != TLS_F64)  // packed kernel with explicit strip lengths
            for (int spb : {4, 8, 32})
                if (spb * tx <= 256) c.push_back({TLS_KERNEL_MRHS, vb, 256, {spb, 2, 0}});
        if (rows) c.push_back({TLS_KERNEL_MRHS_ROWS, vb, 0, {0, 0, 0}});
    }
    if (storage == TLS_F32 && G % 8 == 0)  // eight FP32 vectors per thread, packed kernel
        for (int t : {128, 256})
            if (t >= G / 8) c.push_back({TLS_KERNEL_MRHS, 8, t, {0, 2, 0}});
    const int vmax = storage == TLS_F64 ? 4 : 8;
    for (int vb : {1, 4, 8})
        if (vb <= vmax && (vb == 1 || vb <= 2 * nvec))
            for (int mb : {48, 96})  // L2 budget of one group of blocks (MB)
                c.push_back({TLS_KERNEL_PERSISTENT, vb, 256, {mb, 0, 0}});
    if (onchip)  // every block's W and iterates in one CTA's shared memory
        for (int vb : {1, 4})
            if (vb <= vmax)
                for (int t : {512, 1024}) c.push_back({TLS_KERNEL_PERSISTENT, vb, t, {0, 1, 0}});
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
    const int G = std::min(nvec, 256);
    const bool rows = storage != TLS_F64 && rows_applicable(gg.wfmt, storage, gg.g, G, 1, ctx->max_smem);
    int nvg = 0, smem = 0;
    const bool onchip = onchip_plan(gg.g, wfmt_bytes(gg.wfmt), storage == TLS_F64 ? 48 : 24, nvec, ctx->max_smem,
                                    &nvg, &smem);
    for (const Cand &c : candidates(nvec, storage, rows, onchip)) {
        if (c.kernel == TLS_KERNEL_MRHS_ROWS && !rows_applicable(gg.wfmt, storage, gg.g, G, c.vb, ctx->max_smem))
            continue;
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
