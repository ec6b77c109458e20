// api.cu -- the C ABI (include/tls.h): context, gauge fields, two-link build, smearing.
//
// The hot path of the paper (Sec. 2-3): W_i(x) = U_i(x) U_i(x+i) is built once
// per gauge field and kept resident; each smearing call applies N steps of
// psi <- psi + (sigma/(4N)) Delta psi (Eq. tlSmear with Eq. tlLapl1) to a
// batch of vectors.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "api_internal.h"

namespace tls {

static thread_local std::string g_err;

tls_status fail(tls_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

tls_status ok()
{
    g_err.clear();
    return TLS_OK;
}

tls_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? TLS_ERR_NOMEM : TLS_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

tls_status dev_alloc(tls_ctx *ctx, void **p, size_t bytes, const char *what)
{
    *p = nullptr;
    if (bytes == 0) return TLS_OK;
    if (ctx->cap && ctx->used.load() + bytes > ctx->cap)
        return fail(TLS_ERR_ADMIT, "%s: %zu bytes would exceed the HBM cap (%llu in use of %llu)", what, bytes,
                    (unsigned long long)ctx->used.load(), (unsigned long long)ctx->cap);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(TLS_ERR_NOMEM, "%s: cudaMalloc(%zu) failed: %s", what, bytes, cudaGetErrorString(e));
    }
    ctx->used += bytes;
    return TLS_OK;
}

void dev_free(tls_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    ctx->used -= bytes;
}

tls_status ensure(tls_ctx *ctx, DevBuf &b, size_t bytes, const char *what)
{
    if (b.n >= bytes) return TLS_OK;
    release(ctx, b);
    tls_status s = dev_alloc(ctx, &b.p, bytes, what);
    if (s != TLS_OK) return s;
    b.n = bytes;
    cudaError_t e = cudaMemset(b.p, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return TLS_OK;
}

void release(tls_ctx *ctx, DevBuf &b)
{
    dev_free(ctx, b.p, b.n);
    b.p = nullptr;
    b.n = 0;
}

static int wfmt_of(int prec, int recon)
{
    if (prec == TLS_F64 && recon == TLS_R18) return W_F64_18;
    if (prec == TLS_F32) return recon == TLS_R18 ? W_F32_18 : recon == TLS_R12 ? W_F32_12 : recon == TLS_R8 ? W_F32_8 : -1;
    if (prec == TLS_F16) return recon == TLS_R18 ? W_F16_18 : recon == TLS_R12 ? W_F16_12 : -1;
    if (prec == TLS_BF16) return recon == TLS_R18 ? W_BF16_18 : recon == TLS_R12 ? W_BF16_12 : -1;
    return -1;
}

tls_status check_smear_combo(const Gauge &gg, int storage)
{
    const int wf = gg.wfmt;
    bool okc = false;
    switch (storage) {
    case TLS_F64: okc = wf == W_F64_18; break;
    case TLS_F32: okc = wf == W_F32_18 || wf == W_F32_12 || wf == W_F32_8; break;
    case TLS_F16: okc = wf == W_F32_18 || wf == W_F32_12 || wf == W_F16_18 || wf == W_F16_12; break;
    case TLS_BF16: okc = wf == W_F32_18 || wf == W_F32_12 || wf == W_BF16_18 || wf == W_BF16_12; break;
    default: return fail(TLS_ERR_ARG, "storage precision %d is not a TLS_F* value", storage);
    }
    if (!okc)
        return fail(TLS_ERR_UNSUPPORTED, "vector storage %d cannot run with the W format of this gauge (format %d)",
                    storage, wf);
    return TLS_OK;
}

int default_vb(int storage, int nvec)
{
    const int cap = storage == TLS_F64 ? 4 : 8;
    int vb = 1;
    while (vb < cap && vb < nvec) vb *= 2;
    return vb;
}

int default_il_vb(int storage, int nvec)
{
    const int cap = storage == TLS_F64 ? 2 : 4;
    for (int vb = cap; vb > 1; vb /= 2)
        if (nvec % vb == 0) return vb;
    return 1;
}

cudaError_t launch_step(const StepArgs &a)
{
    switch (a.prec_in) {
    case P_F64: return launch_step_f64(a);
    case P_F32: return launch_step_f32(a);
    case P_F16: return launch_step_f16(a);
    case P_BF16: return launch_step_bf16(a);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_step_il(const StepArgs &a)
{
    switch (a.prec_in) {
    case P_F64: return launch_step_il_f64(a);
    case P_F32: return launch_step_il_f32(a);
    case P_F16: return launch_step_il_f16(a);
    case P_BF16: return launch_step_il_bf16(a);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_hop(const StepArgs &a)
{
    switch (a.prec_in) {
    case P_F64: return launch_hop_f64(a);
    case P_F32: return launch_hop_f32(a);
    case P_F16: return launch_hop_f16(a);
    case P_BF16: return launch_hop_bf16(a);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_step_zm(const StepArgs &a)
{
    switch (a.prec_in) {
    case P_F64: return launch_step_zm_f64(a);
    case P_F32: return launch_step_zm_f32(a);
    case P_F16: return launch_step_zm_f16(a);
    case P_BF16: return launch_step_zm_bf16(a);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_step_rows(const StepArgs &a, int *err)
{
    switch (a.prec_in) {
    case P_F32: return launch_step_rows_f32(a, err);
    case P_F16: return launch_step_rows_f16(a, err);
    case P_BF16: return launch_step_rows_bf16(a, err);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_persistent(const PersistArgs &a)
{
    switch (a.prec) {
    case P_F64: return launch_persistent_f64(a);
    case P_F32: return launch_persistent_f32(a);
    case P_F16: return launch_persistent_f16(a);
    case P_BF16: return launch_persistent_bf16(a);
    default: return cudaErrorNotSupported;
    }
}

int persistent_occupancy(int wfmt, int prec, int, int vb, int threads)
{
    switch (prec) {
    case P_F64: return persistent_occupancy_f64(wfmt, vb, threads);
    case P_F32: return persistent_occupancy_f32(wfmt, vb, threads);
    case P_F16: return persistent_occupancy_f16(wfmt, vb, threads);
    case P_BF16: return persistent_occupancy_bf16(wfmt, vb, threads);
    default: return 0;
    }
}

static void free_gauge(tls_ctx *ctx, Gauge &gg)
{
    dev_free(ctx, gg.Up, gg.Up_bytes);
    dev_free(ctx, gg.W, gg.W_bytes);
    dev_free(ctx, gg.L1, gg.L1_bytes);
    gg.Up = nullptr;
    gg.W = nullptr;
    gg.L1 = nullptr;
    gg.Up_bytes = gg.W_bytes = gg.L1_bytes = 0;
    gg.built = false;
    gg.l1fmt = -1;
}

static Gauge *find_gauge(tls_ctx *ctx, tls_gauge_id id)
{
    auto it = ctx->gauges.find(id);
    return it == ctx->gauges.end() ? nullptr : &it->second;
}

static const long long kDefaultBudget = 20000000LL;  // polls of ~64 ns: about a second or more

}  // namespace tls

using namespace tls;

extern "C" {

int tls_version(void) { return 10000; }

const char *tls_last_error(void) { return g_err.c_str(); }

uint64_t tls_bytes_in_use(const tls_ctx *ctx) { return ctx ? ctx->used.load() : 0; }

tls_status tls_create(tls_ctx **out, int device, uint64_t hbm_cap_bytes)
{
    if (!out) return fail(TLS_ERR_ARG, "tls_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "tls_create: cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(TLS_ERR_ARG, "tls_create: device %d of %d", device, ndev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "tls_create: cudaSetDevice");
    std::unique_ptr<tls_ctx> ctx(new tls_ctx());
    ctx->device = device;
    ctx->cap = hbm_cap_bytes;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    tls_status s = dev_alloc(ctx.get(), (void **)&ctx->d_err, 256, "tls_create: error word");
    if (s != TLS_OK) return s;
    s = dev_alloc(ctx.get(), (void **)&ctx->d_bar, 256, "tls_create: barrier words");
    if (s != TLS_OK) {
        dev_free(ctx.get(), ctx->d_err, 256);
        return s;
    }
    cudaMemset(ctx->d_err, 0, 256);
    cudaMemset(ctx->d_bar, 0, 256);
    e = cudaMallocHost(&ctx->h_err, 256);
    if (e != cudaSuccess) return cuda_fail(e, "tls_create: pinned error word");
    for (auto &ev : ctx->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e, "tls_create: cudaEventCreate");
    }
    e = cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&ctx->e_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->e_done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->e_out[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->e_sync[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->e_sync[1], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "tls_create: copy streams and events");
    *out = ctx.release();
    return ok();
}

void tls_destroy(tls_ctx *ctx)
{
    if (!ctx) return;
    serve_shutdown(ctx);
    {
        std::lock_guard<FairMutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        for (auto &kv : ctx->gauges) free_gauge(ctx, kv.second);
        ctx->gauges.clear();
        for (DevBuf *b : {&ctx->A, &ctx->B, &ctx->S0, &ctx->S1, &ctx->staging, &ctx->alpha, &ctx->partials,
                          &ctx->norms})
            release(ctx, *b);
        dev_free(ctx, ctx->d_err, 256);
        dev_free(ctx, ctx->d_bar, 256);
        if (ctx->h_alpha) cudaFreeHost(ctx->h_alpha);
        if (ctx->h_norms) cudaFreeHost(ctx->h_norms);
        if (ctx->h_err) cudaFreeHost(ctx->h_err);
        for (auto &ev : ctx->ev)
            if (ev) cudaEventDestroy(ev);
        for (cudaEvent_t ev : ctx->evp) cudaEventDestroy(ev);
        for (int k = 0; k < 3; ++k)
            for (cudaEvent_t ev : {ctx->e_in[k], ctx->e_done[k], ctx->e_out[k]})
                if (ev) cudaEventDestroy(ev);
        for (cudaEvent_t ev : ctx->e_sync)
            if (ev) cudaEventDestroy(ev);
        if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
        if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
    }
    delete ctx;
}

tls_status tls_set_profiling(tls_ctx *ctx, int on)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_set_profiling: ctx is NULL");
    std::lock_guard<FairMutex> lk(ctx->mu);
    ctx->profiling = on != 0;
    return ok();
}

tls_status tls_get_profile(tls_ctx *ctx, tls_profile *out)
{
    if (!ctx || !out) return fail(TLS_ERR_ARG, "tls_get_profile: NULL argument");
    std::lock_guard<FairMutex> lk(ctx->mu);
    *out = ctx->prof;
    return ok();
}

tls_status tls_set_barrier_budget(tls_ctx *ctx, int64_t polls)
{
    if (!ctx || polls < 0) return fail(TLS_ERR_ARG, "tls_set_barrier_budget: bad argument");
    std::lock_guard<FairMutex> lk(ctx->mu);
    ctx->barrier_budget = polls;
    return ok();
}

tls_status tls_load_gauge(tls_ctx *ctx, const double *U, int nd, const int dims[4], int on_device, void *stream,
                          tls_gauge_id *out)
{
    if (!ctx || !U || !dims || !out) return fail(TLS_ERR_ARG, "tls_load_gauge: NULL argument");
    if (nd != 3 && nd != 4) return fail(TLS_ERR_ARG, "tls_load_gauge: nd = %d, must be 3 or 4", nd);
    for (int k = 0; k < 4; ++k)
        if (dims[k] <= 0) return fail(TLS_ERR_ARG, "tls_load_gauge: dims[%d] = %d", k, dims[k]);
    for (int k = 0; k < 3; ++k)
        if (dims[k] & 1)
            return fail(TLS_ERR_ARG,
                        "tls_load_gauge: spatial extent dims[%d] = %d is odd; the +-2 hops need even extents", k,
                        dims[k]);
    const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
    if (V >= (1LL << 31)) return fail(TLS_ERR_ARG, "tls_load_gauge: %lld sites exceed 2^31", (long long)V);
    std::lock_guard<FairMutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Gauge gg;
    for (int k = 0; k < 4; ++k) gg.L[k] = dims[k];
    gg.g.hx = dims[0] / 2;
    gg.g.hy = dims[1] / 2;
    gg.g.hz = dims[2] / 2;
    gg.g.Vs = gg.g.hx * gg.g.hy * gg.g.hz;
    gg.g.Ps = ((int64_t)gg.g.Vs + 31) / 32 * 32;
    gg.Up_bytes = (size_t)dims[3] * 8 * 3 * 9 * gg.g.Ps * 16;
    tls_status s = dev_alloc(ctx, (void **)&gg.Up, gg.Up_bytes, "tls_load_gauge: packed links");
    if (s != TLS_OK) return s;
    cudaError_t e = cudaMemsetAsync(gg.Up, 0, gg.Up_bytes, st);
    const int64_t Vslice = (int64_t)dims[0] * dims[1] * dims[2];
    const void *U_dev = on_device ? (const void *)U : nullptr;
    if (e == cudaSuccess && U_dev) {
        e = launch_ingest_gauge((const double *)U_dev, nd, gg.Up, gg.g, gg.L, st);
    } else if (e == cudaSuccess) {
        // Host input: only the spatial links travel (a 2-D copy of the first
        // 3 of the nd link groups of every site), in slice groups through two
        // staging slots: the copy of group k+1 (stream s_in) overlaps the
        // ingest of group k on the launch stream.
        const size_t site_b = (size_t)nd * 144, spat_b = 3 * 144;
        const size_t slice_sb = (size_t)Vslice * spat_b;  // staged bytes per slice
        const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(dims[3], (int64_t)(256ULL << 20) / (int64_t)slice_sb));
        const int nslot = dims[3] > chunk ? 2 : 1;
        void *tmp = nullptr;
        s = dev_alloc(ctx, &tmp, slice_sb * chunk * nslot, "tls_load_gauge: staging");
        if (s != TLS_OK) {
            dev_free(ctx, gg.Up, gg.Up_bytes);
            return s;
        }
        e = cudaEventRecord(ctx->e_sync[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_in, ctx->e_sync[0], 0);
        for (int k = 0, t0 = 0; t0 < dims[3] && e == cudaSuccess; ++k, t0 += chunk) {
            const int nsl = std::min(chunk, dims[3] - t0);
            const int slot = k % nslot;
            char *buf = (char *)tmp + (size_t)slot * slice_sb * chunk;
            if (k >= nslot) e = cudaStreamWaitEvent(ctx->s_in, ctx->e_done[slot], 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(buf, spat_b, (const char *)U + (size_t)t0 * Vslice * site_b, site_b, spat_b,
                                      (size_t)Vslice * nsl, cudaMemcpyHostToDevice, ctx->s_in);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->e_in[slot], ctx->s_in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->e_in[slot], 0);
            int Lc[4] = {dims[0], dims[1], dims[2], nsl};
            if (e == cudaSuccess)
                e = launch_ingest_gauge((const double *)buf, 3, gg.Up + (size_t)t0 * 8 * 3 * 9 * gg.g.Ps * 2, gg.g, Lc,
                                        st);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->e_done[slot], st);
        }
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
        e2 = cudaStreamSynchronize(ctx->s_in);
        if (e == cudaSuccess) e = e2;
        dev_free(ctx, tmp, slice_sb * chunk * nslot);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(ctx, gg.Up, gg.Up_bytes);
        return cuda_fail(e, "tls_load_gauge");
    }
    const int64_t id = ctx->next_id++;
    ctx->gauges[id] = gg;
    *out = id;
    return ok();
}

tls_status tls_build_twolink(tls_ctx *ctx, tls_gauge_id id, int wprec, int recon, int keep_U, void *stream)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_build_twolink: ctx is NULL");
    std::lock_guard<FairMutex> lk(ctx->mu);
    Gauge *gg = find_gauge(ctx, id);
    if (!gg) return fail(TLS_ERR_NOT_FOUND, "tls_build_twolink: unknown gauge id %lld", (long long)id);
    if (!gg->Up) return fail(TLS_ERR_STATE, "tls_build_twolink: the links of gauge %lld were released", (long long)id);
    const int wf = wfmt_of(wprec, recon);
    if (wf < 0) return fail(TLS_ERR_UNSUPPORTED, "tls_build_twolink: precision %d with %d reals", wprec, recon);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = gg->L[3] * 8;
    const size_t wbytes = (size_t)nblk * 3 * gg->g.Ps * wfmt_bytes(wf);
    if (gg->W && gg->W_bytes != wbytes) {
        dev_free(ctx, gg->W, gg->W_bytes);
        gg->W = nullptr;
        gg->W_bytes = 0;
    }
    gg->built = false;
    if (!gg->W) {
        tls_status s = dev_alloc(ctx, (void **)&gg->W, wbytes, "tls_build_twolink: W");
        if (s != TLS_OK) return s;
        gg->W_bytes = wbytes;
        cudaMemsetAsync(gg->W, 0, wbytes, st);
    }
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
    if (ctx->profiling) cudaEventRecord(ctx->ev[0], st);
    cudaError_t e = launch_build_twolink(gg->Up, gg->W, wf, gg->g, nblk, ctx->d_err, st);
    if (ctx->profiling) cudaEventRecord(ctx->ev[1], st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tls_build_twolink");
    if (ctx->profiling) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
        ctx->prof = tls_profile{};
        ctx->prof.ms_build = ms;
        ctx->prof.ms_total = ms;
        ctx->prof.launches = 1;
    }
    if (herr & DERR_RECON8)
        return fail(TLS_ERR_DEVICE, "tls_build_twolink: a two-link matrix has |W00| too close to 1 for the 8-real form");
    gg->wfmt = wf;
    gg->built = true;
    if (!keep_U) {
        dev_free(ctx, gg->Up, gg->Up_bytes);
        gg->Up = nullptr;
        gg->Up_bytes = 0;
    }
    return ok();
}

tls_status tls_ape_smear(tls_ctx *ctx, tls_gauge_id id, double alpha, int n_steps, void *stream)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_ape_smear: ctx is NULL");
    std::lock_guard<FairMutex> lk(ctx->mu);
    Gauge *gg = find_gauge(ctx, id);
    if (!gg) return fail(TLS_ERR_NOT_FOUND, "tls_ape_smear: unknown gauge id %lld", (long long)id);
    if (!gg->Up) return fail(TLS_ERR_STATE, "tls_ape_smear: the links of gauge %lld were released", (long long)id);
    if (n_steps < 0 || !(alpha >= 0.0 && alpha <= 1.0))
        return fail(TLS_ERR_ARG, "tls_ape_smear: n_steps %d, alpha %g", n_steps, alpha);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    // the derived fields no longer match the links
    gg->built = false;
    if (gg->L1) {
        dev_free(ctx, gg->L1, gg->L1_bytes);
        gg->L1 = nullptr;
        gg->L1_bytes = 0;
        gg->l1fmt = -1;
    }
    if (n_steps == 0) return ok();
    double *tmp = nullptr;
    tls_status s = dev_alloc(ctx, (void **)&tmp, gg->Up_bytes, "tls_ape_smear: link copy");
    if (s != TLS_OK) return s;
    cudaError_t e = cudaMemsetAsync(tmp, 0, gg->Up_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
    if (ctx->profiling) cudaEventRecord(ctx->ev[0], st);
    double *cur = gg->Up, *nxt = tmp;
    const int nblk = gg->L[3] * 8;
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
        e = launch_ape_step(cur, nxt, gg->g, nblk, alpha, ctx->d_err, st);
        std::swap(cur, nxt);
    }
    if (ctx->profiling) cudaEventRecord(ctx->ev[1], st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(ctx, tmp, gg->Up_bytes);
        return cuda_fail(e, "tls_ape_smear");
    }
    // keep the buffer that holds the result, free the other
    gg->Up = cur;
    dev_free(ctx, nxt, gg->Up_bytes);
    if (ctx->profiling) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
        ctx->prof = tls_profile{};
        ctx->prof.ms_total = ms;
        ctx->prof.launches = n_steps;
    }
    if (herr & DERR_PROJECT)
        return fail(TLS_ERR_DEVICE, "tls_ape_smear: a link projection met a singular matrix or did not settle");
    return ok();
}

tls_status tls_build_links(tls_ctx *ctx, tls_gauge_id id, int prec, int keep_U, void *stream)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_build_links: ctx is NULL");
    std::lock_guard<FairMutex> lk(ctx->mu);
    Gauge *gg = find_gauge(ctx, id);
    if (!gg) return fail(TLS_ERR_NOT_FOUND, "tls_build_links: unknown gauge id %lld", (long long)id);
    if (!gg->Up) return fail(TLS_ERR_STATE, "tls_build_links: the links of gauge %lld were released", (long long)id);
    const int fmt = prec == TLS_F64 ? W_F64_18 : prec == TLS_F32 ? W_F32_18 : -1;
    if (fmt < 0) return fail(TLS_ERR_UNSUPPORTED, "tls_build_links: precision %d (TLS_F64 or TLS_F32)", prec);
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)gg->L[3] * 8 * 3 * gg->g.Ps * wfmt_bytes(fmt);
    if (gg->L1 && gg->L1_bytes != bytes) {
        dev_free(ctx, gg->L1, gg->L1_bytes);
        gg->L1 = nullptr;
        gg->L1_bytes = 0;
    }
    if (!gg->L1) {
        tls_status s = dev_alloc(ctx, (void **)&gg->L1, bytes, "tls_build_links: link field");
        if (s != TLS_OK) return s;
        gg->L1_bytes = bytes;
        cudaMemsetAsync(gg->L1, 0, bytes, st);
    }
    cudaError_t e = launch_build_links(gg->Up, gg->L1, fmt, gg->g, gg->L[3] * 8, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tls_build_links");
    gg->l1fmt = fmt;
    if (!keep_U) {
        dev_free(ctx, gg->Up, gg->Up_bytes);
        gg->Up = nullptr;
        gg->Up_bytes = 0;
    }
    return ok();
}

tls_status tls_smear_onelink(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int vecs_on_device, int nvec,
                             int N, double alpha, int timeslice, int storage, void *stream, double *norms_out)
{
    return smear_impl(ctx, id, vecs, io_prec, vecs_on_device, nvec, N, alpha, timeslice, storage, TLS_KERNEL_MRHS, 0,
                      0, nullptr, stream, norms_out, 1);
}

tls_status tls_free_gauge(tls_ctx *ctx, tls_gauge_id id)
{
    if (!ctx) return fail(TLS_ERR_ARG, "tls_free_gauge: ctx is NULL");
    std::lock_guard<FairMutex> lk(ctx->mu);
    Gauge *gg = find_gauge(ctx, id);
    if (!gg) return fail(TLS_ERR_NOT_FOUND, "tls_free_gauge: unknown gauge id %lld", (long long)id);
    cudaSetDevice(ctx->device);
    if (serve_gauge_busy(ctx, id))
        return fail(TLS_ERR_STATE, "tls_free_gauge: serving jobs still use gauge %lld", (long long)id);
    cudaDeviceSynchronize();
    free_gauge(ctx, *gg);
    ctx->gauges.erase(id);
    return ok();
}

static tls_status export_common(tls_ctx *ctx, tls_gauge_id id, double *out, int on_device, void *stream, bool w)
{
    if (!ctx || !out) return fail(TLS_ERR_ARG, "tls_export: NULL argument");
    std::lock_guard<FairMutex> lk(ctx->mu);
    Gauge *gg = find_gauge(ctx, id);
    if (!gg) return fail(TLS_ERR_NOT_FOUND, "tls_export: unknown gauge id %lld", (long long)id);
    if (w && !gg->built) return fail(TLS_ERR_NOT_BUILT, "tls_export_twolink: W not built");
    if (!w && !gg->Up) return fail(TLS_ERR_STATE, "tls_export_gauge: links released");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)gg->L[0] * gg->L[1] * gg->L[2] * gg->L[3] * 3 * 144;
    double *dst = out;
    void *tmp = nullptr;
    if (!on_device) {
        tls_status s = dev_alloc(ctx, &tmp, bytes, "tls_export: staging");
        if (s != TLS_OK) return s;
        dst = (double *)tmp;
    }
    cudaError_t e = w ? launch_export_twolink(gg->W, gg->wfmt, dst, gg->g, gg->L, st)
                      : launch_export_gauge(gg->Up, dst, gg->g, gg->L, st);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (tmp) dev_free(ctx, tmp, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "tls_export");
    return ok();
}

tls_status tls_export_twolink(tls_ctx *ctx, tls_gauge_id id, double *out, int on_device, void *stream)
{
    return export_common(ctx, id, out, on_device, stream, true);
}

tls_status tls_export_gauge(tls_ctx *ctx, tls_gauge_id id, double *out, int on_device, void *stream)
{
    return export_common(ctx, id, out, on_device, stream, false);
}

static float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

tls_status tls_smear(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int vecs_on_device, int nvec, int N,
                     double width, int timeslice, int storage, int kernel, void *stream, double *norms_out)
{
    return smear_impl(ctx, id, vecs, io_prec, vecs_on_device, nvec, N, width, timeslice, storage, kernel, 0, 0,
                      nullptr, stream, norms_out);
}

}  // extern "C"

namespace tls {

// Bytes of caller vectors per slice group when they come from host memory.
constexpr size_t kGroupBytes = size_t(2) << 30;

tls_status smear_impl(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int vecs_on_device, int nvec, int N,
                      double width, int timeslice, int storage, int kernel, int force_vb, int force_threads,
                      const int *force_tile, void *stream, double *norms_out, int op)
{
    if (!ctx || !vecs) return fail(TLS_ERR_ARG, "tls_smear: NULL argument");
    if (io_prec != TLS_F64 && io_prec != TLS_F32)
        return fail(TLS_ERR_ARG, "tls_smear: io_prec %d must be TLS_F64 or TLS_F32", io_prec);
    if (nvec < 1 || nvec > 65535) return fail(TLS_ERR_ARG, "tls_smear: nvec = %d", nvec);
    if (N < 0) return fail(TLS_ERR_ARG, "tls_smear: N = %d < 0", N);
    if (!std::isfinite(width)) return fail(TLS_ERR_ARG, "tls_smear: width is not finite");
    if (kernel < TLS_KERNEL_AUTO || kernel > TLS_KERNEL_MRHS_ZM)
        return fail(TLS_ERR_ARG, "tls_smear: kernel %d", kernel);
    std::lock_guard<FairMutex> lk(ctx->mu);
    Gauge *gg = find_gauge(ctx, id);
    if (!gg) return fail(TLS_ERR_NOT_FOUND, "tls_smear: unknown gauge id %lld", (long long)id);
    if (op == 0 && !gg->built)
        return fail(TLS_ERR_NOT_BUILT, "tls_smear: tls_build_twolink has not run for gauge %lld", (long long)id);
    if (op == 1 && !gg->L1)
        return fail(TLS_ERR_NOT_BUILT, "tls_smear_onelink: tls_build_links has not run for gauge %lld", (long long)id);
    if (timeslice < TLS_ALL_T || timeslice >= gg->L[3])
        return fail(TLS_ERR_ARG, "tls_smear: timeslice %d outside [-1, %d)", timeslice, gg->L[3]);
    tls_status s = TLS_OK;
    if (op == 0) {
        s = check_smear_combo(*gg, storage);
        if (s != TLS_OK) return s;
    } else {
        const bool okc = storage == TLS_F64 ? gg->l1fmt == W_F64_18 : gg->l1fmt == W_F32_18;
        if (storage < TLS_F64 || storage > TLS_BF16) return fail(TLS_ERR_ARG, "tls_smear_onelink: storage %d", storage);
        if (!okc)
            return fail(TLS_ERR_UNSUPPORTED, "tls_smear_onelink: storage %d with link format %d", storage, gg->l1fmt);
    }
    const int fmt = op == 0 ? gg->wfmt : gg->l1fmt;
    const char *field = op == 0 ? gg->W : gg->L1;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;

    const SubGeom &g = gg->g;
    const int nsl = timeslice < 0 ? gg->L[3] : 1;
    const int t_first = timeslice < 0 ? 0 : timeslice;
    const int nblk = nsl * 8;
    const int64_t Vslice = (int64_t)gg->L[0] * gg->L[1] * gg->L[2];
    const int64_t V = Vslice * gg->L[3];
    const int VBY = vfmt_bytes(storage);
    const int64_t vs = (int64_t)nblk * g.Ps * VBY;        // packed bytes per vector
    const size_t io_elem = io_prec == TLS_F64 ? 8 : 4;
    const size_t io_slice_bytes = (size_t)Vslice * 6 * io_elem;

    // Kernel choice: explicit kernel, or the autotune table, or the planner's default.
    int kern = kernel;
    int vb = 0;
    int threads = 0;
    int tile[3] = {0, 0, 0};
    {
        TuneKey key{{gg->L[0], gg->L[1], gg->L[2], gg->L[3]}, nsl, nvec, storage, gg->wfmt};
        auto it = ctx->tune.find(key);
        const bool have = it != ctx->tune.end();
        if (kern == TLS_KERNEL_AUTO) {
            kern = have ? it->second.kernel : (nvec == 1 ? TLS_KERNEL_SINGLE : TLS_KERNEL_MRHS);
        }
        if (have && it->second.kernel == kern) {
            vb = it->second.vb;
            threads = it->second.threads;
            for (int k = 0; k < 3; ++k) tile[k] = it->second.tile[k];
        }
    }
    if (force_vb > 0) vb = force_vb;
    if (force_threads > 0) threads = force_threads;
    if (force_tile)
        for (int k = 0; k < 3; ++k) tile[k] = force_tile[k];
    if (op == 1) {  // one-link hops: the interleaved kernel only
        kern = TLS_KERNEL_MRHS;
        for (int k = 0; k < 3; ++k) tile[k] = 0;
    }
    // FP32 and 16-bit records of the interleaved layout come in vector pairs:
    // a group of an odd number of vectors carries one padding record
    // (computed, never unpacked).
    const bool pad_pairs = storage != TLS_F64;
    auto rec_of = [&](int n) { return pad_pairs ? (n + 1) & ~1 : n; };
    const int G0 = rec_of(std::min(nvec, 256));
    if (kern == TLS_KERNEL_SINGLE) {
        vb = 1;
        if (threads <= 0) threads = 128;
    } else if (kern == TLS_KERNEL_MRHS || kern == TLS_KERNEL_MRHS_ROWS || kern == TLS_KERNEL_MRHS_ZM) {
        // eight vectors per thread: FP32 storage, packed kernel (tile[1] = 2) only
        const bool vb8 = vb == 8 && storage == TLS_F32 && (tile[1] == 2 || (tile[1] >= 6 && tile[1] <= 8)) &&
                         kern == TLS_KERNEL_MRHS;
        if (vb <= 0 || (vb > 4 && !vb8) || G0 % vb != 0 || (storage == TLS_F64 && vb > 2))
            vb = default_il_vb(storage, G0);
        if (threads == 0) threads = 256;  // < 0: the register-capped variant
        // TMA row staging needs 16-byte copies and a row that fits in shared memory
        if (kern == TLS_KERNEL_MRHS_ROWS &&
            !(rows_applicable(fmt, storage, gg->g, G0, vb, ctx->max_smem) &&
              rows_applicable(fmt, storage, gg->g, rec_of(nvec % 256 ? nvec % 256 : 256), vb, ctx->max_smem)))
            kern = TLS_KERNEL_MRHS;
    } else {
        if (vb <= 0) vb = default_vb(storage, nvec);
        if (vb == 2) vb = 1;
        if (threads <= 0) threads = 256;
    }
    // The multi-RHS kernel works on the interleaved layout in groups of <= 256 vectors.
    const bool il_layout = kern == TLS_KERNEL_MRHS || kern == TLS_KERNEL_MRHS_ROWS || kern == TLS_KERNEL_MRHS_ZM;
    const int G = il_layout ? std::min(nvec, 256) : nvec;

    // Host vectors go through bulk copies (DMA) into a staging buffer.  On a
    // GB300 these measured faster than letting the layout kernels read and
    // write pinned host memory over NVLink-C2C directly (1236 ms against
    // 1436-1450 ms for the 64^3x96 step), so zero-copy is not used.
    void *vecs_dev = vecs_on_device ? vecs : nullptr;
    const bool staged = vecs_dev == nullptr;

    // Workspace.
    size_t a_bytes = (size_t)vs * (il_layout ? rec_of(G) : G);
    s = ensure(ctx, ctx->A, a_bytes, "tls_smear: vector buffer A");
    if (s == TLS_OK) s = ensure(ctx, ctx->B, a_bytes, "tls_smear: vector buffer B");
    // alpha per vector in FP64, then the same rounded to FP32 (read by the FP32-arithmetic
    // kernels); one more entry of each for a padding record
    const int nalpha = nvec + 1;
    const size_t alpha_bytes = sizeof(double) * nalpha + sizeof(float) * nalpha;
    if (s == TLS_OK) s = ensure(ctx, ctx->alpha, alpha_bytes, "tls_smear: alpha");
    if (s == TLS_OK && norms_out)
        s = ensure(ctx, ctx->partials, sizeof(double) * kNormPartsPerSlice * nsl * nvec, "tls_smear: partials");
    if (s == TLS_OK && norms_out) s = ensure(ctx, ctx->norms, sizeof(double) * nvec, "tls_smear: norms");
    // Host vectors go through slice groups of about kGroupBytes in up to three
    // rotating staging slots, so that copies in and out overlap the smearing
    // of other groups.  The persistent kernel takes all slices in one group.
    int tg = nsl, ngroup = 1, nslot = 1;
    size_t slot_bytes = 0;
    if (staged) {
        const size_t total = io_slice_bytes * nsl * nvec;
        if (kern != TLS_KERNEL_PERSISTENT && nsl >= 2) {
            const int64_t want = std::max<int64_t>(4, (int64_t)((total + kGroupBytes - 1) / kGroupBytes));
            tg = (int)((nsl + std::min<int64_t>(nsl, want) - 1) / std::min<int64_t>(nsl, want));
            ngroup = (nsl + tg - 1) / tg;
        }
        nslot = std::min(ngroup, 3);
        slot_bytes = (io_slice_bytes * tg * nvec + 255) / 256 * 256;
        if (s == TLS_OK) s = ensure(ctx, ctx->staging, slot_bytes * nslot, "tls_smear: host staging");
    }
    if (s != TLS_OK) return s;
    if (ctx->h_alpha_n < (size_t)nalpha) {
        if (ctx->h_alpha) cudaFreeHost(ctx->h_alpha);
        ctx->h_alpha = nullptr;
        cudaError_t e = cudaMallocHost(&ctx->h_alpha, alpha_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "tls_smear: pinned alpha");
        ctx->h_alpha_n = nalpha;
    }
    if (ctx->h_norms_n < (size_t)nvec) {
        if (ctx->h_norms) cudaFreeHost(ctx->h_norms);
        ctx->h_norms = nullptr;
        cudaError_t e = cudaMallocHost(&ctx->h_norms, sizeof(double) * nvec);
        if (e != cudaSuccess) return cuda_fail(e, "tls_smear: pinned norms");
        ctx->h_norms_n = nvec;
    }

    // Persistent-kernel plan: co-resident grid, L2-sized groups, scratch.
    PersistArgs pa{};
    // tile[1] = 1: the on-chip form, when a block's W and scratch fit in shared memory
    if (kern == TLS_KERNEL_PERSISTENT && N > 0 && tile[1] == 1 &&
        onchip_plan(g, wfmt_bytes(fmt), vfmt_bytes(storage == TLS_F64 ? P_F64 : P_F32), nvec,
                    ctx->max_smem, &pa.nvg, &pa.smem)) {
        pa.onchip = 1;
        pa.sprec = storage == TLS_F64 ? P_F64 : P_F32;
    } else if (kern == TLS_KERNEL_PERSISTENT && N > 0) {
        threads = std::min(threads, 256);  // the grid-wide form is built for CTAs of <= 256 threads
        const int sprec = storage == TLS_F64 ? P_F64 : P_F32;
        const int occ = persistent_occupancy(fmt, storage, sprec, vb, threads);
        if (occ <= 0) return fail(TLS_ERR_UNSUPPORTED, "tls_smear: persistent kernel cannot be resident");
        const int SBY = vfmt_bytes(sprec);
        const double per_blk = (double)g.Ps * (3.0 * wfmt_bytes(fmt) + 2.0 * nvec * SBY);
        // L2 budget of one group: tile[0] MB from the tune table, else 48 MB
        const double budget = (tile[0] > 0 ? tile[0] : 48) * double(1 << 20);
        int gb = (int)std::max(1.0, std::floor(budget / per_blk));
        const int64_t want_items = (int64_t)occ * ctx->num_sms * threads;
        const int nchunk = (nvec + vb - 1) / vb;
        while (gb < nblk && (int64_t)gb * g.Vs * nchunk < want_items) ++gb;
        gb = std::min(gb, nblk);
        pa.group_blocks = gb;
        pa.sstride = (int64_t)gb * g.Ps * SBY;
        s = ensure(ctx, ctx->S0, (size_t)pa.sstride * nvec, "tls_smear: scratch 0");
        if (s == TLS_OK) s = ensure(ctx, ctx->S1, (size_t)pa.sstride * nvec, "tls_smear: scratch 1");
        if (s != TLS_OK) return s;
        const int64_t items = ((int64_t)gb * g.Vs + 31) / 32 * 32 * nchunk;
        pa.grid = (int)std::min<int64_t>((int64_t)occ * ctx->num_sms, std::max<int64_t>(1, (items + threads - 1) / threads));
        pa.sprec = sprec;
    }

    const double a = N > 0 ? (op == 0 ? width / (4.0 * N) : width) : 0.0;
    for (int v = 0; v < nalpha; ++v) ctx->h_alpha[v] = a;
    float *h_alphaf = reinterpret_cast<float *>(ctx->h_alpha + nalpha);
    for (int v = 0; v < nalpha; ++v) h_alphaf[v] = (float)a;  // round to nearest, as the kernels' conversion

    cudaError_t e = cudaSuccess;
    int64_t launches = 0, iter_launches = 0;
    const bool prof = ctx->profiling;
    // Profiling: (begin, end) event pairs per phase, read after the final synchronisation.
    enum { PH_H2D, PH_PACK, PH_ITER, PH_UNPACK, PH_D2H, PH_N };
    struct Span {
        int a, b, phase;
    };
    std::vector<Span> spans;
    int nev = 0;
    auto ev_rec = [&](cudaStream_t s) -> int {
        if (!prof) return -1;
        if (nev >= (int)ctx->evp.size()) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreate(&ev) != cudaSuccess) return -1;
            ctx->evp.push_back(ev);
        }
        cudaEventRecord(ctx->evp[nev], s);
        return nev++;
    };
    auto span = [&](int a0, int a1, int phase) {
        if (a0 >= 0 && a1 >= 0) spans.push_back(Span{a0, a1, phase});
    };
    const int ev_begin = ev_rec(st);
    e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->alpha.p, ctx->h_alpha, alpha_bytes, cudaMemcpyHostToDevice, st);

    // One pass of the method over slices [t_abs, t_abs + ns): their canonical
    // vectors are at src / dst (vector stride vsites sites; slice t_abs is
    // relative slice t_rel0 there).  Packs, runs the N steps, unpacks, and
    // writes the norm partials of these slices at their place in the
    // per-slice partials of the call (so any split into slice groups gives
    // the same norms).
    const size_t io_elem_b = io_elem;
    auto run_slices = [&](const char *src_io, char *dst_io, int64_t vsites, int t_rel0, int t_abs, int ns) {
        const int nb = ns * 8;
        const int64_t vsg = (int64_t)nb * g.Ps * VBY;  // packed bytes per vector of these slices
        const char *Wg = field + (size_t)t_abs * 8 * 3 * g.Ps * wfmt_bytes(fmt);
        const size_t io_vec_bytes = (size_t)vsites * 6 * io_elem_b;
        for (int g0 = 0; g0 < nvec && e == cudaSuccess; g0 += G) {
            const int gn = std::min(G, nvec - g0);
            const int rn = il_layout ? rec_of(gn) : gn;  // records per site in the packed buffers
            const char *src_g = src_io + (size_t)g0 * io_vec_bytes;
            char *dst_g = dst_io + (size_t)g0 * io_vec_bytes;
            const bool il = il_layout;
            const int m0 = ev_rec(st);
            e = il ? launch_pack_il(src_g, io_prec, vsites, (char *)ctx->A.p, storage, g, gg->L, t_rel0, ns, gn, rn, 0,
                                    st)
                   : launch_pack_vectors(src_g, io_prec, vsites, (char *)ctx->A.p, storage, vsg, g, gg->L, t_rel0, ns,
                                         gn, st);
            ++launches;
            const int m1 = ev_rec(st);
            char *result = (char *)ctx->A.p;
            const double *alpha_g = (const double *)ctx->alpha.p + g0;
            const float *alphaf_g = reinterpret_cast<const float *>((const double *)ctx->alpha.p + nalpha) + g0;
            if (N > 0 && e == cudaSuccess) {
                if (kern == TLS_KERNEL_PERSISTENT) {
                    pa.W = Wg;
                    pa.in = (const char *)ctx->A.p;
                    pa.out = (char *)ctx->B.p;
                    pa.scr[0] = (char *)ctx->S0.p;
                    pa.scr[1] = (char *)ctx->S1.p;
                    pa.alpha = alpha_g;
                    pa.g = g;
                    pa.nblk = nb;
                    pa.nvec = gn;
                    pa.N = N;
                    pa.vstride = vsg;
                    pa.wfmt = fmt;
                    pa.prec = storage;
                    pa.vb = vb;
                    pa.threads = threads;
                    pa.bar = ctx->d_bar;
                    pa.err = ctx->d_err;
                    pa.budget = ctx->barrier_budget > 0 ? ctx->barrier_budget : kDefaultBudget;
                    pa.stream = st;
                    e = cudaMemsetAsync(ctx->d_bar, 0, 2 * sizeof(unsigned), st);
                    if (e == cudaSuccess) e = launch_persistent(pa);
                    ++launches;
                    ++iter_launches;
                    result = (char *)ctx->B.p;
                } else {
                    StepArgs sa{};
                    sa.W = Wg;
                    sa.g = g;
                    sa.nblk = nb;
                    sa.wfmt = fmt;
                    sa.prec_in = sa.prec_out = storage;
                    sa.vb = vb;
                    sa.threads = threads;
                    sa.stream = st;
                    sa.err = ctx->d_err;
                    sa.vstride_in = sa.vstride_out = vsg;
                    for (int k = 0; k < 3; ++k) sa.tile[k] = tile[k];
                    const int sub_groups = kern == TLS_KERNEL_SINGLE ? gn : 1;
                    sa.nvec = kern == TLS_KERNEL_SINGLE ? 1 : rn;
                    for (int gi = 0; gi < sub_groups && e == cudaSuccess; ++gi) {
                        char *x = (char *)ctx->A.p + (size_t)gi * vsg;
                        char *y = (char *)ctx->B.p + (size_t)gi * vsg;
                        for (int it = 0; it < N && e == cudaSuccess; ++it) {
                            sa.in = (it & 1) ? y : x;
                            sa.out = (it & 1) ? x : y;
                            sa.alpha = alpha_g + gi;
                            sa.alphaf = alphaf_g + gi;
                            e = op == 1                         ? launch_hop(sa)
                                : kern == TLS_KERNEL_MRHS_ROWS  ? launch_step_rows(sa, ctx->d_err)
                                : kern == TLS_KERNEL_MRHS_ZM    ? launch_step_zm(sa)
                                : il                            ? launch_step_il(sa)
                                                                : launch_step(sa);
                            ++launches;
                            ++iter_launches;
                        }
                    }
                    result = (N & 1) ? (char *)ctx->B.p : (char *)ctx->A.p;
                }
            }
            const int m2 = ev_rec(st);
            if (e == cudaSuccess) {
                e = il ? launch_unpack_il(result, storage, dst_g, io_prec, vsites, g, gg->L, t_rel0, ns, gn, rn, 0, st)
                       : launch_unpack_vectors(result, storage, vsg, dst_g, io_prec, vsites, g, gg->L, t_rel0, ns, gn,
                                               nullptr, nullptr, st);
                ++launches;
            }
            const int m3 = ev_rec(st);
            span(m0, m1, PH_PACK);
            span(m1, m2, PH_ITER);
            span(m2, m3, PH_UNPACK);
        }
        if (e == cudaSuccess && norms_out) {
            const int m0 = ev_rec(st);
            e = launch_norm_partials(dst_io + (size_t)t_rel0 * io_slice_bytes, io_prec, vsites, Vslice, ns, nvec,
                                     (double *)ctx->partials.p, (int64_t)nsl * kNormPartsPerSlice,
                                     (int64_t)(t_abs - t_first) * kNormPartsPerSlice, st);
            ++launches;
            span(m0, ev_rec(st), PH_UNPACK);
        }
    };

    if (!staged) {
        run_slices((const char *)vecs_dev, (char *)vecs_dev, V, t_first, t_first, nsl);
    } else {
        // Host vectors: slice groups through rotating staging slots.  Group k
        // is copied in on s_in while group k-1 is smeared on the launch stream
        // and group k-2 is copied out on s_out; each slot is refilled only after
        // its previous group has left (events).  One 2-D copy per group and
        // direction (all vectors, the group's slices).
        const char *hsrc = (const char *)vecs;
        const size_t pitch = (size_t)V * 6 * io_elem;
        auto group_slices = [&](int k) { return std::min(tg, nsl - k * tg); };
        e = e == cudaSuccess ? cudaEventRecord(ctx->e_sync[0], st) : e;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_in, ctx->e_sync[0], 0);
        auto h2d = [&](int k) {
            const int slot = k % nslot;
            const int ns = group_slices(k);
            const size_t width_b = io_slice_bytes * ns;
            if (k >= nslot && e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_in, ctx->e_out[slot], 0);
            const int c0 = ev_rec(ctx->s_in);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync((char *)ctx->staging.p + slot * slot_bytes, width_b,
                                      hsrc + (size_t)(t_first + k * tg) * io_slice_bytes, pitch, width_b, nvec,
                                      cudaMemcpyHostToDevice, ctx->s_in);
            span(c0, ev_rec(ctx->s_in), PH_H2D);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->e_in[slot], ctx->s_in);
        };
        h2d(0);
        if (ngroup > 1) h2d(1);
        for (int k = 0; k < ngroup && e == cudaSuccess; ++k) {
            const int slot = k % nslot;
            const int ns = group_slices(k);
            char *buf = (char *)ctx->staging.p + slot * slot_bytes;
            e = cudaStreamWaitEvent(st, ctx->e_in[slot], 0);
            if (e == cudaSuccess) run_slices(buf, buf, Vslice * ns, 0, t_first + k * tg, ns);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->e_done[slot], st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_out, ctx->e_done[slot], 0);
            const size_t width_b = io_slice_bytes * ns;
            const int c0 = ev_rec(ctx->s_out);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync((char *)vecs + (size_t)(t_first + k * tg) * io_slice_bytes, pitch, buf, width_b,
                                      width_b, nvec, cudaMemcpyDeviceToHost, ctx->s_out);
            span(c0, ev_rec(ctx->s_out), PH_D2H);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->e_out[slot], ctx->s_out);
            if (k + 2 < ngroup) h2d(k + 2);
        }
        // the launch stream resumes after the last copy out (copies on s_out are in order)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->e_out[(ngroup - 1) % nslot], 0);
    }
    if (e == cudaSuccess && norms_out) {
        e = launch_reduce_norms((const double *)ctx->partials.p, nsl * kNormPartsPerSlice, nvec,
                                (double *)ctx->norms.p, st);
        ++launches;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->h_norms, ctx->norms.p, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st);
    }
    const int ev_end = ev_rec(st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (staged) {  // nothing may still be copying from or to the caller's host buffer
        es = cudaStreamSynchronize(ctx->s_in);
        if (e == cudaSuccess) e = es;
        es = cudaStreamSynchronize(ctx->s_out);
        if (e == cudaSuccess) e = es;
    }
    if (e != cudaSuccess) return cuda_fail(e, "tls_smear");
    herr = *ctx->h_err;
    if (prof) {
        tls_profile &p = ctx->prof;
        p = tls_profile{};
        double ph[PH_N] = {0, 0, 0, 0, 0};
        for (const Span &sp : spans) ph[sp.phase] += elapsed(ctx->evp[sp.a], ctx->evp[sp.b]);
        p.ms_total = ev_begin >= 0 && ev_end >= 0 ? elapsed(ctx->evp[ev_begin], ctx->evp[ev_end]) : 0.0;
        p.ms_h2d = ph[PH_H2D];
        p.ms_pack = ph[PH_PACK];
        p.ms_iter = ph[PH_ITER];
        p.ms_unpack = ph[PH_UNPACK];
        p.ms_d2h = ph[PH_D2H];
        p.launches = launches;
        p.iter_launches = iter_launches;
        const double sites = (double)nblk * g.Vs;
        const double wb = 3.0 * wfmt_bytes(fmt), vbb = 2.0 * VBY;
        p.iter_bytes = kern == TLS_KERNEL_SINGLE ? (double)N * nvec * sites * (wb + vbb)
                                                 : (double)N * sites * (wb * ((nvec + G - 1) / G) + nvec * vbb);
        p.iter_flops = (op == 0 ? 450.0 : 438.0) * N * nvec * sites;
        p.kernel = kern;
        p.vecs_per_thread = vb;
    }
    if (herr & DERR_TIMEOUT)
        return fail(TLS_ERR_TIMEOUT, "tls_smear: a bounded device wait (barrier or copy completion) ran out");
    if (herr) return fail(TLS_ERR_DEVICE, "tls_smear: device error word 0x%x", herr);
    if (norms_out) std::memcpy(norms_out, ctx->h_norms, sizeof(double) * nvec);
    return ok();
}

}  // namespace tls
