// noalloc.cu -- tls_smear_noalloc: the persistent smearing path with its
// scratch in a fixed, library-owned device array instead of cudaMalloc.
//
// Who needs it: code that must not allocate device memory while it runs.
// Examples are a host thread on a latency-critical path, where cudaFree
// synchronises the whole device, and a process whose device memory is owned
// by another allocator (a framework's caching pool) that must stay the only
// one handing out memory.  The call itself synchronises its stream and reads
// the error word back into host memory before it returns.  Such callers still pass
// their vectors in and get them back in place; everything else the call
// needs (the packed copies of the vectors, the persistent kernel's scratch
// ping-pong, its barrier words, the per-vector alpha and the error word)
// comes from one static __device__ array of TLS_NOALLOC_SCRATCH_BYTES.
//
// The array exists once per device that loads the library and lives until
// the process exits.  Its device address is looked up once per device, on
// the first call made with that device current (cudaGetSymbolAddress).
// Every call reuses the same array, which keeps whatever the previous call left:
// the words that must start at zero (barrier, error) are cleared by each
// call, and two calls whose work overlaps on the GPU (different streams or
// host threads without ordering) race on the array.  When the call returns
// TLS_ERR_TIMEOUT or TLS_ERR_DEVICE the caller's vectors hold an unspecified
// mix of input and partial results.
#include <cmath>
#include <mutex>

#include "api_internal.h"

namespace tls {

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[TLS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char *g_addr[kMaxDevices] = {};

// Device address of the static array on `device` (which must be current).
tls_status scratch_address(int device, char **out)
{
    if (device < 0 || device >= kMaxDevices)
        return fail(TLS_ERR_ARG, "tls_smear_noalloc: device %d beyond the %d supported", device, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "tls_smear_noalloc: cudaGetSymbolAddress");
        g_addr[device] = (char *)p;
    }
    *out = g_addr[device];
    return TLS_OK;
}

__global__ void k_fill_alpha(double *a, double v, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

size_t up256(size_t n) { return (n + 255) / 256 * 256; }

const long long kBudget = 20000000LL;

}  // namespace

}  // namespace tls

using namespace tls;

extern "C" tls_status tls_smear_noalloc(tls_ctx *ctx, tls_gauge_id id, void *vecs, int io_prec, int nvec, int N,
                                        double width, int timeslice, int storage, void *stream)
{
    if (!ctx || !vecs) return fail(TLS_ERR_ARG, "tls_smear_noalloc: NULL argument");
    if (io_prec != TLS_F64 && io_prec != TLS_F32)
        return fail(TLS_ERR_ARG, "tls_smear_noalloc: io_prec %d must be TLS_F64 or TLS_F32", io_prec);
    if (nvec < 1 || nvec > 65535) return fail(TLS_ERR_ARG, "tls_smear_noalloc: nvec = %d", nvec);
    if (N < 0) return fail(TLS_ERR_ARG, "tls_smear_noalloc: N = %d < 0", N);
    if (!std::isfinite(width)) return fail(TLS_ERR_ARG, "tls_smear_noalloc: width is not finite");
    std::lock_guard<FairMutex> lk(ctx->mu);
    auto git = ctx->gauges.find(id);
    if (git == ctx->gauges.end()) return fail(TLS_ERR_NOT_FOUND, "tls_smear_noalloc: unknown gauge id %lld", (long long)id);
    const Gauge &gg = git->second;
    if (!gg.built) return fail(TLS_ERR_NOT_BUILT, "tls_smear_noalloc: W of gauge %lld not built", (long long)id);
    if (timeslice < TLS_ALL_T || timeslice >= gg.L[3])
        return fail(TLS_ERR_ARG, "tls_smear_noalloc: timeslice %d outside [-1, %d)", timeslice, gg.L[3]);
    tls_status s = check_smear_combo(gg, storage);
    if (s != TLS_OK) return s;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "tls_smear_noalloc: cudaSetDevice");
    cudaPointerAttributes pattr{};
    e = cudaPointerGetAttributes(&pattr, vecs);
    if (e != cudaSuccess || pattr.type != cudaMemoryTypeDevice || pattr.device != ctx->device) {
        cudaGetLastError();
        return fail(TLS_ERR_ARG, "tls_smear_noalloc: vecs must be device memory of the context's device");
    }
    char *base = nullptr;
    s = scratch_address(ctx->device, &base);
    if (s != TLS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;

    const SubGeom &g = gg.g;
    const int nsl = timeslice < 0 ? gg.L[3] : 1;
    const int t_first = timeslice < 0 ? 0 : timeslice;
    const int nblk = nsl * 8;
    const int64_t V = (int64_t)gg.L[0] * gg.L[1] * gg.L[2] * gg.L[3];
    const int VBY = vfmt_bytes(storage);
    const int64_t vs = (int64_t)nblk * g.Ps * VBY;
    const int sprec = storage == TLS_F64 ? P_F64 : P_F32;
    const int SBY = vfmt_bytes(sprec);
    int vb = default_vb(storage, nvec);
    if (vb == 2) vb = 1;
    const int threads = 256;

    // Persistent plan (same rules as tls_smear): co-resident grid, L2-sized groups.
    PersistArgs pa{};
    size_t scr_bytes = 0;
    if (N > 0) {
        const int occ = persistent_occupancy(gg.wfmt, storage, sprec, vb, threads);
        if (occ <= 0) return fail(TLS_ERR_UNSUPPORTED, "tls_smear_noalloc: persistent kernel cannot be resident");
        const double per_blk = (double)g.Ps * (3.0 * wfmt_bytes(gg.wfmt) + 2.0 * nvec * SBY);
        int gb = (int)std::max(1.0, std::floor(48.0 * (1 << 20) / per_blk));
        const int64_t want_items = (int64_t)occ * ctx->num_sms * threads;
        const int nchunk = (nvec + vb - 1) / vb;
        while (gb < nblk && (int64_t)gb * g.Vs * nchunk < want_items) ++gb;
        gb = std::min(gb, nblk);
        pa.group_blocks = gb;
        pa.sstride = (int64_t)gb * g.Ps * SBY;
        scr_bytes = up256((size_t)pa.sstride * nvec);
        const int64_t items = ((int64_t)gb * g.Vs + 31) / 32 * 32 * nchunk;
        pa.grid = (int)std::min<int64_t>((int64_t)occ * ctx->num_sms,
                                         std::max<int64_t>(1, (items + threads - 1) / threads));
    }
    // Carve the static array: words | alpha | A | B | scratch 0 | scratch 1.
    const size_t words = 256;
    const size_t alpha_b = up256(sizeof(double) * nvec);
    const size_t vec_b = up256((size_t)vs * nvec);
    const size_t need = words + alpha_b + 2 * vec_b + 2 * scr_bytes;
    if (need > (size_t)TLS_NOALLOC_SCRATCH_BYTES)
        return fail(TLS_ERR_ARG,
                    "tls_smear_noalloc: this smear needs %zu bytes of scratch; the static scratch holds %zu "
                    "(TLS_NOALLOC_SCRATCH_BYTES); use tls_smear",
                    need, (size_t)TLS_NOALLOC_SCRATCH_BYTES);
    unsigned *bar = (unsigned *)base;
    int *err = (int *)(base + 128);
    double *alpha = (double *)(base + words);
    char *A = base + words + alpha_b;
    char *B = A + vec_b;
    char *S0 = B + vec_b;
    char *S1 = S0 + scr_bytes;

    const double a = N > 0 ? width / (4.0 * N) : 0.0;
    e = cudaMemsetAsync(base, 0, words, st);  // barrier and error words start at zero
    if (e == cudaSuccess) {
        k_fill_alpha<<<(nvec + 255) / 256, 256, 0, st>>>(alpha, a, nvec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_pack_vectors(vecs, io_prec, V, A, storage, vs, g, gg.L, t_first, nsl, nvec, st);
    char *result = A;
    if (e == cudaSuccess && N > 0) {
        pa.W = gg.W + (size_t)t_first * 8 * 3 * g.Ps * wfmt_bytes(gg.wfmt);
        pa.in = A;
        pa.out = B;
        pa.scr[0] = S0;
        pa.scr[1] = S1;
        pa.alpha = alpha;
        pa.g = g;
        pa.nblk = nblk;
        pa.nvec = nvec;
        pa.N = N;
        pa.vstride = vs;
        pa.wfmt = gg.wfmt;
        pa.prec = storage;
        pa.sprec = sprec;
        pa.vb = vb;
        pa.threads = threads;
        pa.bar = bar;
        pa.err = err;
        pa.budget = ctx->barrier_budget > 0 ? ctx->barrier_budget : kBudget;
        pa.stream = st;
        e = launch_persistent(pa);
        result = B;
    }
    if (e == cudaSuccess)
        e = launch_unpack_vectors(result, storage, vs, vecs, io_prec, V, g, gg.L, t_first, nsl, nvec, nullptr, nullptr,
                                  st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) return cuda_fail(e, "tls_smear_noalloc");
    if (herr & DERR_TIMEOUT)
        return fail(TLS_ERR_TIMEOUT, "tls_smear_noalloc: a bounded inter-block barrier ran out");
    if (herr) return fail(TLS_ERR_DEVICE, "tls_smear_noalloc: device error word 0x%x", herr);
    return ok();
}
