// k_layout.cu -- gauge ingest, two-link build, vector pack/unpack, norms.
//
//   ingest      canonical FP64 U[t][z][y][x][mu][3][3] -> sublattice planes
//               (bit-exact permutation; U_t is never read)
//   build       W_i(x) = U_i(x) U_i(x+i) in FP64 (Sec. 2), rounded to nearest
//               into the chosen W storage (Sec. 3: computed once, reused)
//   pack        caller vectors (FP64/FP32, canonical) -> packed storage
//   unpack      packed storage -> caller layout, with FP64 |psi|^2 partial sums
//   norms       fixed-order reduction of the partial sums (deterministic)
//
// Packed U layout: block b = t * 8 + sub, direction d, entry k = 0..8:
//   Up[((b * 3 + d) * 9 + k) * Ps + i]  (double2 = one complex entry)
#include <algorithm>

#include "tls_dev.cuh"
#include "tls_internal.h"

namespace tls {

namespace {

struct Coords {
    int x, y, z;
};

// Site i of sublattice `sub` -> spatial coordinates.
__device__ __forceinline__ Coords coords_of(const SubGeom &g, int sub, int i)
{
    int xq = i % g.hx;
    int r = i / g.hx;
    int yq = r % g.hy;
    int zq = r / g.hy;
    Coords c;
    c.x = 2 * xq + (sub & 1);
    c.y = 2 * yq + ((sub >> 1) & 1);
    c.z = 2 * zq + ((sub >> 2) & 1);
    return c;
}

// Thread per (canonical site, direction, complex entry), entry fastest: a warp
// reads 512 contiguous bytes of the canonical links (host memory over C2C
// included) and scatters them into the 9 planes of each (block, direction).
__global__ void k_ingest_gauge(const double *__restrict__ U, int nd, double2 *__restrict__ Up, SubGeom g, int Lx,
                               int Ly, int Lz, int64_t total)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int k = (int)(idx % 27);
    const int64_t site = idx / 27;
    const int d = k / 9, e = k - d * 9;
    const int x = (int)(site % Lx);
    const int64_t r1 = site / Lx;
    const int y = (int)(r1 % Ly);
    const int64_t r2 = r1 / Ly;
    const int z = (int)(r2 % Lz);
    const int t = (int)(r2 / Lz);
    const int sub = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    const int i = ((z >> 1) * g.hy + (y >> 1)) * g.hx + (x >> 1);
    const int b = t * 8 + sub;
    const double2 v = reinterpret_cast<const double2 *>(U)[(site * nd + d) * 9 + e];
    Up[(((int64_t)b * 3 + d) * 9 + e) * g.Ps + i] = v;
}

__global__ void k_export_gauge(const double2 *__restrict__ Up, double *__restrict__ out, SubGeom g, int Lx, int Ly,
                               int Lz, int64_t total)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (int)(idx % g.Vs);
    const int64_t r = idx / g.Vs;
    const int d = (int)(r % 3);
    const int b = (int)(r / 3);
    const int t = b >> 3, sub = b & 7;
    Coords c = coords_of(g, sub, i);
    const int64_t site = (((int64_t)t * Lz + c.z) * Ly + c.y) * Lx + c.x;
    double2 *dst = reinterpret_cast<double2 *>(out) + (site * 3 + d) * 9;
    const double2 *src = Up + ((int64_t)b * 3 + d) * 9 * g.Ps + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[k] = src[k * g.Ps];
}

// W_d(x) = U_d(x) U_d(x + d).  In sublattice terms x + d flips bit d of the
// sublattice index, and the half coordinate advances (with wrap) only when
// the coordinate was odd.
template <int WF, bool ONE = false>
__global__ void k_build_twolink(const double2 *__restrict__ Up, char *__restrict__ W, SubGeom g, int64_t total,
                                int *err)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (int)(idx % g.Vs);
    const int64_t r = idx / g.Vs;
    const int d = (int)(r % 3);
    const int b = (int)(r / 3);
    const int sub = b & 7;
    int fw[3], bw[3];
    sub_neighbours(g, i, fw, bw);
    const int odd = (sub >> d) & 1;
    const int ip = odd ? fw[d] : i;
    const int bp = (b & ~7) | (sub ^ (1 << d));
    const double2 *A = Up + ((int64_t)b * 3 + d) * 9 * g.Ps + i;
    const double2 *B = Up + ((int64_t)bp * 3 + d) * 9 * g.Ps + ip;
    double2 a[9], bb[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        a[k] = A[k * g.Ps];
        bb[k] = B[k * g.Ps];
    }
    double w[18];
    if constexpr (ONE) {  // one-link field: U_d(x) itself
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            w[2 * k] = a[k].x;
            w[2 * k + 1] = a[k].y;
        }
    } else {
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double2 x = a[rr * 3 + k], y = bb[k * 3 + cc];
                re = fma(x.x, y.x, re);
                re = fma(-x.y, y.y, re);
                im = fma(x.x, y.y, im);
                im = fma(x.y, y.x, im);
            }
            w[2 * (rr * 3 + cc)] = re;
            w[2 * (rr * 3 + cc) + 1] = im;
        }
    }
    char *blk = W + ((int64_t)b * 3 + d) * g.Ps * wfmt_bytes(WF);
    if constexpr (WF == W_F32_8) {
        if (!WFmt<WF>::store(blk, g.Ps, i, w)) atomicOr(err, DERR_RECON8);
    } else {
        WFmt<WF>::store(blk, g.Ps, i, w);
    }
}

template <int WF>
__global__ void k_export_twolink(const char *__restrict__ W, double *__restrict__ out, SubGeom g, int Lx, int Ly,
                                 int Lz, int64_t total)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (int)(idx % g.Vs);
    const int64_t r = idx / g.Vs;
    const int d = (int)(r % 3);
    const int b = (int)(r / 3);
    const int t = b >> 3, sub = b & 7;
    Coords c = coords_of(g, sub, i);
    const int64_t site = (((int64_t)t * Lz + c.z) * Ly + c.y) * Lx + c.x;
    typedef typename WFmt<WF>::R R;
    cpx<R> m[9];
    WFmt<WF>::load(W + ((int64_t)b * 3 + d) * g.Ps * wfmt_bytes(WF), g.Ps, i, m);
    double *dst = out + ((site * 3 + d) * 9) * 2;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        dst[2 * k] = (double)m[k].re;
        dst[2 * k + 1] = (double)m[k].im;
    }
}

template <typename IO, int VP>
__global__ void k_pack(const IO *__restrict__ src, int64_t svs, char *__restrict__ dst, int64_t dvs, SubGeom g,
                       int Lx, int Ly, int Lz, int t_first, int64_t nsite)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsite) return;
    const int v = blockIdx.y;
    const int b = (int)(s / g.Vs);
    const int i = (int)(s - (int64_t)b * g.Vs);
    const int t = t_first + (b >> 3), sub = b & 7;
    Coords c = coords_of(g, sub, i);
    const int64_t site = (((int64_t)t * Lz + c.z) * Ly + c.y) * Lx + c.x;
    const IO *p = src + ((int64_t)v * svs + site) * 6;
    typedef typename VFmt<VP>::R R;
    cpx<R> val[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        val[k].re = (R)p[2 * k];
        val[k].im = (R)p[2 * k + 1];
    }
    VFmt<VP>::template store<false>(dst + (int64_t)v * dvs + (int64_t)b * g.Ps * vfmt_bytes(VP), g.Ps, i, val);
}

template <typename IO, int VP>
__global__ void __launch_bounds__(256) k_unpack(const char *__restrict__ src, int64_t svs, IO *__restrict__ dst,
                                                int64_t dvs, SubGeom g, int Lx, int Ly, int Lz, int t_first,
                                                int64_t nsite, double *__restrict__ partials)
{
    __shared__ double red[256 / 32];
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    double n2 = 0.0;
    if (s < nsite) {
        const int b = (int)(s / g.Vs);
        const int i = (int)(s - (int64_t)b * g.Vs);
        const int t = t_first + (b >> 3), sub = b & 7;
        Coords c = coords_of(g, sub, i);
        const int64_t site = (((int64_t)t * Lz + c.z) * Ly + c.y) * Lx + c.x;
        typedef typename VFmt<VP>::R R;
        cpx<R> val[3];
        VFmt<VP>::template load<false>(src + (int64_t)v * svs + (int64_t)b * g.Ps * vfmt_bytes(VP), g.Ps, i, val);
        IO *p = dst + ((int64_t)v * dvs + site) * 6;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const IO re = (IO)val[k].re, im = (IO)val[k].im;
            p[2 * k] = re;
            p[2 * k + 1] = im;
            n2 = fma((double)re, (double)re, n2);
            n2 = fma((double)im, (double)im, n2);
        }
    }
    if (partials == nullptr) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_down_sync(0xffffffffu, n2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        partials[(int64_t)v * gridDim.x + blockIdx.x] = tot;
    }
}

// One CTA per vector sums its partials in a fixed order.
__global__ void __launch_bounds__(256) k_reduce_norms(const double *__restrict__ partials, int nparts,
                                                      double *__restrict__ norms)
{
    __shared__ double red[256];
    const int v = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) acc += partials[(int64_t)v * nparts + k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) norms[v] = red[0];
}

// Interleaved layout: CTA = (nvec, spb); threadIdx.x = vector, threadIdx.y = site.
template <typename IO, int VP>
__global__ void k_pack_il(const IO *__restrict__ src, int64_t svs, char *__restrict__ dst, SubGeom g, int Lx, int Ly,
                          int Lz, int t_first, int64_t nsite, int rec_n, int rec_v0)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= nsite) return;
    const int v = threadIdx.x;
    const int b = (int)(s / g.Vs);
    const int i = (int)(s - (int64_t)b * g.Vs);
    const int t = t_first + (b >> 3), sub = b & 7;
    Coords c = coords_of(g, sub, i);
    const int64_t site = (((int64_t)t * Lz + c.z) * Ly + c.y) * Lx + c.x;
    const IO *p = src + ((int64_t)v * svs + site) * 6;
    typedef typename VRec<VP>::R R;
    cpx<R> val[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        val[k].re = (R)p[2 * k];
        val[k].im = (R)p[2 * k + 1];
    }
    VRec<VP>::store(dst + (int64_t)b * g.Ps * rec_n * vfmt_bytes(VP) + (int64_t)i * rec_n * VRec<VP>::SB, g.Ps * rec_n,
                    rec_v0 + v, val);
}

template <typename IO, int VP>
__global__ void k_unpack_il(const char *__restrict__ src, IO *__restrict__ dst, int64_t dvs, SubGeom g, int Lx,
                            int Ly, int Lz, int t_first, int64_t nsite, int rec_n, int rec_v0)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= nsite) return;
    const int v = threadIdx.x;
    const int b = (int)(s / g.Vs);
    const int i = (int)(s - (int64_t)b * g.Vs);
    const int t = t_first + (b >> 3), sub = b & 7;
    Coords c = coords_of(g, sub, i);
    const int64_t site = (((int64_t)t * Lz + c.z) * Ly + c.y) * Lx + c.x;
    typedef typename VRec<VP>::R R;
    cpx<R> val[3];
    VRec<VP>::load(src + (int64_t)b * g.Ps * rec_n * vfmt_bytes(VP) + (int64_t)i * rec_n * VRec<VP>::SB, g.Ps * rec_n,
                   rec_v0 + v, val);
    IO *p = dst + ((int64_t)v * dvs + site) * 6;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[2 * k] = (IO)val[k].re;
        p[2 * k + 1] = (IO)val[k].im;
    }
}

// Partial sums of |psi|^2 of canonical vectors, per (vector, slice, part):
// CTA (s * kNormPartsPerSlice + p, v) takes a fixed strided subset of the
// reals of slice s of vector v, so each partial depends only on its own slice
// and the sum order is fixed.  Partial (v, s, p) goes to
// partials[v * part_stride + part_off + s * kNormPartsPerSlice + p].
template <typename IO>
__global__ void __launch_bounds__(256) k_norm_partials(const IO *__restrict__ base, int64_t vstride, int64_t slice_sites,
                                                       double *__restrict__ partials, int64_t part_stride,
                                                       int64_t part_off)
{
    __shared__ double red[256];
    const int v = blockIdx.y;
    const int sl = blockIdx.x / kNormPartsPerSlice, part = blockIdx.x - sl * kNormPartsPerSlice;
    const IO *p = base + ((int64_t)v * vstride + (int64_t)sl * slice_sites) * 6;
    const int64_t n = slice_sites * 6;
    double acc = 0.0;
    for (int64_t k = (int64_t)part * blockDim.x + threadIdx.x; k < n; k += (int64_t)kNormPartsPerSlice * blockDim.x) {
        const double x = (double)p[k];
        acc = fma(x, x, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(int64_t)v * part_stride + part_off + blockIdx.x] = red[0];
}

// Copies the interleaved records of one x'-row (hx sites starting at site r of
// block b, all rec_n vectors) between global memory and a shared-memory row
// of the same layout (colour planes hx * rec_n elements apart), 16 bytes per
// thread and step.  to_smem selects the direction.
template <int VP>
__device__ __forceinline__ void row_copy(unsigned char *smr, const void *gbase, int b, int r, const SubGeom &g, int hx,
                                         int rec_n, bool to_smem)
{
    constexpr int SB = VRec<VP>::SB;
    const int segB = hx * rec_n * SB;  // one colour (or the whole row for 16-bit records)
    const int nseg = il_planes(VP) ? 3 : 1;
    char *blk = (char *)gbase + (int64_t)b * g.Ps * rec_n * vfmt_bytes(VP);
    for (int c = 0; c < nseg; ++c) {
        uint4 *gs = reinterpret_cast<uint4 *>(blk + ((int64_t)c * g.Ps + r) * rec_n * SB);
        uint4 *ss = reinterpret_cast<uint4 *>(smr + c * segB);
        if (to_smem)
            for (int k = threadIdx.x; k < segB / 16; k += blockDim.x) ss[k] = gs[k];
        else
            for (int k = threadIdx.x; k < segB / 16; k += blockDim.x) gs[k] = ss[k];
    }
}

// Row transposes between the canonical layout and the interleaved records.
// One CTA per canonical x-row (t, z, y): the row's Lx sites are two x'-rows
// of hx records groups in sublattices (x even) and (x odd), each a contiguous
// segment of hx * nvec records.  Both segments go through shared memory so
// that the global side of either layout is read and written in contiguous
// runs (nvec canonical rows of Lx sites, two record segments).
template <typename IO, int VP>
__global__ void __launch_bounds__(256) k_unpack_rows(const char *__restrict__ src, IO *__restrict__ dst, int64_t dvs,
                                                     SubGeom g, int Lx, int Ly, int Lz, int t_first, int nvec,
                                                     int rec_n, int rec_v0)
{
    extern __shared__ __align__(16) unsigned char smr[];
    constexpr int VBY = vfmt_bytes(VP);
    const int y = blockIdx.x % Ly, z = blockIdx.x / Ly;
    const int ts = blockIdx.y;
    const int hx = g.hx;
    const int sub0 = ((y & 1) << 1) | ((z & 1) << 2);
    const int r = ((z >> 1) * g.hy + (y >> 1)) * hx;
    const int segB = hx * rec_n * VBY;
    // stage both x'-rows (all rec_n records) with 16-byte loads
    for (int par = 0; par < 2; ++par) row_copy<VP>(smr + par * segB, src, ts * 8 + (sub0 | par), r, g, hx, rec_n, true);
    __syncthreads();
    typedef typename VRec<VP>::R R;
    const int64_t site0 = (((int64_t)(t_first + ts) * Lz + z) * Ly + y) * Lx;
    for (int k = threadIdx.x; k < nvec * Lx; k += blockDim.x) {
        const int v = k / Lx, x = k - v * Lx;
        cpx<R> val[3];
        VRec<VP>::load(reinterpret_cast<const char *>(smr) + (x & 1) * segB + (x >> 1) * rec_n * VRec<VP>::SB, hx * rec_n,
                       rec_v0 + v, val);
        IO *p = dst + ((int64_t)v * dvs + site0 + x) * 6;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p[2 * c] = (IO)val[c].re;
            p[2 * c + 1] = (IO)val[c].im;
        }
    }
}

template <typename IO, int VP>
__global__ void __launch_bounds__(256) k_pack_rows(const IO *__restrict__ src, int64_t svs, char *__restrict__ dst,
                                                   SubGeom g, int Lx, int Ly, int Lz, int t_first, int nvec, int rec_n,
                                                   int rec_v0)
{
    extern __shared__ __align__(16) unsigned char smr[];
    constexpr int VBY = vfmt_bytes(VP);
    const int y = blockIdx.x % Ly, z = blockIdx.x / Ly;
    const int ts = blockIdx.y;
    const int hx = g.hx;
    const int sub0 = ((y & 1) << 1) | ((z & 1) << 2);
    const int r = ((z >> 1) * g.hy + (y >> 1)) * hx;
    const int segB = hx * rec_n * VBY;
    const bool partial = nvec != rec_n;
    if (partial) {  // keep the records of the other slots: start from the current segments
        for (int par = 0; par < 2; ++par)
            row_copy<VP>(smr + par * segB, dst, ts * 8 + (sub0 | par), r, g, hx, rec_n, true);
        __syncthreads();
    }
    typedef typename VRec<VP>::R R;
    const int64_t site0 = (((int64_t)(t_first + ts) * Lz + z) * Ly + y) * Lx;
    for (int k = threadIdx.x; k < nvec * Lx; k += blockDim.x) {
        const int v = k / Lx, x = k - v * Lx;
        const IO *p = src + ((int64_t)v * svs + site0 + x) * 6;
        cpx<R> val[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            val[c].re = (R)p[2 * c];
            val[c].im = (R)p[2 * c + 1];
        }
        VRec<VP>::store(reinterpret_cast<char *>(smr) + (x & 1) * segB + (x >> 1) * rec_n * VRec<VP>::SB, hx * rec_n,
                        rec_v0 + v, val);
    }
    __syncthreads();
    for (int par = 0; par < 2; ++par)
        row_copy<VP>(smr + par * segB, dst, ts * 8 + (sub0 | par), r, g, hx, rec_n, false);
}

inline int spb_of(int nvec) { return std::max(1, 256 / nvec); }

inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename IO>
cudaError_t pack_io(const IO *src, int64_t svs, char *dst, int prec, int64_t dvs, const SubGeom &g, const int L[4],
                    int t_first, int64_t nsite, int nvec, cudaStream_t s)
{
    dim3 grid(nblocks(nsite, 256), nvec);
    switch (prec) {
    case P_F64: k_pack<IO, P_F64><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite); break;
    case P_F32: k_pack<IO, P_F32><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite); break;
    case P_F16: k_pack<IO, P_F16><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite); break;
    case P_BF16: k_pack<IO, P_BF16><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

template <typename IO>
cudaError_t unpack_io(const char *src, int prec, int64_t svs, IO *dst, int64_t dvs, const SubGeom &g, const int L[4],
                      int t_first, int64_t nsite, int nvec, double *partials, cudaStream_t s)
{
    dim3 grid(nblocks(nsite, 256), nvec);
    switch (prec) {
    case P_F64: k_unpack<IO, P_F64><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, partials); break;
    case P_F32: k_unpack<IO, P_F32><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, partials); break;
    case P_F16: k_unpack<IO, P_F16><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, partials); break;
    case P_BF16: k_unpack<IO, P_BF16><<<grid, 256, 0, s>>>(src, svs, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, partials); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ingest_gauge(const double *U, int nd, double *Up, const SubGeom &g, const int L[4], cudaStream_t s)
{
    const int64_t total = (int64_t)L[0] * L[1] * L[2] * L[3] * 27;
    if (total == 0) return cudaSuccess;
    k_ingest_gauge<<<nblocks(total, 256), 256, 0, s>>>(U, nd, reinterpret_cast<double2 *>(Up), g, L[0], L[1], L[2],
                                                       total);
    return cudaGetLastError();
}

cudaError_t launch_export_gauge(const double *Up, double *out, const SubGeom &g, const int L[4], cudaStream_t s)
{
    const int64_t total = (int64_t)L[3] * 8 * 3 * g.Vs;
    if (total == 0) return cudaSuccess;
    k_export_gauge<<<nblocks(total, 256), 256, 0, s>>>(reinterpret_cast<const double2 *>(Up), out, g, L[0], L[1],
                                                       L[2], total);
    return cudaGetLastError();
}

cudaError_t launch_build_twolink(const double *Up, char *W, int wfmt, const SubGeom &g, int nblk, int *err,
                                 cudaStream_t s)
{
    const int64_t total = (int64_t)nblk * 3 * g.Vs;
    if (total == 0) return cudaSuccess;
    const double2 *u = reinterpret_cast<const double2 *>(Up);
    const unsigned nb = nblocks(total, 128);
    switch (wfmt) {
    case W_F64_18: k_build_twolink<W_F64_18><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_F32_18: k_build_twolink<W_F32_18><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_F32_12: k_build_twolink<W_F32_12><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_F32_8: k_build_twolink<W_F32_8><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_F16_18: k_build_twolink<W_F16_18><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_F16_12: k_build_twolink<W_F16_12><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_BF16_18: k_build_twolink<W_BF16_18><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    case W_BF16_12: k_build_twolink<W_BF16_12><<<nb, 128, 0, s>>>(u, W, g, total, err); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_build_links(const double *Up, char *L1, int wfmt, const SubGeom &g, int nblk, cudaStream_t s)
{
    const int64_t total = (int64_t)nblk * 3 * g.Vs;
    if (total == 0) return cudaSuccess;
    const double2 *u = reinterpret_cast<const double2 *>(Up);
    const unsigned nb = nblocks(total, 128);
    switch (wfmt) {
    case W_F64_18: k_build_twolink<W_F64_18, true><<<nb, 128, 0, s>>>(u, L1, g, total, nullptr); break;
    case W_F32_18: k_build_twolink<W_F32_18, true><<<nb, 128, 0, s>>>(u, L1, g, total, nullptr); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_twolink(const char *W, int wfmt, double *out, const SubGeom &g, const int L[4],
                                  cudaStream_t s)
{
    const int64_t total = (int64_t)L[3] * 8 * 3 * g.Vs;
    if (total == 0) return cudaSuccess;
    const unsigned nb = nblocks(total, 128);
    switch (wfmt) {
    case W_F64_18: k_export_twolink<W_F64_18><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_F32_18: k_export_twolink<W_F32_18><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_F32_12: k_export_twolink<W_F32_12><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_F32_8: k_export_twolink<W_F32_8><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_F16_18: k_export_twolink<W_F16_18><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_F16_12: k_export_twolink<W_F16_12><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_BF16_18: k_export_twolink<W_BF16_18><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    case W_BF16_12: k_export_twolink<W_BF16_12><<<nb, 128, 0, s>>>(W, out, g, L[0], L[1], L[2], total); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_vectors(const void *src, int io_prec, int64_t src_vstride_sites, char *dst, int prec,
                                int64_t dst_vstride, const SubGeom &g, const int L[4], int t_first, int nsl,
                                int nvec, cudaStream_t s)
{
    const int64_t nsite = (int64_t)nsl * 8 * g.Vs;
    if (nsite == 0 || nvec == 0) return cudaSuccess;
    if (io_prec == P_F64)
        return pack_io<double>((const double *)src, src_vstride_sites, dst, prec, dst_vstride, g, L, t_first, nsite,
                               nvec, s);
    if (io_prec == P_F32)
        return pack_io<float>((const float *)src, src_vstride_sites, dst, prec, dst_vstride, g, L, t_first, nsite,
                              nvec, s);
    return cudaErrorNotSupported;
}

int unpack_parts(const SubGeom &g, int nsl) { return (int)nblocks((int64_t)nsl * 8 * g.Vs, 256); }

cudaError_t launch_unpack_vectors(const char *src, int prec, int64_t src_vstride, void *dst, int io_prec,
                                  int64_t dst_vstride_sites, const SubGeom &g, const int L[4], int t_first,
                                  int nsl, int nvec, double *partials, int *nparts, cudaStream_t s)
{
    const int64_t nsite = (int64_t)nsl * 8 * g.Vs;
    if (nparts) *nparts = unpack_parts(g, nsl);
    if (nsite == 0 || nvec == 0) return cudaSuccess;
    if (io_prec == P_F64)
        return unpack_io<double>(src, prec, src_vstride, (double *)dst, dst_vstride_sites, g, L, t_first, nsite,
                                 nvec, partials, s);
    if (io_prec == P_F32)
        return unpack_io<float>(src, prec, src_vstride, (float *)dst, dst_vstride_sites, g, L, t_first, nsite, nvec,
                                partials, s);
    return cudaErrorNotSupported;
}

template <typename IO>
static cudaError_t pack_il_io(const IO *src, int64_t svs, char *dst, int prec, const SubGeom &g, const int L[4],
                              int t_first, int64_t nsite, int nvec, int rec_n, int rec_v0, cudaStream_t s)
{
    const int spb = spb_of(nvec);
    dim3 block(nvec, spb), grid(nblocks(nsite, spb));
    switch (prec) {
    case P_F64: k_pack_il<IO, P_F64><<<grid, block, 0, s>>>(src, svs, dst, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    case P_F32: k_pack_il<IO, P_F32><<<grid, block, 0, s>>>(src, svs, dst, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    case P_F16: k_pack_il<IO, P_F16><<<grid, block, 0, s>>>(src, svs, dst, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    case P_BF16: k_pack_il<IO, P_BF16><<<grid, block, 0, s>>>(src, svs, dst, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

template <typename IO>
static cudaError_t unpack_il_io(const char *src, int prec, IO *dst, int64_t dvs, const SubGeom &g, const int L[4],
                                int t_first, int64_t nsite, int nvec, int rec_n, int rec_v0, cudaStream_t s)
{
    const int spb = spb_of(nvec);
    dim3 block(nvec, spb), grid(nblocks(nsite, spb));
    switch (prec) {
    case P_F64: k_unpack_il<IO, P_F64><<<grid, block, 0, s>>>(src, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    case P_F32: k_unpack_il<IO, P_F32><<<grid, block, 0, s>>>(src, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    case P_F16: k_unpack_il<IO, P_F16><<<grid, block, 0, s>>>(src, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    case P_BF16: k_unpack_il<IO, P_BF16><<<grid, block, 0, s>>>(src, dst, dvs, g, L[0], L[1], L[2], t_first, nsite, rec_n, rec_v0); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

bool rows_transpose_ok(const SubGeom &g, int rec_n, int prec, const int L[4])
{
    // each colour plane's (or the 16-bit row's) segment is copied in 16-byte words
    const int colB = g.hx * rec_n * il_site_bytes(prec);
    const int rowB = g.hx * rec_n * vfmt_bytes(prec);
    return colB % 16 == 0 && 2 * rowB <= 48 * 1024 && (int64_t)L[1] * L[2] <= 0x7fffffff;
}

template <typename IO>
static cudaError_t rows_io(bool pack, const void *src, int64_t svs, void *dst, int prec, const SubGeom &g,
                           const int L[4], int t_first, int nsl, int nvec, int rec_n, int rec_v0, cudaStream_t s)
{
    dim3 grid((unsigned)(L[1] * L[2]), nsl);
    const int smem = 2 * g.hx * rec_n * vfmt_bytes(prec);
#define TLS_ROWS_CASE(P)                                                                                            \
    case P:                                                                                                         \
        if (pack)                                                                                                   \
            k_pack_rows<IO, P><<<grid, 256, smem, s>>>((const IO *)src, svs, (char *)dst, g, L[0], L[1], L[2],       \
                                                      t_first, nvec, rec_n, rec_v0);                                \
        else                                                                                                        \
            k_unpack_rows<IO, P><<<grid, 256, smem, s>>>((const char *)src, (IO *)dst, svs, g, L[0], L[1], L[2],     \
                                                        t_first, nvec, rec_n, rec_v0);                              \
        break;
    switch (prec) {
        TLS_ROWS_CASE(P_F64)
        TLS_ROWS_CASE(P_F32)
        TLS_ROWS_CASE(P_F16)
        TLS_ROWS_CASE(P_BF16)
    default: return cudaErrorNotSupported;
    }
#undef TLS_ROWS_CASE
    return cudaGetLastError();
}

cudaError_t launch_pack_il(const void *src, int io_prec, int64_t src_vstride_sites, char *dst, int prec,
                           const SubGeom &g, const int L[4], int t_first, int nsl, int nvec, int rec_n, int rec_v0,
                           cudaStream_t s)
{
    const int64_t nsite = (int64_t)nsl * 8 * g.Vs;
    if (nsite == 0 || nvec == 0) return cudaSuccess;
    if (nvec > 256 || rec_v0 < 0 || rec_v0 + nvec > rec_n) return cudaErrorInvalidValue;
    if (rows_transpose_ok(g, rec_n, prec, L)) {
        if (io_prec == P_F64)
            return rows_io<double>(true, src, src_vstride_sites, dst, prec, g, L, t_first, nsl, nvec, rec_n, rec_v0, s);
        if (io_prec == P_F32)
            return rows_io<float>(true, src, src_vstride_sites, dst, prec, g, L, t_first, nsl, nvec, rec_n, rec_v0, s);
    }
    if (io_prec == P_F64)
        return pack_il_io<double>((const double *)src, src_vstride_sites, dst, prec, g, L, t_first, nsite, nvec, rec_n,
                                  rec_v0, s);
    if (io_prec == P_F32)
        return pack_il_io<float>((const float *)src, src_vstride_sites, dst, prec, g, L, t_first, nsite, nvec, rec_n,
                                 rec_v0, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_unpack_il(const char *src, int prec, void *dst, int io_prec, int64_t dst_vstride_sites,
                             const SubGeom &g, const int L[4], int t_first, int nsl, int nvec, int rec_n, int rec_v0,
                             cudaStream_t s)
{
    const int64_t nsite = (int64_t)nsl * 8 * g.Vs;
    if (nsite == 0 || nvec == 0) return cudaSuccess;
    if (nvec > 256 || rec_v0 < 0 || rec_v0 + nvec > rec_n) return cudaErrorInvalidValue;
    if (rows_transpose_ok(g, rec_n, prec, L)) {
        if (io_prec == P_F64)
            return rows_io<double>(false, src, dst_vstride_sites, dst, prec, g, L, t_first, nsl, nvec, rec_n, rec_v0, s);
        if (io_prec == P_F32)
            return rows_io<float>(false, src, dst_vstride_sites, dst, prec, g, L, t_first, nsl, nvec, rec_n, rec_v0, s);
    }
    if (io_prec == P_F64)
        return unpack_il_io<double>(src, prec, (double *)dst, dst_vstride_sites, g, L, t_first, nsite, nvec, rec_n,
                                    rec_v0, s);
    if (io_prec == P_F32)
        return unpack_il_io<float>(src, prec, (float *)dst, dst_vstride_sites, g, L, t_first, nsite, nvec, rec_n,
                                   rec_v0, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_norm_partials(const void *base, int io_prec, int64_t vstride_sites, int64_t slice_sites, int nsl,
                                 int nvec, double *partials, int64_t part_stride, int64_t part_off, cudaStream_t s)
{
    if (nvec == 0 || nsl == 0) return cudaSuccess;
    if ((int64_t)nsl * kNormPartsPerSlice > 0x7fffffff || nvec > 65535) return cudaErrorInvalidValue;
    dim3 grid(nsl * kNormPartsPerSlice, nvec);
    if (io_prec == P_F64)
        k_norm_partials<double><<<grid, 256, 0, s>>>((const double *)base, vstride_sites, slice_sites, partials,
                                                      part_stride, part_off);
    else if (io_prec == P_F32)
        k_norm_partials<float><<<grid, 256, 0, s>>>((const float *)base, vstride_sites, slice_sites, partials,
                                                     part_stride, part_off);
    else
        return cudaErrorNotSupported;
    return cudaGetLastError();
}

cudaError_t launch_reduce_norms(const double *partials, int nparts, int nvec, double *norms, cudaStream_t s)
{
    if (nvec == 0) return cudaSuccess;
    k_reduce_norms<<<nvec, 256, 0, s>>>(partials, nparts, norms);
    return cudaGetLastError();
}

}  // namespace tls
