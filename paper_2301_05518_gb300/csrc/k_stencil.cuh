// k_stencil.cuh -- the two-link Laplacian fused with the smearing update.
//
// One smearing step (Sec. 2, Eq. tlSmear with Eq. tlLapl1):
//   psi'(x) = psi(x) + alpha [ sum_i W_i(x) psi(x+2i) + W_i^dag(x-2i) psi(x-2i)
//                              - 6 psi(x) ],            alpha = sigma / (4N)
// evaluated out of place.  In the sublattice layout (tls_dev.cuh) the +-2 hops
// are +-1 steps inside one (slice, sublattice) block, so every operand of a
// site lives in its own block.
//
// Work decomposition: a warp owns 32 consecutive sites of one block and a
// chunk of VB vectors; the nchunk = ceil(nvec / VB) warps of the same 32 sites
// are adjacent, so W(x) and W(x-2i) come from DRAM once and are shared through
// L1/L2 by all vectors (multi-right-hand-side).  VB = 1 with nvec = 1 is the
// plain single-vector form.
//
// This header is included by one translation unit per vector precision
// (k_step_<prec>.cu) with TLS_VP defined.
#pragma once

#include <algorithm>

#include "k_ilt.cuh"
#include "tls_dev.cuh"
#include "tls_internal.h"

namespace tls {

template <int VP, int WF> __host__ __device__ constexpr bool combo_ok()
{
    return VP == P_F64   ? WF == W_F64_18
         : VP == P_F32   ? (WF == W_F32_18 || WF == W_F32_12 || WF == W_F32_8)
         : VP == P_F16   ? (WF == W_F32_18 || WF == W_F32_12 || WF == W_F16_18 || WF == W_F16_12)
         : VP == P_BF16  ? (WF == W_F32_18 || WF == W_F32_12 || WF == W_BF16_18 || WF == W_BF16_12)
                         : false;
}

// Scratch precision of the persistent kernel: FP64 stays FP64, everything
// else keeps FP32 iterates between steps.
template <int VP> __host__ __device__ constexpr int scratch_prec() { return VP == P_F64 ? P_F64 : P_F32; }

// One site, VB vectors starting at v0.  bin / bout are the byte offsets of the
// site's block in `in` / `out` (vector 0); wblk is the absolute block for W.
template <int VPI, int VPO, int WF, int VB, bool CGI, bool CGO>
__device__ __forceinline__ void site_step(const char *__restrict__ W, const char *__restrict__ in,
                                          char *__restrict__ out, const double *__restrict__ alpha,
                                          const SubGeom &g, int wblk, int i, int v0, int nvec, int64_t vs_in,
                                          int64_t vs_out, int64_t bin, int64_t bout,
                                          const int *__restrict__ active = nullptr)
{
    typedef typename VFmt<VPI>::R R;
    constexpr int WB = wfmt_bytes(WF);
    int fw[3], bw[3];
    sub_neighbours(g, i, fw, bw);
    const char *wb = W + (int64_t)wblk * 3 * g.Ps * WB;
    const char *ib = in + bin;
    bool on[VB];
    bool any = false;
#pragma unroll
    for (int v = 0; v < VB; ++v) {
        on[v] = v0 + v < nvec && (active == nullptr || active[v0 + v] != 0);
        any = any || on[v];
    }
    if (!any) return;
    cpx<R> acc[VB][3];
#pragma unroll
    for (int v = 0; v < VB; ++v)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[v][c].re = acc[v][c].im = R(0);

#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cpx<R> m[9];
        WFmt<WF>::load(wb + d * g.Ps * WB, g.Ps, i, m);
#pragma unroll
        for (int v = 0; v < VB; ++v) {
            if (on[v]) {
                cpx<R> p[3];
                VFmt<VPI>::template load<CGI>(ib + (int64_t)(v0 + v) * vs_in, g.Ps, fw[d], p);
                mv_add(m, p, acc[v]);
            }
        }
        WFmt<WF>::load(wb + d * g.Ps * WB, g.Ps, bw[d], m);
#pragma unroll
        for (int v = 0; v < VB; ++v) {
            if (on[v]) {
                cpx<R> p[3];
                VFmt<VPI>::template load<CGI>(ib + (int64_t)(v0 + v) * vs_in, g.Ps, bw[d], p);
                mdv_add(m, p, acc[v]);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < VB; ++v) {
        if (on[v]) {
            cpx<R> c[3], o[3];
            VFmt<VPI>::template load<CGI>(ib + (int64_t)(v0 + v) * vs_in, g.Ps, i, c);
            const R a = (R)alpha[v0 + v];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o[k].re = fma(a, fma(R(-6), c[k].re, acc[v][k].re), c[k].re);
                o[k].im = fma(a, fma(R(-6), c[k].im, acc[v][k].im), c[k].im);
            }
            VFmt<VPO>::template store<CGO>(out + bout + (int64_t)(v0 + v) * vs_out, g.Ps, i, o);
        }
    }
}

// Work item w -> (site, chunk): warps own 32 consecutive sites, the nchunk
// warps of one 32-site tile are consecutive.
__device__ __forceinline__ void item_of(int64_t w, int nchunk, int64_t &site, int &chunk)
{
    int64_t tile = w / (32 * nchunk);
    int r = (int)(w - tile * 32 * nchunk);
    chunk = r >> 5;
    site = tile * 32 + (r & 31);
}

template <int VP, int WF, int VB>
__global__ void __launch_bounds__(256) k_step(const char *__restrict__ W, const char *__restrict__ in,
                                              char *__restrict__ out, const double *__restrict__ alpha,
                                              const int *__restrict__ active, SubGeom g, int nblk, int nvec,
                                              int64_t vs_in, int64_t vs_out)
{
    const int nchunk = (nvec + VB - 1) / VB;
    int64_t site;
    int chunk;
    item_of((int64_t)blockIdx.x * blockDim.x + threadIdx.x, nchunk, site, chunk);
    if (site >= (int64_t)nblk * g.Vs) return;
    const int blk = (int)(site / g.Vs);
    const int i = (int)(site - (int64_t)blk * g.Vs);
    constexpr int VBY = vfmt_bytes(VP);
    const int64_t boff = (int64_t)blk * g.Ps * VBY;
    site_step<VP, VP, WF, VB, false, false>(W, in, out, alpha, g, blk, i, chunk * VB, nvec, vs_in, vs_out, boff,
                                            boff, active);
}

// --------------------------------------------------------------------------
// Multi-RHS step on the interleaved layout (vectors innermost).
// CTA = (nvec, spb) threads: threadIdx.x is the vector, threadIdx.y one of
// spb consecutive sites along x' of the row (y' = blockIdx.y, z' and the
// block from blockIdx.z).  All lanes of a site read the same W words (one
// broadcast), and the records of consecutive (site, vector) pairs are
// contiguous, so every vector load and store is coalesced.  No index
// division: the neighbours come from the grid coordinates.  The arithmetic
// per vector is the same sequence as site_step, so results are bitwise equal
// to the planar kernels.
// --------------------------------------------------------------------------
template <int VP, int WF, int VB>
__device__ __forceinline__ void step_il_body(const char *__restrict__ W, const char *__restrict__ in,
                                             char *__restrict__ out, const double *__restrict__ alpha,
                                             const int *__restrict__ active, const SubGeom &g, int nvec)
{
    typedef typename VRec<VP>::R R;
    constexpr int WB = wfmt_bytes(WF);
    constexpr int VBY = vfmt_bytes(VP);
    const int t = threadIdx.x, T = nvec / VB;  // nvec is a multiple of VB
    const int xq = blockIdx.x * blockDim.y + threadIdx.y;
    if (xq >= g.hx) return;
    bool on[VB];
    bool any = false;
#pragma unroll
    for (int k = 0; k < VB; ++k) {
        on[k] = active == nullptr || active[il_vec<VP, VB>(t, T, k)] != 0;
        any = any || on[k];
    }
    if (!any) return;
    const int yq = blockIdx.y;
    const int blk = blockIdx.z / g.hz;
    const int zq = blockIdx.z - blk * g.hz;
    const int sy = g.hx, sz = g.hx * g.hy;
    const int i = zq * sz + yq * sy + xq;
    int fw[3], bw[3];
    fw[0] = xq == g.hx - 1 ? i - (g.hx - 1) : i + 1;
    bw[0] = xq == 0 ? i + (g.hx - 1) : i - 1;
    fw[1] = yq == g.hy - 1 ? i - (g.hy - 1) * sy : i + sy;
    bw[1] = yq == 0 ? i + (g.hy - 1) * sy : i - sy;
    fw[2] = zq == g.hz - 1 ? i - (g.hz - 1) * sz : i + sz;
    bw[2] = zq == 0 ? i + (g.hz - 1) * sz : i - sz;
    const char *wb = W + (int64_t)blk * 3 * g.Ps * WB;
    // record group of site s of this block at rin + s * nvec * VBY
    const char *rin = in + (int64_t)blk * g.Ps * nvec * VBY;
    char *rout = out + (int64_t)blk * g.Ps * nvec * VBY;
    const unsigned rstride = (unsigned)nvec * VRec<VP>::SB;  // site stride
    const int cs = g.Ps * nvec;                                    // colour planes
    cpx<R> acc[VB][3];
#pragma unroll
    for (int k = 0; k < VB; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[k][c].re = acc[k][c].im = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cpx<R> m[9], p[VB][3];
        WFmt<WF>::load(wb + d * g.Ps * WB, g.Ps, i, m);
        RecGroup<VP, VB>::load(rin + (unsigned)fw[d] * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mv_add(m, p[k], acc[k]);
        WFmt<WF>::load(wb + d * g.Ps * WB, g.Ps, bw[d], m);
        RecGroup<VP, VB>::load(rin + (unsigned)bw[d] * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mdv_add(m, p[k], acc[k]);
    }
    cpx<R> c[VB][3], o[VB][3];
    RecGroup<VP, VB>::load(rin + (unsigned)i * rstride, cs, t, T, c);
#pragma unroll
    for (int k = 0; k < VB; ++k) {
        const R a = (R)alpha[il_vec<VP, VB>(t, T, k)];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            o[k][q].re = fma(a, fma(R(-6), c[k][q].re, acc[k][q].re), c[k][q].re);
            o[k][q].im = fma(a, fma(R(-6), c[k][q].im, acc[k][q].im), c[k][q].im);
        }
        if (!on[k]) {
#pragma unroll
            for (int q = 0; q < 3; ++q) o[k][q] = c[k][q];
        }
    }
    if (VB == 1 || (on[0] && on[VB - 1] && [&] {
            bool all = true;
#pragma unroll
            for (int k = 0; k < VB; ++k) all = all && on[k];
            return all;
        }())) {
        RecGroup<VP, VB>::store(rout + (unsigned)i * rstride, cs, t, T, o);
    } else {
#pragma unroll
        for (int k = 0; k < VB; ++k)
            if (on[k]) VRec<VP>::store(rout + (unsigned)i * rstride, cs, il_vec<VP, VB>(t, T, k), o[k]);
    }
}

template <int VP, int WF, int VB>
__global__ void __launch_bounds__(256) k_step_il(const char *__restrict__ W, const char *__restrict__ in,
                                                 char *__restrict__ out, const double *__restrict__ alpha,
                                                 const int *__restrict__ active, SubGeom g, int nvec)
{
    step_il_body<VP, WF, VB>(W, in, out, alpha, active, g, nvec);
}

// The same kernel held to 64 registers (CTAs of at most 128 threads, 8 per
// SM): more warps in flight for the latency of the neighbour loads.
template <int VP, int WF, int VB>
__global__ void __launch_bounds__(128, 8) k_step_il_occ(const char *__restrict__ W, const char *__restrict__ in,
                                                        char *__restrict__ out, const double *__restrict__ alpha,
                                                        const int *__restrict__ active, SubGeom g, int nvec)
{
    step_il_body<VP, WF, VB>(W, in, out, alpha, active, g, nvec);
}

// alpha of vector v in the arithmetic precision: FP32 kernels read the copy
// rounded to FP32 beforehand (the same value as converting the FP64 one).
template <typename R>
__device__ __forceinline__ R alpha_of(const double *__restrict__ alpha, const float *__restrict__ alphaf, int v)
{
    if constexpr (sizeof(R) == 4)
        return alphaf[v];
    else
        return (R)alpha[v];
}

// Packed FP32 pair forms of mv_add / mdv_add for VB vectors: every (re, im)
// accumulator gets, lane by lane, the FMA sequence of cmac / cmacc, with the
// broadcast W pairs built once per element for all VB vectors.

template <int VB>
__device__ __forceinline__ void mv_add_x2(const cpx<float> m[9], const cpx<float> p[VB][3], float2 acc[VB][3])
{
    float2 pp[VB][3], ps[VB][3];
#pragma unroll
    for (int v = 0; v < VB; ++v)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pp[v][c] = make_float2(p[v][c].re, p[v][c].im);
            ps[v][c] = f2swap(pp[v][c]);
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cpx<float> w = m[r * 3 + c];
            const float2 wa = make_float2(w.re, w.re), wc = make_float2(-w.im, w.im);
#pragma unroll
            for (int v = 0; v < VB; ++v) {
                acc[v][r] = __ffma2_rn(wa, pp[v][c], acc[v][r]);
                acc[v][r] = __ffma2_rn(wc, ps[v][c], acc[v][r]);
            }
        }
}

template <int VB>
__device__ __forceinline__ void mdv_add_x2(const cpx<float> m[9], const cpx<float> p[VB][3], float2 acc[VB][3])
{
    float2 pp[VB][3], ps[VB][3];
#pragma unroll
    for (int v = 0; v < VB; ++v)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pp[v][c] = make_float2(p[v][c].re, p[v][c].im);
            ps[v][c] = f2swap(pp[v][c]);
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cpx<float> w = m[c * 3 + r];
            const float2 wa = make_float2(w.re, w.re), wc = make_float2(w.im, -w.im);
#pragma unroll
            for (int v = 0; v < VB; ++v) {
                acc[v][r] = __ffma2_rn(wa, pp[v][c], acc[v][r]);
                acc[v][r] = __ffma2_rn(wc, ps[v][c], acc[v][r]);
            }
        }
}

// --------------------------------------------------------------------------
// Interleaved multi-RHS step with the strip's W staged in shared memory.
// The CTA's spb sites need six W matrices each (W_d(x) and W_d(x - 2d) for
// d = x, y, z).  They are copied once per CTA into shared memory, in the same
// plane layout with plane stride spb, and every thread of a site reads them
// from there: one cooperative copy instead of 30 global loads per thread.
// Same FMA sequence as site_step.
// --------------------------------------------------------------------------
template <int VP, int WF, int VB, bool PK>
__global__ void __launch_bounds__(256) k_step_ilw(const char *__restrict__ W, const char *__restrict__ in,
                                                  char *__restrict__ out, const double *__restrict__ alpha,
                                                  const float *__restrict__ alphaf, SubGeom g, int nvec)
{
    typedef typename VRec<VP>::R R;
    constexpr int WB = wfmt_bytes(WF);
    constexpr int VBY = vfmt_bytes(VP);
    constexpr int NQ = WB / 16, REM = WB % 16;
    extern __shared__ __align__(16) unsigned char wsm[];
    const int spb = blockDim.y;
    const int x0 = blockIdx.x * spb;
    const int yq = blockIdx.y;
    const int blk = blockIdx.z / g.hz;
    const int zq = blockIdx.z - blk * g.hz;
    const int sy = g.hx, sz = g.hx * g.hy;
    const int row = zq * sz + yq * sy;
    const int ym = yq == 0 ? g.hy - 1 : yq - 1;
    const int zm = zq == 0 ? g.hz - 1 : zq - 1;
    const char *wb = W + (int64_t)blk * 3 * g.Ps * WB;
    const int nsite = min(spb, g.hx - x0);
    // set q = 0..5: (fwd x, bwd x, fwd y, bwd y, fwd z, bwd z), site k -> global site
    auto gsite = [&](int q, int k) {
        const int xq = x0 + k;
        switch (q) {
        case 1: return row + (xq == 0 ? g.hx - 1 : xq - 1);
        case 3: return zq * sz + ym * sy + xq;
        case 5: return zm * sz + yq * sy + xq;
        default: return row + xq;
        }
    };
    const int setB = (spb * WB + 15) / 16 * 16;  // one set: planes of spb words, 16-byte aligned
    {
        constexpr int words = NQ + (REM ? 1 : 0);
        const int total = 6 * nsite * words;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        // site index fastest: consecutive lanes copy consecutive words of one plane
        for (int e = tid; e < total; e += blockDim.x * blockDim.y) {
            const int r = e / nsite;
            const int k = e - r * nsite;
            const int q = r / words;
            const int j = r - q * words;
            const int d = q >> 1;
            const char *src = wb + (int64_t)d * g.Ps * WB;
            char *dst = reinterpret_cast<char *>(wsm) + q * setB;
            const int gi = gsite(q, k);
            if (j < NQ)
                reinterpret_cast<uint4 *>(dst)[j * spb + k] = reinterpret_cast<const uint4 *>(src)[(int64_t)j * g.Ps + gi];
            else if (REM == 8)
                reinterpret_cast<uint2 *>(dst + NQ * spb * 16)[k] =
                    reinterpret_cast<const uint2 *>(src + (int64_t)NQ * g.Ps * 16)[gi];
            else
                reinterpret_cast<uint32_t *>(dst + NQ * spb * 16)[k] =
                    reinterpret_cast<const uint32_t *>(src + (int64_t)NQ * g.Ps * 16)[gi];
        }
    }
    __syncthreads();
    const int k = threadIdx.y;
    if (k >= nsite) return;
    const int t = threadIdx.x, T = nvec / VB;
    const int xq = x0 + k;
    const int i = row + xq;
    int fw[3], bw[3];
    fw[0] = xq == g.hx - 1 ? i - (g.hx - 1) : i + 1;
    bw[0] = xq == 0 ? i + (g.hx - 1) : i - 1;
    fw[1] = yq == g.hy - 1 ? i - (g.hy - 1) * sy : i + sy;
    bw[1] = yq == 0 ? i + (g.hy - 1) * sy : i - sy;
    fw[2] = zq == g.hz - 1 ? i - (g.hz - 1) * sz : i + sz;
    bw[2] = zq == 0 ? i + (g.hz - 1) * sz : i - sz;
    const char *rin = in + (int64_t)blk * g.Ps * nvec * VBY;
    char *rout = out + (int64_t)blk * g.Ps * nvec * VBY;
    const unsigned rstride = (unsigned)nvec * VRec<VP>::SB;  // site stride
    const int cs = g.Ps * nvec;                                    // colour planes
    const char *ws = reinterpret_cast<const char *>(wsm);
    cpx<R> c[VB][3], o[VB][3];
    if constexpr (PK) {
        // packed FP32 pairs: the same FMA sequence lane by lane (VP is not FP64)
        float2 acc[VB][3];
#pragma unroll
        for (int kk = 0; kk < VB; ++kk)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[kk][q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cpx<float> m[9], p[VB][3];
            WFmt<WF>::load(ws + (2 * d) * setB, spb, k, m);
            RecGroup<VP, VB>::load(rin + (unsigned)fw[d] * rstride, cs, t, T, p);
            mv_add_x2<VB>(m, p, acc);
            WFmt<WF>::load(ws + (2 * d + 1) * setB, spb, k, m);
            RecGroup<VP, VB>::load(rin + (unsigned)bw[d] * rstride, cs, t, T, p);
            mdv_add_x2<VB>(m, p, acc);
        }
        RecGroup<VP, VB>::load(rin + (unsigned)i * rstride, cs, t, T, c);
        const float2 m6 = make_float2(-6.f, -6.f);
#pragma unroll
        for (int kk = 0; kk < VB; ++kk) {
            const float a = alphaf[il_vec<VP, VB>(t, T, kk)];
            const float2 a2 = make_float2(a, a);
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float2 c2 = make_float2(c[kk][q].re, c[kk][q].im);
                const float2 u = __ffma2_rn(a2, __ffma2_rn(m6, c2, acc[kk][q]), c2);
                o[kk][q].re = u.x;
                o[kk][q].im = u.y;
            }
        }
    } else {
        cpx<R> acc[VB][3];
#pragma unroll
        for (int kk = 0; kk < VB; ++kk)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[kk][q].re = acc[kk][q].im = R(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cpx<R> m[9], p[VB][3];
            WFmt<WF>::load(ws + (2 * d) * setB, spb, k, m);
            RecGroup<VP, VB>::load(rin + (unsigned)fw[d] * rstride, cs, t, T, p);
#pragma unroll
            for (int kk = 0; kk < VB; ++kk) mv_add(m, p[kk], acc[kk]);
            WFmt<WF>::load(ws + (2 * d + 1) * setB, spb, k, m);
            RecGroup<VP, VB>::load(rin + (unsigned)bw[d] * rstride, cs, t, T, p);
#pragma unroll
            for (int kk = 0; kk < VB; ++kk) mdv_add(m, p[kk], acc[kk]);
        }
        RecGroup<VP, VB>::load(rin + (unsigned)i * rstride, cs, t, T, c);
#pragma unroll
        for (int kk = 0; kk < VB; ++kk) {
            const R a = alpha_of<R>(alpha, alphaf, il_vec<VP, VB>(t, T, kk));
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                o[kk][q].re = fma(a, fma(R(-6), c[kk][q].re, acc[kk][q].re), c[kk][q].re);
                o[kk][q].im = fma(a, fma(R(-6), c[kk][q].im, acc[kk][q].im), c[kk][q].im);
            }
        }
    }
    RecGroup<VP, VB>::store(rout + (unsigned)i * rstride, cs, t, T, o);
}

// --------------------------------------------------------------------------
// Interleaved multi-RHS step with packed FP32 pairs (fma.rn.f32x2).
// The strip's six W sets are staged in shared memory as one 16-byte word per
// complex element, already broadcast for a paired complex multiply-add:
//   forward  W(x)       element (r, k):            {re, re, -im, im}
//   backward W(x - 2d)  element (k, r) (the dagger): {re, re, im, -im}
// so that acc_r += w * p is two packed FMAs on (re, im) pairs,
//   acc = fma2({re, re}, {p.re, p.im}, acc);  acc = fma2({-im, im}, {p.im, p.re}, acc)
// which performs, lane by lane, the same FMA sequence as cmac / cmacc: the
// results are bitwise equal to every other kernel.  Arithmetic in FP32 (FP32
// and 16-bit storage).
// --------------------------------------------------------------------------
template <int VP, int WF, int VB, bool PRE, bool ACT>
__device__ __forceinline__ void ilx_body(const char *__restrict__ W, const char *__restrict__ in,
                                         char *__restrict__ out, const double *__restrict__ alpha,
                                         const float *__restrict__ alphaf, const int *__restrict__ active,
                                         const SubGeom &g, int nvec)
{
    static_assert(VP != P_F64, "packed FP32 pairs only");
    constexpr int WB = wfmt_bytes(WF);
    constexpr int VBY = vfmt_bytes(VP);
    extern __shared__ __align__(16) float4 wpk[];  // [set 6][element 9][site spb]
    const int spb = blockDim.y;
    const int x0 = blockIdx.x * spb;
    const int yq = blockIdx.y;
    const int blk = blockIdx.z / g.hz;
    const int zq = blockIdx.z - blk * g.hz;
    const int sy = g.hx, sz = g.hx * g.hy;
    const int row = zq * sz + yq * sy;
    const char *wb = W + (int64_t)blk * 3 * g.Ps * WB;
    const int nsite = min(spb, g.hx - x0);
    const int k = threadIdx.y;
    const bool act = k < nsite;
    const int t = threadIdx.x, T = nvec / VB;
    const int xq = x0 + k;
    const int i = row + xq;
    int nb[7];  // the six hops in the order of site_step, then the site itself
    nb[0] = xq == g.hx - 1 ? i - (g.hx - 1) : i + 1;
    nb[1] = xq == 0 ? i + (g.hx - 1) : i - 1;
    nb[2] = yq == g.hy - 1 ? i - (g.hy - 1) * sy : i + sy;
    nb[3] = yq == 0 ? i + (g.hy - 1) * sy : i - sy;
    nb[4] = zq == g.hz - 1 ? i - (g.hz - 1) * sz : i + sz;
    nb[5] = zq == 0 ? i + (g.hz - 1) * sz : i - sz;
    nb[6] = i;
    const char *rin = in + (int64_t)blk * g.Ps * nvec * VBY;
    char *rout = out + (int64_t)blk * g.Ps * nvec * VBY;
    const unsigned rstride = (unsigned)nvec * VRec<VP>::SB;  // site stride
    const int cs = g.Ps * nvec;                                    // colour planes
    // PRE: all seven record groups are requested before the W staging, so
    // their latencies overlap one another and the staging.
    cpx<float> pre[PRE ? 7 : 1][VB][3];
    if constexpr (PRE) {
        if (act) {
#pragma unroll
            for (int q = 0; q < 7; ++q) RecGroup<VP, VB>::load(rin + (unsigned)nb[q] * rstride, cs, t, T, pre[q]);
        }
    }
    {
        // stage: (set q, site kk) per thread; q = 2d + (0 forward, 1 backward)
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        for (int e = tid; e < 6 * nsite; e += blockDim.x * blockDim.y) {
            const int q = e / nsite, kk = e - q * nsite;
            const int d = q >> 1, xs = x0 + kk;
            int gi;
            if (q == 1)
                gi = row + (xs == 0 ? g.hx - 1 : xs - 1);
            else if (q == 3)
                gi = zq * sz + (yq == 0 ? g.hy - 1 : yq - 1) * sy + xs;
            else if (q == 5)
                gi = (zq == 0 ? g.hz - 1 : zq - 1) * sz + yq * sy + xs;
            else
                gi = row + xs;
            cpx<float> m[9];
            WFmt<WF>::load(wb + (int64_t)d * g.Ps * WB, g.Ps, gi, m);
            float4 *dst = wpk + q * 9 * spb + kk;
            if (q & 1) {
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const cpx<float> w = m[c * 3 + r];
                        dst[(r * 3 + c) * spb] = make_float4(w.re, w.re, w.im, -w.im);
                    }
            } else {
#pragma unroll
                for (int j = 0; j < 9; ++j) dst[j * spb] = make_float4(m[j].re, m[j].re, -m[j].im, m[j].im);
            }
        }
    }
    __syncthreads();
    if (!act) return;
    // ACT (serving): vectors whose slot is inactive are not stored
    bool on[VB];
    bool any = false, all = true;
#pragma unroll
    for (int k = 0; k < VB; ++k) {
        on[k] = !ACT || active[il_vec<VP, VB>(t, T, k)] != 0;
        any = any || on[k];
        all = all && on[k];
    }
    if (!any) return;
    float2 acc[VB][3];
#pragma unroll
    for (int v = 0; v < VB; ++v)
#pragma unroll
        for (int r = 0; r < 3; ++r) acc[v][r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        cpx<float> pl[VB][3];
        if constexpr (!PRE) RecGroup<VP, VB>::load(rin + (unsigned)nb[q] * rstride, cs, t, T, pl);
        const float4 *wq = wpk + q * 9 * spb + k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 p[VB], ps[VB];
#pragma unroll
            for (int v = 0; v < VB; ++v) {
                cpx<float> x;
                if constexpr (PRE)
                    x = pre[q][v][c];
                else
                    x = pl[v][c];
                p[v] = make_float2(x.re, x.im);
                ps[v] = f2swap(p[v]);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float4 w = wq[(r * 3 + c) * spb];
                const float2 wa = make_float2(w.x, w.y), wc = make_float2(w.z, w.w);
#pragma unroll
                for (int v = 0; v < VB; ++v) {
                    acc[v][r] = __ffma2_rn(wa, p[v], acc[v][r]);
                    acc[v][r] = __ffma2_rn(wc, ps[v], acc[v][r]);
                }
            }
        }
    }
    cpx<float> cc[VB][3], o[VB][3];
    if constexpr (PRE) {
#pragma unroll
        for (int v = 0; v < VB; ++v)
#pragma unroll
            for (int r = 0; r < 3; ++r) cc[v][r] = pre[6 % (PRE ? 7 : 1)][v][r];
    } else {
        RecGroup<VP, VB>::load(rin + (unsigned)i * rstride, cs, t, T, cc);
    }
    const float2 m6 = make_float2(-6.f, -6.f);
#pragma unroll
    for (int v = 0; v < VB; ++v) {
        const float a = alphaf[il_vec<VP, VB>(t, T, v)];
        const float2 a2 = make_float2(a, a);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float2 c2 = make_float2(cc[v][r].re, cc[v][r].im);
            const float2 u = __ffma2_rn(a2, __ffma2_rn(m6, c2, acc[v][r]), c2);
            o[v][r].re = u.x;
            o[v][r].im = u.y;
        }
    }
    if (all) {
        RecGroup<VP, VB>::store(rout + (unsigned)i * rstride, cs, t, T, o);
    } else {
#pragma unroll
        for (int k = 0; k < VB; ++k)
            if (on[k]) VRec<VP>::store(rout + (unsigned)i * rstride, cs, il_vec<VP, VB>(t, T, k), o[k]);
    }
}

template <int VP, int WF, int VB, bool PRE, bool ACT = false>
__global__ void __launch_bounds__(256) k_step_ilx(const char *__restrict__ W, const char *__restrict__ in,
                                                  char *__restrict__ out, const double *__restrict__ alpha,
                                                  const float *__restrict__ alphaf, const int *__restrict__ active,
                                                  SubGeom g, int nvec)
{
    ilx_body<VP, WF, VB, PRE, ACT>(W, in, out, alpha, alphaf, active, g, nvec);
}

// The same held to 56 registers in CTAs of at most 96 threads (12 CTAs per SM).
template <int VP, int WF, int VB>
__global__ void __launch_bounds__(96, 12) k_step_ilx_occ(const char *__restrict__ W, const char *__restrict__ in,
                                                         char *__restrict__ out, const double *__restrict__ alpha,
                                                         const float *__restrict__ alphaf, SubGeom g, int nvec)
{
    ilx_body<VP, WF, VB, false, false>(W, in, out, alpha, alphaf, nullptr, g, nvec);
}

// --------------------------------------------------------------------------
// Multi-RHS step on the interleaved layout, marching along z'.
// CTA = (nvec/VB, spb): threadIdx.x picks VB adjacent vectors, threadIdx.y
// one of spb consecutive x' of row y' = blockIdx.y in block blockIdx.z; each
// thread then walks its column z' = 0 .. hz-1.  psi(z-1), psi(z), psi(z+1)
// and W_z(z-1) stay in registers from one site to the next, so per site only
// psi(z+2)'s prefetch, the x and y neighbours and five W matrices are loaded.
// Same per-vector FMA sequence as site_step (bitwise equal results).
// --------------------------------------------------------------------------
template <int VP, int WF, int VB>
__global__ void __launch_bounds__(256) k_step_zm(const char *__restrict__ W, const char *__restrict__ in,
                                                 char *__restrict__ out, const double *__restrict__ alpha,
                                                 SubGeom g, int nvec)
{
    typedef typename VRec<VP>::R R;
    constexpr int WB = wfmt_bytes(WF);
    constexpr int VBY = vfmt_bytes(VP);
    const int t = threadIdx.x, T = nvec / VB;
    const int xq = blockIdx.x * blockDim.y + threadIdx.y;
    if (xq >= g.hx) return;
    const int yq = blockIdx.y;
    const int blk = blockIdx.z;
    const int sy = g.hx, sz = g.hx * g.hy, hz = g.hz;
    const int xp = xq == g.hx - 1 ? xq - (g.hx - 1) : xq + 1;
    const int xm = xq == 0 ? xq + (g.hx - 1) : xq - 1;
    const int yp = yq == g.hy - 1 ? 0 : yq + 1;
    const int ym = yq == 0 ? g.hy - 1 : yq - 1;
    const char *wb = W + (int64_t)blk * 3 * g.Ps * WB;
    const char *rin = in + (int64_t)blk * g.Ps * nvec * VBY;
    char *rout = out + (int64_t)blk * g.Ps * nvec * VBY;
    const unsigned rstride = (unsigned)nvec * VRec<VP>::SB;  // site stride
    const int cs = g.Ps * nvec;                                    // colour planes
    R a_v[VB];
#pragma unroll
    for (int k = 0; k < VB; ++k) a_v[k] = (R)alpha[il_vec<VP, VB>(t, T, k)];
    const int col = yq * sy + xq;       // site index at z' = 0
    auto site = [&](int z) { return z * sz + col; };
    // column state: psi(z-1), psi(z), psi(z+1) and W_z(z-1)
    cpx<R> pm[VB][3], pc[VB][3], pp[VB][3], wzm[9];
    RecGroup<VP, VB>::load(rin + (unsigned)site(hz - 1) * rstride, cs, t, T, pm);
    RecGroup<VP, VB>::load(rin + (unsigned)site(0) * rstride, cs, t, T, pc);
    RecGroup<VP, VB>::load(rin + (unsigned)site(1 % hz) * rstride, cs, t, T, pp);
    WFmt<WF>::load(wb + 2 * g.Ps * WB, g.Ps, site(hz - 1), wzm);
    for (int z = 0; z < hz; ++z) {
        const int i = site(z);
        const int zn = (z + 2) % hz;
        cpx<R> pn[VB][3];  // psi(z+2): next iteration's psi(z+1)
        RecGroup<VP, VB>::load(rin + (unsigned)site(zn) * rstride, cs, t, T, pn);
        cpx<R> acc[VB][3];
#pragma unroll
        for (int k = 0; k < VB; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[k][c].re = acc[k][c].im = R(0);
        cpx<R> m[9], p[VB][3], wz[9];
        // x forward / backward
        WFmt<WF>::load(wb, g.Ps, i, m);
        RecGroup<VP, VB>::load(rin + (unsigned)(i - xq + xp) * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mv_add(m, p[k], acc[k]);
        WFmt<WF>::load(wb, g.Ps, i - xq + xm, m);
        RecGroup<VP, VB>::load(rin + (unsigned)(i - xq + xm) * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mdv_add(m, p[k], acc[k]);
        // y forward / backward
        WFmt<WF>::load(wb + g.Ps * WB, g.Ps, i, m);
        RecGroup<VP, VB>::load(rin + (unsigned)(i + (yp - yq) * sy) * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mv_add(m, p[k], acc[k]);
        WFmt<WF>::load(wb + g.Ps * WB, g.Ps, i + (ym - yq) * sy, m);
        RecGroup<VP, VB>::load(rin + (unsigned)(i + (ym - yq) * sy) * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mdv_add(m, p[k], acc[k]);
        // z forward (W_z(z), psi(z+1)) / backward (W_z(z-1), psi(z-1)), from registers
        WFmt<WF>::load(wb + 2 * g.Ps * WB, g.Ps, i, wz);
#pragma unroll
        for (int k = 0; k < VB; ++k) mv_add(wz, pp[k], acc[k]);
#pragma unroll
        for (int k = 0; k < VB; ++k) mdv_add(wzm, pm[k], acc[k]);
        cpx<R> o[VB][3];
#pragma unroll
        for (int k = 0; k < VB; ++k) {
            const R a = a_v[k];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                o[k][q].re = fma(a, fma(R(-6), pc[k][q].re, acc[k][q].re), pc[k][q].re);
                o[k][q].im = fma(a, fma(R(-6), pc[k][q].im, acc[k][q].im), pc[k][q].im);
            }
        }
        RecGroup<VP, VB>::store(rout + (unsigned)i * rstride, cs, t, T, o);
        // slide the column window
#pragma unroll
        for (int k = 0; k < VB; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                pm[k][q] = pc[k][q];
                pc[k][q] = pp[k][q];
                pp[k][q] = pn[k][q];
            }
#pragma unroll
        for (int q = 0; q < 9; ++q) wzm[q] = wz[q];
    }
}

// --------------------------------------------------------------------------
// Bounded grid barrier.  Generation-counting barrier over all co-resident CTAs
// of a cooperative launch.  Every wait polls at most `budget` times; on
// expiry the CTA sets DERR_TIMEOUT in *err and returns false, and every other
// CTA stops waiting as soon as it sees that bit.  Nothing here can spin
// forever.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, long long budget)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_relaxed_s32(err) & DERR_TIMEOUT) {
            ok = 0;
        } else {
            unsigned *count = bar, *gen = bar + 1;
            const unsigned g0 = ld_acquire_u32(gen);
            __threadfence();
            const unsigned arrived = atomicAdd(count, 1u);
            if (arrived == gridDim.x - 1) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(gen, 1u);
            } else {
                long long polls = 0;
                while (ld_acquire_u32(gen) == g0) {
                    if (++polls > budget || (ld_relaxed_s32(err) & DERR_TIMEOUT)) {
                        atomicOr(err, DERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Persistent multi-step kernel: the (slice, sublattice) blocks are taken in
// groups sized to stay resident in L2; each group runs all N steps before the
// next group starts, with a grid barrier between steps.  Step 0 reads the
// storage-precision input, steps 1..N-1 read the scratch ping-pong (SP
// precision, L2-only loads), step N-1 writes the storage-precision output.
template <int VP, int WF, int VB>
__global__ void __launch_bounds__(256) k_persist(const char *__restrict__ W, const char *__restrict__ in,
                                                 char *__restrict__ out, char *scr0, char *scr1,
                                                 const double *__restrict__ alpha, SubGeom g, int nblk, int nvec,
                                                 int N, int gb, int64_t vs, int64_t ss, unsigned *bar, int *err,
                                                 long long budget)
{
    constexpr int SP = scratch_prec<VP>();
    constexpr int VBY = vfmt_bytes(VP), SBY = vfmt_bytes(SP);
    const int nchunk = (nvec + VB - 1) / VB;
    const int ngroups = (nblk + gb - 1) / gb;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int grp = 0; grp < ngroups; ++grp) {
        const int b0 = grp * gb;
        const int nb = min(gb, nblk - b0);
        const int64_t nsite = (int64_t)nb * g.Vs;
        const int64_t items = ((nsite + 31) / 32) * 32 * nchunk;
        for (int it = 0; it < N; ++it) {
            const bool first = it == 0, last = it == N - 1;
            const char *src = (it & 1) ? scr0 : scr1;  // scratch written by step it-1
            char *dst = (it & 1) ? scr1 : scr0;
            for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < items; w += stride) {
                int64_t site;
                int chunk;
                item_of(w, nchunk, site, chunk);
                if (site >= nsite) continue;
                const int rb = (int)(site / g.Vs);
                const int i = (int)(site - (int64_t)rb * g.Vs);
                const int ab = b0 + rb;
                const int64_t aoff = (int64_t)ab * g.Ps * VBY;  // absolute block in in/out
                const int64_t soff = (int64_t)rb * g.Ps * SBY;  // group-relative block in scratch
                if (first && last)
                    site_step<VP, VP, WF, VB, false, false>(W, in, out, alpha, g, ab, i, chunk * VB, nvec, vs, vs,
                                                            aoff, aoff);
                else if (first)
                    site_step<VP, SP, WF, VB, false, true>(W, in, dst, alpha, g, ab, i, chunk * VB, nvec, vs, ss,
                                                           aoff, soff);
                else if (last)
                    site_step<SP, VP, WF, VB, true, false>(W, src, out, alpha, g, ab, i, chunk * VB, nvec, ss, vs,
                                                           soff, aoff);
                else
                    site_step<SP, SP, WF, VB, true, true>(W, src, dst, alpha, g, ab, i, chunk * VB, nvec, ss, ss,
                                                          soff, soff);
            }
            if (grp == ngroups - 1 && last) break;
            if (!grid_barrier(bar, err, budget)) return;
        }
    }
}

// --------------------------------------------------------------------------
// Host-side launchers (per vector precision).
// --------------------------------------------------------------------------
template <int VP, int WF, int VB> cudaError_t step_launch(const StepArgs &a)
{
    const int nchunk = (a.nvec + VB - 1) / VB;
    const int64_t nsite = (int64_t)a.nblk * a.g.Vs;
    const int64_t items = ((nsite + 31) / 32) * 32 * nchunk;
    const int threads = a.threads > 0 ? a.threads : 128;
    const int64_t blocks = (items + threads - 1) / threads;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_step<VP, WF, VB><<<(unsigned)blocks, threads, 0, a.stream>>>(a.W, a.in, a.out, a.alpha, a.active, a.g,
                                                                   a.nblk, a.nvec, a.vstride_in, a.vstride_out);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// On-chip persistent form: the (slice, sublattice) blocks never couple, so
// one CTA per (block, vector group) runs all N steps inside its own shared
// memory: W of the block and two scratch copies of the group's iterates
// (plane stride Pss = Vs rounded up to 4), with __syncthreads between steps
// and no inter-CTA wait.  The iterates stay in the scratch precision (FP32,
// FP64 for FP64 storage) and are converted to the storage precision only on
// the way in and out, which is what k_persist computes: the results are
// bitwise equal.
// --------------------------------------------------------------------------
template <int VP, int WF, int VB>
__global__ void __launch_bounds__(1024) k_persist_blk(const char *__restrict__ W, const char *__restrict__ in,
                                                     char *__restrict__ out, const double *__restrict__ alpha,
                                                     SubGeom g, int nvec, int N, int nvg, int64_t vs)
{
    constexpr int SP = scratch_prec<VP>();
    constexpr int WB = wfmt_bytes(WF);
    constexpr int VBY = vfmt_bytes(VP), SBY = vfmt_bytes(SP);
    constexpr int NQ = WB / 16, REM = WB % 16;
    typedef typename VFmt<SP>::R R;
    extern __shared__ __align__(16) unsigned char sm[];
    const int b = blockIdx.x;
    const int v0 = blockIdx.y * nvg;
    const int nv = min(nvg, nvec - v0);
    const int Pss = (g.Vs + 3) / 4 * 4;
    SubGeom gs = g;
    gs.Ps = Pss;
    char *Ws = reinterpret_cast<char *>(sm);
    char *S0 = Ws + (int64_t)3 * Pss * WB;
    char *S1 = S0 + (int64_t)nvg * Pss * SBY;
    const int tid = threadIdx.x, nth = blockDim.x;
    // W of block b, plane by plane (16-byte words, then the remainder plane)
    for (int d = 0; d < 3; ++d) {
        const char *src = W + ((int64_t)b * 3 + d) * g.Ps * WB;
        char *dst = Ws + (int64_t)d * Pss * WB;
        for (int e = tid; e < NQ * g.Vs; e += nth) {
            const int j = e / g.Vs, i = e - j * g.Vs;
            reinterpret_cast<uint4 *>(dst)[(int64_t)j * Pss + i] = reinterpret_cast<const uint4 *>(src)[(int64_t)j * g.Ps + i];
        }
        if constexpr (REM == 8) {
            for (int i = tid; i < g.Vs; i += nth)
                reinterpret_cast<uint2 *>(dst + (int64_t)NQ * Pss * 16)[i] =
                    reinterpret_cast<const uint2 *>(src + (int64_t)NQ * g.Ps * 16)[i];
        } else if constexpr (REM == 4) {
            for (int i = tid; i < g.Vs; i += nth)
                reinterpret_cast<uint32_t *>(dst + (int64_t)NQ * Pss * 16)[i] =
                    reinterpret_cast<const uint32_t *>(src + (int64_t)NQ * g.Ps * 16)[i];
        }
    }
    // the group's vectors, converted to the scratch precision
    for (int e = tid; e < nv * g.Vs; e += nth) {
        const int v = e / g.Vs, i = e - v * g.Vs;
        cpx<R> p[3];
        VFmt<VP>::template load<false>(in + (int64_t)(v0 + v) * vs + (int64_t)b * g.Ps * VBY, g.Ps, i, p);
        VFmt<SP>::template store<false>(S0 + (int64_t)v * Pss * SBY, Pss, i, p);
    }
    __syncthreads();
    const int nchunk = (nv + VB - 1) / VB;
    const int64_t sst = (int64_t)Pss * SBY;
    for (int it = 0; it < N; ++it) {
        const char *src = (it & 1) ? S1 : S0;
        char *dst = (it & 1) ? S0 : S1;
        for (int w = tid; w < nchunk * g.Vs; w += nth) {
            const int c = w / g.Vs, i = w - c * g.Vs;
            site_step<SP, SP, WF, VB, false, false>(Ws, src, dst, alpha + v0, gs, 0, i, c * VB, nv, sst, sst, 0, 0);
        }
        __syncthreads();
    }
    const char *res = (N & 1) ? S1 : S0;
    for (int e = tid; e < nv * g.Vs; e += nth) {
        const int v = e / g.Vs, i = e - v * g.Vs;
        cpx<R> p[3];
        VFmt<SP>::template load<false>(res + (int64_t)v * Pss * SBY, Pss, i, p);
        VFmt<VP>::template store<false>(out + (int64_t)(v0 + v) * vs + (int64_t)b * g.Ps * VBY, g.Ps, i, p);
    }
}

template <int VP, int WF, int VB> cudaError_t persist_launch(const PersistArgs &a)
{
    if (a.onchip) {
        cudaError_t e = cudaFuncSetAttribute(k_persist_blk<VP, WF, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             a.smem);
        if (e != cudaSuccess) return e;
        dim3 grid(a.nblk, (a.nvec + a.nvg - 1) / a.nvg);
        if (grid.y > 65535) return cudaErrorInvalidConfiguration;
        k_persist_blk<VP, WF, VB><<<grid, a.threads, a.smem, a.stream>>>(a.W, a.in, a.out, a.alpha, a.g, a.nvec, a.N,
                                                                           a.nvg, a.vstride);
        return cudaGetLastError();
    }
    void *args[] = {(void *)&a.W,  (void *)&a.in,   (void *)&a.out,    (void *)&a.scr[0], (void *)&a.scr[1],
                    (void *)&a.alpha, (void *)&a.g, (void *)&a.nblk, (void *)&a.nvec,   (void *)&a.N,
                    (void *)&a.group_blocks, (void *)&a.vstride, (void *)&a.sstride, (void *)&a.bar,
                    (void *)&a.err, (void *)&a.budget};
    return cudaLaunchCooperativeKernel((const void *)k_persist<VP, WF, VB>, dim3(a.grid), dim3(a.threads), args, 0,
                                       a.stream);
}

template <int VP, int WF, int VB> int persist_occ(int threads)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist<VP, WF, VB>, threads, 0) != cudaSuccess) return 0;
    return n;
}

// Sites per CTA for the interleaved kernels: nvec * spb <= threads, with a
// whole number of warps when possible.
inline int il_spb(int nvec, int threads)
{
    if (threads <= 0) threads = 256;
    int spb = std::max(1, threads / nvec);
    for (int s = spb; s >= 1; --s)
        if ((s * nvec) % 32 == 0) return s;
    return spb;
}

// ONLYX: only the packed FP32 pair kernel is instantiated (eight vectors per thread).
template <int VP, int WF, int VB, bool ONLYX = false> cudaError_t step_il_launch(const StepArgs &a)
{
    // whole-row CTAs with the W rows staged by TMA bulk copies (k_ilt.cuh); a
    // shape or format it does not cover runs the packed kernel instead
    const bool ilt = a.tile[1] == 6 || a.tile[1] == 7 || a.tile[1] == 8;
    if (ilt) {
        const cudaError_t e = ilt_launch<VP, WF, VB>(a);
        if (e != cudaErrorNotSupported) return e;
    }
    const int tx = a.nvec / VB;
    // a strip of spb consecutive x' per CTA; tile[0] > 0 sets spb explicitly
    // threads = -128 selects the 64-register variant (CTAs of <= 128 threads)
    const bool occ = a.threads < 0;
    const bool xocc = a.tile[1] == 5;  // packed kernel, register-capped CTAs of <= 96 threads
    const int cap = xocc ? 96 : occ ? 128 : 256;
    int spb = a.tile[0] > 0 ? a.tile[0] : il_spb(tx, occ ? 128 : a.threads);
    spb = std::max(1, std::min(spb, cap / tx));
    spb = std::min(spb, a.g.hx);  // a strip never spans more than one row
    // the packed kernel also serves slot batches (active table); the other staged forms do not
    const bool packed = (a.tile[1] == 2 || ilt || ((a.tile[1] == 3 || a.tile[1] == 5) && a.active == nullptr)) &&
                        a.alphaf && VP != P_F64;
    const bool staged = a.tile[1] > 0 && a.active == nullptr && a.alphaf;
    constexpr int kPackB = 6 * 9 * 16;  // W packs per site of the packed kernel
    // shared memory within the default dynamic limit (48 KB)
    if (packed)
        spb = std::min(spb, (48 << 10) / kPackB);
    else if (staged)
        spb = std::min(spb, ((48 << 10) / 6 - 16) / wfmt_bytes(WF));
    if (tx * spb > cap) return cudaErrorInvalidConfiguration;
    dim3 block(tx, spb);
    dim3 grid((a.g.hx + spb - 1) / spb, a.g.hy, (unsigned)a.g.hz * a.nblk);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    if constexpr (ONLYX) {
        if (!packed || (a.tile[1] != 2 && !ilt) || a.active) return cudaErrorNotSupported;
        k_step_ilx<VP, WF, VB, false><<<grid, block, kPackB * spb, a.stream>>>(a.W, a.in, a.out, a.alpha, a.alphaf,
                                                                               nullptr, a.g, a.nvec);
        return cudaGetLastError();
    } else {
    if (packed) {
        // packed FP32 pairs with W packs in shared memory; 3 = all records requested up front
        if constexpr (VP != P_F64) {
            if (a.active)
                k_step_ilx<VP, WF, VB, false, true><<<grid, block, kPackB * spb, a.stream>>>(
                    a.W, a.in, a.out, a.alpha, a.alphaf, a.active, a.g, a.nvec);
            else if (a.tile[1] == 3)
                k_step_ilx<VP, WF, VB, true><<<grid, block, kPackB * spb, a.stream>>>(a.W, a.in, a.out, a.alpha,
                                                                                      a.alphaf, nullptr, a.g, a.nvec);
            else if (a.tile[1] == 5)
                k_step_ilx_occ<VP, WF, VB><<<grid, block, kPackB * spb, a.stream>>>(a.W, a.in, a.out, a.alpha,
                                                                                      a.alphaf, a.g, a.nvec);
            else
                k_step_ilx<VP, WF, VB, false><<<grid, block, kPackB * spb, a.stream>>>(a.W, a.in, a.out, a.alpha,
                                                                                       a.alphaf, nullptr, a.g, a.nvec);
        }
    } else if (staged && a.tile[1] == 4 && VP != P_F64) {
        // W of the strip staged in shared memory as stored, packed FP32 pair FMAs
        if constexpr (VP != P_F64)
            k_step_ilw<VP, WF, VB, true><<<grid, block, 6 * ((spb * wfmt_bytes(WF) + 15) / 16 * 16), a.stream>>>(
                a.W, a.in, a.out, a.alpha, a.alphaf, a.g, a.nvec);
    } else if (staged)  // W of the strip staged in shared memory
        k_step_ilw<VP, WF, VB, false><<<grid, block, 6 * ((spb * wfmt_bytes(WF) + 15) / 16 * 16), a.stream>>>(
            a.W, a.in, a.out, a.alpha, a.alphaf, a.g, a.nvec);
    else if (occ)
        k_step_il_occ<VP, WF, VB><<<grid, block, 0, a.stream>>>(a.W, a.in, a.out, a.alpha, a.active, a.g,
                                                                     a.nvec);
    else
        k_step_il<VP, WF, VB><<<grid, block, 0, a.stream>>>(a.W, a.in, a.out, a.alpha, a.active, a.g, a.nvec);
    return cudaGetLastError();
    }
}

template <int VP, int WF, int VB> cudaError_t step_zm_launch(const StepArgs &a)
{
    const int tx = a.nvec / VB;
    const int spb = il_spb(tx, a.threads);
    dim3 block(tx, spb);
    dim3 grid((a.g.hx + spb - 1) / spb, a.g.hy, (unsigned)a.nblk);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    k_step_zm<VP, WF, VB><<<grid, block, 0, a.stream>>>(a.W, a.in, a.out, a.alpha, a.g, a.nvec);
    return cudaGetLastError();
}

template <int VP, int WF> cudaError_t step_zm_w(const StepArgs &a)
{
    if constexpr (!combo_ok<VP, WF>()) {
        return cudaErrorNotSupported;
    } else {
        if (a.nvec < 1 || a.nvec > 256) return cudaErrorInvalidValue;
        int vb = a.vb > 0 ? a.vb : 1;
        if (a.nvec % vb != 0) vb = 1;
        if constexpr (VP == P_F32) {
            switch (vb) {
            case 2: return step_zm_launch<VP, WF, 2>(a);
            case 4: return step_zm_launch<VP, WF, 4>(a);
            default: return step_zm_launch<VP, WF, 1>(a);
            }
        } else if constexpr (VP == P_F64) {
            if (vb == 2) return step_zm_launch<VP, WF, 2>(a);
            return step_zm_launch<VP, WF, 1>(a);
        } else {
            switch (vb) {
            case 2: return step_zm_launch<VP, WF, 2>(a);
            case 4: return step_zm_launch<VP, WF, 4>(a);
            default: return step_zm_launch<VP, WF, 1>(a);
            }
        }
    }
}

// vb = vectors per thread; it must divide nvec (else 1 is used).  FP32 groups
// of an even count on an even nvec are 16-byte aligned.
template <int VP, int WF> cudaError_t step_il_w(const StepArgs &a)
{
    if constexpr (!combo_ok<VP, WF>()) {
        return cudaErrorNotSupported;
    } else {
        if (a.nvec < 1 || a.nvec > 256) return cudaErrorInvalidValue;
        int vb = a.vb > 0 ? a.vb : 1;
        if (a.nvec % vb != 0) vb = 1;
        if constexpr (VP == P_F32) {
            switch (vb) {
            case 2: return step_il_launch<VP, WF, 2>(a);
            case 4: return step_il_launch<VP, WF, 4>(a);
            case 8: return step_il_launch<VP, WF, 8, true>(a);  // packed kernel only
            default: return step_il_launch<VP, WF, 1>(a);
            }
        } else if constexpr (VP == P_F64) {
            if (vb == 2) return step_il_launch<VP, WF, 2>(a);
            return step_il_launch<VP, WF, 1>(a);
        } else {
            switch (vb) {
            case 2: return step_il_launch<VP, WF, 2>(a);
            case 4: return step_il_launch<VP, WF, 4>(a);
            default: return step_il_launch<VP, WF, 1>(a);
            }
        }
    }
}

template <int VP, int WF> cudaError_t step_w(const StepArgs &a)
{
    if constexpr (!combo_ok<VP, WF>()) {
        return cudaErrorNotSupported;
    } else {
        switch (a.vb) {
        case 1: return step_launch<VP, WF, 1>(a);
        case 2: return step_launch<VP, WF, 2>(a);
        case 4: return step_launch<VP, WF, 4>(a);
        case 8:
            if constexpr (VP != P_F64) return step_launch<VP, WF, 8>(a);
            else return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
        }
    }
}

template <int VP, int WF> cudaError_t persist_w(const PersistArgs &a)
{
    if constexpr (!combo_ok<VP, WF>()) {
        return cudaErrorNotSupported;
    } else {
        switch (a.vb) {
        case 1: return persist_launch<VP, WF, 1>(a);
        case 4: return persist_launch<VP, WF, 4>(a);
        case 8:
            if constexpr (VP != P_F64) return persist_launch<VP, WF, 8>(a);
            else return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
        }
    }
}

template <int VP, int WF> int occ_w(int vb, int threads)
{
    if constexpr (!combo_ok<VP, WF>()) {
        return 0;
    } else {
        switch (vb) {
        case 1: return persist_occ<VP, WF, 1>(threads);
        case 4: return persist_occ<VP, WF, 4>(threads);
        case 8:
            if constexpr (VP != P_F64) return persist_occ<VP, WF, 8>(threads);
            else return 0;
        default: return 0;
        }
    }
}

#define TLS_WFMT_SWITCH(FN, VP, ARG, FAIL)                 \
    switch (wf) {                                          \
    case W_F64_18: return FN<VP, W_F64_18> ARG;            \
    case W_F32_18: return FN<VP, W_F32_18> ARG;            \
    case W_F32_12: return FN<VP, W_F32_12> ARG;            \
    case W_F32_8: return FN<VP, W_F32_8> ARG;              \
    case W_F16_18: return FN<VP, W_F16_18> ARG;            \
    case W_F16_12: return FN<VP, W_F16_12> ARG;            \
    case W_BF16_18: return FN<VP, W_BF16_18> ARG;          \
    case W_BF16_12: return FN<VP, W_BF16_12> ARG;          \
    default: return FAIL;                                  \
    }

template <int VP> cudaError_t step_dispatch(const StepArgs &a)
{
    const int wf = a.wfmt;
    TLS_WFMT_SWITCH(step_w, VP, (a), cudaErrorNotSupported)
}

template <int VP> cudaError_t step_il_dispatch(const StepArgs &a)
{
    const int wf = a.wfmt;
    TLS_WFMT_SWITCH(step_il_w, VP, (a), cudaErrorNotSupported)
}

template <int VP> cudaError_t step_zm_dispatch(const StepArgs &a)
{
    const int wf = a.wfmt;
    TLS_WFMT_SWITCH(step_zm_w, VP, (a), cudaErrorNotSupported)
}

template <int VP> cudaError_t persist_dispatch(const PersistArgs &a)
{
    const int wf = a.wfmt;
    TLS_WFMT_SWITCH(persist_w, VP, (a), cudaErrorNotSupported)
}

template <int VP> int occ_dispatch(int wf, int vb, int threads)
{
    TLS_WFMT_SWITCH(occ_w, VP, (vb, threads), 0)
}

}  // namespace tls
