// k_hop.cuh -- one-link Gaussian smearing step on the interleaved layout.
//
// Sec. 2, Eq. 2-3: psi' = psi + alpha H psi with the one-link hopping operator
//   H psi(x) = sum_mu [ U_mu(x) psi(x + mu) + U_mu^dag(x - mu) psi(x - mu) ]
// (Eq. 3 with C = 1).  A +-1 hop flips bit mu of the spatial parity, so in the
// sublattice layout it reaches the record group of the neighbouring block
// (slice, sub ^ (1 << mu)); the half coordinate moves only when the source
// coordinate is odd (forward) or even (backward):
//   x + mu: block sub ^ bit, site  bit_mu(sub) ? forward(i) : i
//   x - mu: block sub ^ bit, site  bit_mu(sub) ? i : backward(i)
// The links U_mu are stored in a W-format field (rounded U, same planes).
#pragma once

#include "k_stencil.cuh"

namespace tls {

template <int VP, int WF, int VB>
__global__ void __launch_bounds__(512) k_hop_il(const char *__restrict__ L1, const char *__restrict__ in,
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
    const int blk = blockIdx.z / g.hz;
    const int zq = blockIdx.z - blk * g.hz;
    const int sub = blk & 7, bt = blk & ~7;
    const int sy = g.hx, sz = g.hx * g.hy;
    const int i = zq * sz + yq * sy + xq;
    int fw[3], bw[3];
    fw[0] = xq == g.hx - 1 ? i - (g.hx - 1) : i + 1;
    bw[0] = xq == 0 ? i + (g.hx - 1) : i - 1;
    fw[1] = yq == g.hy - 1 ? i - (g.hy - 1) * sy : i + sy;
    bw[1] = yq == 0 ? i + (g.hy - 1) * sy : i - sy;
    fw[2] = zq == g.hz - 1 ? i - (g.hz - 1) * sz : i + sz;
    bw[2] = zq == 0 ? i + (g.hz - 1) * sz : i - sz;
    const unsigned rstride = (unsigned)nvec * VRec<VP>::SB;  // site stride
    const int cs = g.Ps * nvec;                                    // colour planes
    auto recs = [&](int b) { return in + (int64_t)b * g.Ps * nvec * VBY; };
    auto links = [&](int b, int d) { return L1 + ((int64_t)b * 3 + d) * g.Ps * WB; };
    cpx<R> acc[VB][3];
#pragma unroll
    for (int k = 0; k < VB; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[k][c].re = acc[k][c].im = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int odd = (sub >> d) & 1;
        const int nb = bt | (sub ^ (1 << d));
        const int i_f = odd ? fw[d] : i;
        const int i_b = odd ? i : bw[d];
        cpx<R> m[9], p[VB][3];
        WFmt<WF>::load(links(blk, d), g.Ps, i, m);
        RecGroup<VP, VB>::load(recs(nb) + (unsigned)i_f * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mv_add(m, p[k], acc[k]);
        WFmt<WF>::load(links(nb, d), g.Ps, i_b, m);
        RecGroup<VP, VB>::load(recs(nb) + (unsigned)i_b * rstride, cs, t, T, p);
#pragma unroll
        for (int k = 0; k < VB; ++k) mdv_add(m, p[k], acc[k]);
    }
    cpx<R> c[VB][3], o[VB][3];
    RecGroup<VP, VB>::load(recs(blk) + (unsigned)i * rstride, cs, t, T, c);
#pragma unroll
    for (int k = 0; k < VB; ++k) {
        const R a = (R)alpha[il_vec<VP, VB>(t, T, k)];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            o[k][q].re = fma(a, acc[k][q].re, c[k][q].re);
            o[k][q].im = fma(a, acc[k][q].im, c[k][q].im);
        }
    }
    RecGroup<VP, VB>::store(out + (int64_t)blk * g.Ps * nvec * VBY + (unsigned)i * rstride, cs, t, T, o);
}

template <int VP, int WF, int VB> cudaError_t hop_launch(const StepArgs &a)
{
    const int tx = a.nvec / VB;
    const int spb = il_spb(tx, a.threads);
    dim3 block(tx, spb);
    dim3 grid((a.g.hx + spb - 1) / spb, a.g.hy, (unsigned)a.g.hz * a.nblk);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    k_hop_il<VP, WF, VB><<<grid, block, 0, a.stream>>>(a.W, a.in, a.out, a.alpha, a.g, a.nvec);
    return cudaGetLastError();
}

// Link fields are FP64-18 for FP64 vectors and FP32-18 otherwise.
template <int VP> cudaError_t hop_dispatch(const StepArgs &a)
{
    constexpr int WF = VP == P_F64 ? W_F64_18 : W_F32_18;
    if (a.wfmt != WF) return cudaErrorNotSupported;
    if (a.nvec < 1 || a.nvec > 256) return cudaErrorInvalidValue;
    const int vb = (a.vb == 2 && a.nvec % 2 == 0) ? 2 : 1;
    if (vb == 2) return hop_launch<VP, WF, 2>(a);
    return hop_launch<VP, WF, 1>(a);
}

}  // namespace tls
