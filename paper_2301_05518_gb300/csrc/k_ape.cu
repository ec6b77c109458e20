// k_ape.cu -- APE smearing of the spatial links (gauge-smeared links in place
// of U_mu, Sec. 2, the remark after Eq. tlSmear).
//
// One step, every link from the previous iterate (out of place):
//   V_mu(x) = (1 - a) U_mu(x) + (a/4) sum_{nu != mu, spatial} [
//       U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
//   U'_mu(x) = P(V_mu(x))
// P is the projection onto SU(3): the unitary polar factor of V by Newton's
// iteration X <- (X + X^-dag) / 2 (stopped one step after the change falls
// below 1e-12; at most 100 steps), then multiplied by exp(-i phi / 3) with
// phi = arg det X in (-pi, pi].  All arithmetic is FP64 on the packed links
// (sublattice layout, double2 planes).  A singular V or an iteration that
// does not settle sets DERR_PROJECT and leaves that link unchanged.
#include "tls_dev.cuh"
#include "tls_internal.h"

namespace tls {
namespace {

struct M3 {
    double2 e[9];  // row-major complex 3x3
};

__device__ __forceinline__ double2 cm(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 ca(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 c;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            double2 acc = cm(a.e[r * 3], b.e[s]);
            acc = ca(acc, cm(a.e[r * 3 + 1], b.e[3 + s]));
            acc = ca(acc, cm(a.e[r * 3 + 2], b.e[6 + s]));
            c.e[r * 3 + s] = acc;
        }
    return c;
}

__device__ __forceinline__ M3 dag(const M3 &a)
{
    M3 d;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) d.e[r * 3 + s] = make_double2(a.e[s * 3 + r].x, -a.e[s * 3 + r].y);
    return d;
}

// Cofactor C_rs of a 3x3 complex matrix (signed minor).
__device__ __forceinline__ double2 cofactor(const M3 &m, int r, int s)
{
    const int r0 = r == 0 ? 1 : 0, r1 = r == 2 ? 1 : 2;
    const int s0 = s == 0 ? 1 : 0, s1 = s == 2 ? 1 : 2;
    double2 v = cs(cm(m.e[r0 * 3 + s0], m.e[r1 * 3 + s1]), cm(m.e[r0 * 3 + s1], m.e[r1 * 3 + s0]));
    return ((r + s) & 1) ? make_double2(-v.x, -v.y) : v;
}

__device__ __forceinline__ double2 det(const M3 &m)
{
    return ca(ca(cm(m.e[0], cofactor(m, 0, 0)), cm(m.e[1], cofactor(m, 0, 1))), cm(m.e[2], cofactor(m, 0, 2)));
}

// X^-dag = (adj X / det X)^dag: element (r, s) = conj(C_rs / det).
__device__ __forceinline__ bool inv_dag(const M3 &x, M3 &out)
{
    const double2 d = det(x);
    const double n2 = d.x * d.x + d.y * d.y;
    if (!(n2 > 0.0)) return false;
    const double2 rd = make_double2(d.x / n2, -d.y / n2);  // 1 / det
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const double2 v = cm(cofactor(x, r, s), rd);
            out.e[r * 3 + s] = make_double2(v.x, -v.y);
        }
    return true;
}

__device__ bool project_su3(M3 &x)
{
    bool settled = false, done = false;
    for (int it = 0; it < 100 && !done; ++it) {
        M3 xi;
        if (!inv_dag(x, xi)) return false;
        double d2 = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double2 n = make_double2(0.5 * (x.e[k].x + xi.e[k].x), 0.5 * (x.e[k].y + xi.e[k].y));
            const double dx = n.x - x.e[k].x, dy = n.y - x.e[k].y;
            d2 += dx * dx + dy * dy;
            x.e[k] = n;
        }
        if (settled)
            done = true;
        else if (sqrt(d2) < 1e-12)
            settled = true;
    }
    if (!done) return false;
    const double2 d = det(x);
    const double phi = atan2(d.y, d.x);
    double sn, cn;
    sincos(phi / 3.0, &sn, &cn);
    const double2 ph = make_double2(cn, -sn);
#pragma unroll
    for (int k = 0; k < 9; ++k) x.e[k] = cm(x.e[k], ph);
    return true;
}

// Site reached from (block b, site i) by one step along spatial direction d
// (dir = +1 or -1): the sublattice bit d flips; the half coordinate moves only
// when leaving an odd coordinate forwards or an even one backwards.
__device__ __forceinline__ void step1(const SubGeom &g, int &b, int &i, int d, int dir)
{
    const int sub = b & 7;
    const int odd = (sub >> d) & 1;
    const int h[3] = {g.hx, g.hy, g.hz};
    int q[3];
    q[0] = i % g.hx;
    const int r = i / g.hx;
    q[1] = r % g.hy;
    q[2] = r / g.hy;
    if (dir > 0 && odd) q[d] = q[d] + 1 == h[d] ? 0 : q[d] + 1;
    if (dir < 0 && !odd) q[d] = q[d] == 0 ? h[d] - 1 : q[d] - 1;
    b = (b & ~7) | (sub ^ (1 << d));
    i = (q[2] * g.hy + q[1]) * g.hx + q[0];
}

__device__ __forceinline__ M3 load_link(const double2 *__restrict__ U, const SubGeom &g, int b, int i, int d)
{
    M3 m;
    const double2 *p = U + ((int64_t)b * 3 + d) * 9 * g.Ps + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) m.e[k] = p[(int64_t)k * g.Ps];
    return m;
}

// One thread per (block, site, direction mu).
__global__ void __launch_bounds__(128) k_ape_step(const double2 *__restrict__ U, double2 *__restrict__ out, SubGeom g,
                                                  int64_t total, double a, int *err)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (int)(idx % g.Vs);
    const int64_t r = idx / g.Vs;
    const int mu = (int)(r % 3);
    const int b = (int)(r / 3);
    M3 st;
#pragma unroll
    for (int k = 0; k < 9; ++k) st.e[k] = make_double2(0.0, 0.0);
    for (int nu = 0; nu < 3; ++nu) {
        if (nu == mu) continue;
        // forward staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
        int bn = b, in_ = i, bm = b, im = i;
        step1(g, bn, in_, nu, +1);
        step1(g, bm, im, mu, +1);
        M3 f = mul(mul(load_link(U, g, b, i, nu), load_link(U, g, bn, in_, mu)), dag(load_link(U, g, bm, im, nu)));
        // backward staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        int bb = b, ib = i;
        step1(g, bb, ib, nu, -1);
        int bd = bb, id = ib;
        step1(g, bd, id, mu, +1);
        M3 h = mul(mul(dag(load_link(U, g, bb, ib, nu)), load_link(U, g, bb, ib, mu)), load_link(U, g, bd, id, nu));
#pragma unroll
        for (int k = 0; k < 9; ++k) st.e[k] = ca(st.e[k], ca(f.e[k], h.e[k]));
    }
    const M3 u = load_link(U, g, b, i, mu);
    M3 v;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        v.e[k] = make_double2((1.0 - a) * u.e[k].x + 0.25 * a * st.e[k].x, (1.0 - a) * u.e[k].y + 0.25 * a * st.e[k].y);
    const bool ok = project_su3(v);
    if (!ok) atomicOr(err, DERR_PROJECT);
    const M3 &w = ok ? v : u;
    double2 *p = out + ((int64_t)b * 3 + mu) * 9 * g.Ps + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) p[(int64_t)k * g.Ps] = w.e[k];
}

}  // namespace

cudaError_t launch_ape_step(const double *U, double *out, const SubGeom &g, int nblk, double a, int *err,
                            cudaStream_t s)
{
    const int64_t total = (int64_t)nblk * 3 * g.Vs;
    const unsigned nb = (unsigned)((total + 127) / 128);
    k_ape_step<<<nb, 128, 0, s>>>(reinterpret_cast<const double2 *>(U), reinterpret_cast<double2 *>(out), g, total, a,
                                  err);
    return cudaGetLastError();
}

}  // namespace tls
