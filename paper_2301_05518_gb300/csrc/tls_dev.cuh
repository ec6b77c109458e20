// tls_dev.cuh -- device-side data formats of the two-link smearing library.
//
// Sublattice layout.  The +-2 hops of the two-link Laplacian (Sec. 2,
// Eq. tlLapl1) never change the parity of any coordinate, so every time slice
// splits into 8 independent sublattices sub = (x&1) | (y&1)<<1 | (z&1)<<2.
// Inside a sublattice the site (x, y, z) sits at x' = x>>1, y' = y>>1,
// z' = z>>1, i = (z' * hy + y') * hx + x' with h = L/2, and a +-2 hop becomes
// a +-1 step with period h: a unit-stride neighbour.  A (slice, sublattice)
// pair is a "block"; block b = ts * 8 + sub.  Each block holds Vs = hx*hy*hz
// sites and is stored with a plane stride Ps = Vs rounded up to 32, so every
// plane starts on a 128-byte boundary.
//
// Within a block each field is structure-of-arrays: a per-site record is cut
// into 16-byte words, and word j of all sites forms one plane (Ps entries),
// followed by an 8- or 4-byte remainder plane.  A warp of 32 consecutive
// sites then reads 512 contiguous bytes per 16-byte word.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tls_types.h"

namespace tls {

template <typename T> struct cpx {
    T re, im;
};

// Loads and stores with an optional L2-only policy (.cg).  Data that other
// CTAs rewrite during one launch (the persistent kernel's scratch) must not
// be served from a stale L1 line, so it goes through ld.global.cg / st.global.cg.
template <bool CG, typename T> __device__ __forceinline__ T vld(const T *p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}
template <bool CG, typename T> __device__ __forceinline__ void vst(T *p, T v)
{
    if constexpr (CG)
        __stcg(p, v);
    else
        *p = v;
}

template <typename T> __device__ __forceinline__ void cmac(cpx<T> &acc, cpx<T> a, cpx<T> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}

// acc += conj(a) * b
template <typename T> __device__ __forceinline__ void cmacc(cpx<T> &acc, cpx<T> a, cpx<T> b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// out += m v  (m row-major 3x3)
template <typename T> __device__ __forceinline__ void mv_add(const cpx<T> m[9], const cpx<T> v[3], cpx<T> out[3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) cmac(out[r], m[r * 3 + k], v[k]);
}

// out += m^dag v
template <typename T> __device__ __forceinline__ void mdv_add(const cpx<T> m[9], const cpx<T> v[3], cpx<T> out[3])
{
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) cmacc(out[r], m[k * 3 + r], v[k]);
}

// Row 3 of an SU(3) matrix from rows 1 and 2: r2 = conj(r0 x r1).
template <typename T> __device__ __forceinline__ void third_row(cpx<T> m[9])
{
    const cpx<T> *a = m, *b = m + 3;
    cpx<T> c0, c1, c2;
    c0.re = a[1].re * b[2].re - a[1].im * b[2].im - (a[2].re * b[1].re - a[2].im * b[1].im);
    c0.im = a[1].re * b[2].im + a[1].im * b[2].re - (a[2].re * b[1].im + a[2].im * b[1].re);
    c1.re = a[2].re * b[0].re - a[2].im * b[0].im - (a[0].re * b[2].re - a[0].im * b[2].im);
    c1.im = a[2].re * b[0].im + a[2].im * b[0].re - (a[0].re * b[2].im + a[0].im * b[2].re);
    c2.re = a[0].re * b[1].re - a[0].im * b[1].im - (a[1].re * b[0].re - a[1].im * b[0].im);
    c2.im = a[0].re * b[1].im + a[0].im * b[1].re - (a[1].re * b[0].im + a[1].im * b[0].re);
    m[6].re = c0.re; m[6].im = -c0.im;
    m[7].re = c1.re; m[7].im = -c1.im;
    m[8].re = c2.re; m[8].im = -c2.im;
}

// --------------------------------------------------------------------------
// 16-bit helpers
// --------------------------------------------------------------------------
template <typename H> struct H2;
template <> struct H2<__half> {
    typedef __half2 t;
    static __device__ __forceinline__ float2 to2(uint32_t u)
    {
        __half2 h = *reinterpret_cast<__half2 *>(&u);
        return __half22float2(h);
    }
    static __device__ __forceinline__ uint32_t from2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    static __device__ __forceinline__ uint32_t from2d(double a, double b)
    {
        __half lo = __double2half(a), hi = __double2half(b);
        return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
    }
};
template <> struct H2<__nv_bfloat16> {
    typedef __nv_bfloat162 t;
    static __device__ __forceinline__ float2 to2(uint32_t u)
    {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
        return __bfloat1622float2(h);
    }
    static __device__ __forceinline__ uint32_t from2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    static __device__ __forceinline__ uint32_t from2d(double a, double b)
    {
        __nv_bfloat16 lo = __double2bfloat16(a), hi = __double2bfloat16(b);
        return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    }
};

// --------------------------------------------------------------------------
// W formats.  blk points at the (block, direction) record group: planes of
// 16-byte words, Ps entries each, then the remainder plane.
//   load(blk, Ps, i, m)    -> m[9] complex in the arithmetic type
//   store(blk, Ps, i, w)   <- w[18] doubles (row-major, re/im), rounded RN
// --------------------------------------------------------------------------
template <int F> struct WFmt;

template <> struct WFmt<W_F64_18> {
    typedef double R;
    static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<double> m[9])
    {
        const double2 *p = reinterpret_cast<const double2 *>(blk);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 v = p[k * Ps + i];
            m[k].re = v.x;
            m[k].im = v.y;
        }
    }
    static __device__ __forceinline__ void store(char *blk, int64_t Ps, int i, const double w[18])
    {
        double2 *p = reinterpret_cast<double2 *>(blk);
#pragma unroll
        for (int k = 0; k < 9; ++k) p[k * Ps + i] = make_double2(w[2 * k], w[2 * k + 1]);
    }
};

template <> struct WFmt<W_F32_18> {
    typedef float R;
    static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<float> m[9])
    {
        const float4 *q = reinterpret_cast<const float4 *>(blk);
        const float2 *r = reinterpret_cast<const float2 *>(blk + 4 * Ps * 16);
        float f[18];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 v = q[k * Ps + i];
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
        float2 v = r[i];
        f[16] = v.x; f[17] = v.y;
#pragma unroll
        for (int k = 0; k < 9; ++k) { m[k].re = f[2 * k]; m[k].im = f[2 * k + 1]; }
    }
    static __device__ __forceinline__ void store(char *blk, int64_t Ps, int i, const double w[18])
    {
        float4 *q = reinterpret_cast<float4 *>(blk);
        float2 *r = reinterpret_cast<float2 *>(blk + 4 * Ps * 16);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            q[k * Ps + i] = make_float4(__double2float_rn(w[4 * k]), __double2float_rn(w[4 * k + 1]),
                                        __double2float_rn(w[4 * k + 2]), __double2float_rn(w[4 * k + 3]));
        r[i] = make_float2(__double2float_rn(w[16]), __double2float_rn(w[17]));
    }
};

template <> struct WFmt<W_F32_12> {
    typedef float R;
    static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<float> m[9])
    {
        const float4 *q = reinterpret_cast<const float4 *>(blk);
        float f[12];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 v = q[k * Ps + i];
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) { m[k].re = f[2 * k]; m[k].im = f[2 * k + 1]; }
        third_row(m);
    }
    static __device__ __forceinline__ void store(char *blk, int64_t Ps, int i, const double w[18])
    {
        float4 *q = reinterpret_cast<float4 *>(blk);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            q[k * Ps + i] = make_float4(__double2float_rn(w[4 * k]), __double2float_rn(w[4 * k + 1]),
                                        __double2float_rn(w[4 * k + 2]), __double2float_rn(w[4 * k + 3]));
    }
};

// 8 reals: W01, W02, W10 (complex) and the phases of W00 and W20.  With
// row 0 known up to |W00| and column 0 known up to |W20|:
//   |W00|^2 = 1 - |W01|^2 - |W02|^2,   |W20|^2 = 1 - |W00|^2 - |W10|^2,
// and, with n = |W01|^2 + |W02|^2 = 1 - |W00|^2 > 0, unitarity of row 1
// against row 0 plus W20 = conj(W01 W12 - W02 W11) (row 2 = conj(r0 x r1))
// give the 2x2 linear system solved by
//   W11 = -(W10 conj(W00) W01 + conj(W02) conj(W20)) / n
//   W12 =  (conj(W01) conj(W20) - W10 conj(W00) W02) / n
// and row 2 follows as conj(r0 x r1).
template <> struct WFmt<W_F32_8> {
    typedef float R;
    static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<float> m[9])
    {
        const float4 *q = reinterpret_cast<const float4 *>(blk);
        float4 a = q[i], b = q[Ps + i];
        cpx<float> w01 = {a.x, a.y}, w02 = {a.z, a.w}, w10 = {b.x, b.y};
        float n = w01.re * w01.re + w01.im * w01.im + w02.re * w02.re + w02.im * w02.im;
        float a00 = sqrtf(fmaxf(1.0f - n, 0.0f));
        float a20 = sqrtf(fmaxf(n - (w10.re * w10.re + w10.im * w10.im), 0.0f));
        float s0, c0, s2, c2;
        sincosf(b.z, &s0, &c0);
        sincosf(b.w, &s2, &c2);
        cpx<float> w00 = {a00 * c0, a00 * s0}, w20 = {a20 * c2, a20 * s2};
        float inv = 1.0f / n;
        // t = W10 conj(W00)
        cpx<float> t = {w10.re * w00.re + w10.im * w00.im, w10.im * w00.re - w10.re * w00.im};
        cpx<float> w11, w12;
        // W11 = -(t W01 + conj(W02) conj(W20)) / n
        w11.re = -((t.re * w01.re - t.im * w01.im) + (w02.re * w20.re - w02.im * w20.im)) * inv;
        w11.im = -((t.re * w01.im + t.im * w01.re) - (w02.re * w20.im + w02.im * w20.re)) * inv;
        // W12 = (conj(W01) conj(W20) - t W02) / n
        w12.re = ((w01.re * w20.re - w01.im * w20.im) - (t.re * w02.re - t.im * w02.im)) * inv;
        w12.im = (-(w01.re * w20.im + w01.im * w20.re) - (t.re * w02.im + t.im * w02.re)) * inv;
        m[0] = w00; m[1] = w01; m[2] = w02;
        m[3] = w10; m[4] = w11; m[5] = w12;
        third_row(m);
    }
    // Returns false when |W00| is too close to 1 for the parameterisation.
    static __device__ __forceinline__ bool store(char *blk, int64_t Ps, int i, const double w[18])
    {
        float4 *q = reinterpret_cast<float4 *>(blk);
        double th0 = atan2(w[1], w[0]);
        double th2 = atan2(w[13], w[12]);
        q[i] = make_float4(__double2float_rn(w[2]), __double2float_rn(w[3]), __double2float_rn(w[4]),
                           __double2float_rn(w[5]));
        q[Ps + i] = make_float4(__double2float_rn(w[6]), __double2float_rn(w[7]), __double2float_rn(th0),
                                __double2float_rn(th2));
        double n = w[2] * w[2] + w[3] * w[3] + w[4] * w[4] + w[5] * w[5];
        return n > 1e-6;
    }
};

template <typename H, int NR> struct WFmtH {
    // NR = 18 or 12 reals stored as 16-bit: 2 or 1 full 16-byte words + remainder.
    typedef float R;
    static constexpr int NQ = (NR * 2) / 16;
    static constexpr int REM = (NR * 2) % 16;  // 4 or 8
    static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<float> m[9])
    {
        const uint4 *q = reinterpret_cast<const uint4 *>(blk);
        uint32_t u[NR / 2];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            uint4 v = q[k * Ps + i];
            u[4 * k] = v.x; u[4 * k + 1] = v.y; u[4 * k + 2] = v.z; u[4 * k + 3] = v.w;
        }
        if constexpr (REM == 8) {
            uint2 v = reinterpret_cast<const uint2 *>(blk + NQ * Ps * 16)[i];
            u[4 * NQ] = v.x; u[4 * NQ + 1] = v.y;
        } else {
            u[4 * NQ] = reinterpret_cast<const uint32_t *>(blk + NQ * Ps * 16)[i];
        }
#pragma unroll
        for (int k = 0; k < NR / 2; ++k) {
            float2 f = H2<H>::to2(u[k]);
            m[k].re = f.x;
            m[k].im = f.y;
        }
        if constexpr (NR == 12) third_row(m);
    }
    static __device__ __forceinline__ void store(char *blk, int64_t Ps, int i, const double w[18])
    {
        uint32_t u[NR / 2];
#pragma unroll
        for (int k = 0; k < NR / 2; ++k) u[k] = H2<H>::from2d(w[2 * k], w[2 * k + 1]);
        uint4 *q = reinterpret_cast<uint4 *>(blk);
#pragma unroll
        for (int k = 0; k < NQ; ++k) q[k * Ps + i] = make_uint4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
        if constexpr (REM == 8)
            reinterpret_cast<uint2 *>(blk + NQ * Ps * 16)[i] = make_uint2(u[4 * NQ], u[4 * NQ + 1]);
        else
            reinterpret_cast<uint32_t *>(blk + NQ * Ps * 16)[i] = u[4 * NQ];
    }
};
template <> struct WFmt<W_F16_18> : WFmtH<__half, 18> {};
template <> struct WFmt<W_F16_12> : WFmtH<__half, 12> {};
template <> struct WFmt<W_BF16_18> : WFmtH<__nv_bfloat16, 18> {};
template <> struct WFmt<W_BF16_12> : WFmtH<__nv_bfloat16, 12> {};

// --------------------------------------------------------------------------
// Vector formats.  blk points at one (vector, block); site i.
//   F64 : 3 planes of double2 (one complex colour component each)
//   F32 : plane of float4 (colours 0, 1) + plane of float2 (colour 2)
//   F16 / BF16 : one plane of 16-byte records {3 x (re, im) 16-bit, float s};
//         the value is the stored number times s, s = max |re|, |im| of the
//         site (s = 0 stores zeros).
// --------------------------------------------------------------------------
template <int P> struct VFmt;

template <> struct VFmt<P_F64> {
    typedef double R;
    template <bool CG> static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<double> v[3])
    {
        const double2 *p = reinterpret_cast<const double2 *>(blk);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 a = vld<CG>(p + c * Ps + i);
            v[c].re = a.x;
            v[c].im = a.y;
        }
    }
    template <bool CG> static __device__ __forceinline__ void store(char *blk, int64_t Ps, int i, const cpx<double> v[3])
    {
        double2 *p = reinterpret_cast<double2 *>(blk);
#pragma unroll
        for (int c = 0; c < 3; ++c) vst<CG>(p + c * Ps + i, make_double2(v[c].re, v[c].im));
    }
};

template <> struct VFmt<P_F32> {
    typedef float R;
    template <bool CG> static __device__ __forceinline__ void load(const char *blk, int64_t Ps, int i, cpx<float> v[3])
    {
        float4 a = vld<CG>(reinterpret_cast<const float4 *>(blk) + i);
        float2 b = vld<CG>(reinterpret_cast<const float2 *>(blk + Ps * 16) + i);
        v[0].re = a.x; v[0].im = a.y; v[1].re = a.z; v[1].im = a.w; v[2].re = b.x; v[2].im = b.y;
    }
    template <bool CG> static __device__ __forceinline__ void store(char *blk, int64_t Ps, int i, const cpx<float> v[3])
    {
        vst<CG>(reinterpret_cast<float4 *>(blk) + i, make_float4(v[0].re, v[0].im, v[1].re, v[1].im));
        vst<CG>(reinterpret_cast<float2 *>(blk + Ps * 16) + i, make_float2(v[2].re, v[2].im));
    }
};

template <typename H> struct VFmtH {
    typedef float R;
    template <bool CG> static __device__ __forceinline__ void load(const char *blk, int64_t, int i, cpx<float> v[3])
    {
        uint4 a = vld<CG>(reinterpret_cast<const uint4 *>(blk) + i);
        const float s = __uint_as_float(a.w);
        const float2 s2 = make_float2(s, s);
        // packed FP32 multiplies: each lane rounds exactly as f * s
        const float2 f0 = __fmul2_rn(H2<H>::to2(a.x), s2), f1 = __fmul2_rn(H2<H>::to2(a.y), s2),
                     f2 = __fmul2_rn(H2<H>::to2(a.z), s2);
        v[0].re = f0.x; v[0].im = f0.y;
        v[1].re = f1.x; v[1].im = f1.y;
        v[2].re = f2.x; v[2].im = f2.y;
    }
    template <bool CG> static __device__ __forceinline__ void store(char *blk, int64_t, int i, const cpx<float> v[3])
    {
        float m = fmaxf(fmaxf(fmaxf(fabsf(v[0].re), fabsf(v[0].im)), fmaxf(fabsf(v[1].re), fabsf(v[1].im))),
                        fmaxf(fabsf(v[2].re), fabsf(v[2].im)));
        const float inv = m > 0.0f ? 1.0f / m : 0.0f;
        const float2 i2 = make_float2(inv, inv);
        const float2 q0 = __fmul2_rn(make_float2(v[0].re, v[0].im), i2);
        const float2 q1 = __fmul2_rn(make_float2(v[1].re, v[1].im), i2);
        const float2 q2 = __fmul2_rn(make_float2(v[2].re, v[2].im), i2);
        uint4 a;
        a.x = H2<H>::from2(q0.x, q0.y);
        a.y = H2<H>::from2(q1.x, q1.y);
        a.z = H2<H>::from2(q2.x, q2.y);
        a.w = __float_as_uint(m);
        vst<CG>(reinterpret_cast<uint4 *>(blk) + i, a);
    }
};
template <> struct VFmt<P_F16> : VFmtH<__half> {};
template <> struct VFmt<P_BF16> : VFmtH<__nv_bfloat16> {};

// --------------------------------------------------------------------------
// Interleaved (vector-innermost) records, per (slice, sublattice) block of
// Ps sites and nvec vectors:
//   F64 / F32: three colour planes; plane c holds, for every site i, the nvec
//              complex numbers of colour c contiguously: element (c, i, v) in
//              the 16 / 8 bytes at ((c * Ps + i) * nvec + v) * 16 / 8 from the
//              block (F32: the two vectors of a 16-byte word interleave their
//              real and imaginary parts, see VRec<P_F32>), so colour c of
//              consecutive sites is contiguous;
//   16-bit   : 16 bytes per (site, vector), vectors 2u and 2u + 1 of a site
//              sharing the 32-byte record at (i * nvec + 2u) * 16 bytes (see
//              VRecH).
// The block occupies Ps * nvec * vfmt_bytes bytes either way.  A site pointer
// is block + i * nvec * SB; colour planes are cs = Ps * nvec elements apart.
// A thread that owns VB vectors of a site reads vector units t, t + T, ...
// (T = nvec / VB threads per site), a unit being two vectors for F32 and
// 16-bit storage (one 16-byte word per colour, one 32-byte record), one for
// F64; F32 threads with VB = 4 own the adjacent units 2t, 2t+1 and read them
// with one 32-byte load per colour.  Consecutive lanes read consecutive words,
// across site boundaries too.
// --------------------------------------------------------------------------
template <int P> struct VRec;

template <> struct VRec<P_F64> {
    typedef double R;
    static constexpr int U = 1;   // vectors per 16-byte unit of one colour
    static constexpr int SB = 16; // site stride per vector (bytes)
    static __device__ __forceinline__ void load(const char *s, int cs, int w, cpx<double> v[3])
    {
        const double2 *p = reinterpret_cast<const double2 *>(s) + w;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2 a = p[c * cs];
            v[c].re = a.x;
            v[c].im = a.y;
        }
    }
    static __device__ __forceinline__ void store(char *s, int cs, int w, const cpx<double> v[3])
    {
        double2 *p = reinterpret_cast<double2 *>(s) + w;
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c * cs] = make_double2(v[c].re, v[c].im);
    }
};

// F32: in colour plane c of a site, vectors 2u and 2u + 1 share one 16-byte
// word {re_2u, re_2u+1, im_2u, im_2u+1}: a load gives the real parts and the
// imaginary parts of two vectors as aligned register pairs, the operands of
// the packed FP32 FMAs.  An F32 record group holds an even number of vectors.
template <> struct VRec<P_F32> {
    typedef float R;
    static constexpr int U = 2;
    static constexpr int SB = 8;
    static __device__ __forceinline__ void load(const char *s, int cs, int w, cpx<float> v[3])
    {
        const float *p = reinterpret_cast<const float *>(s) + 2 * (w & ~1) + (w & 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[c].re = p[2 * (int64_t)c * cs];
            v[c].im = p[2 * (int64_t)c * cs + 2];
        }
    }
    static __device__ __forceinline__ void store(char *s, int cs, int w, const cpx<float> v[3])
    {
        float *p = reinterpret_cast<float *>(s) + 2 * (w & ~1) + (w & 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p[2 * (int64_t)c * cs] = v[c].re;
            p[2 * (int64_t)c * cs + 2] = v[c].im;
        }
    }
    // unit u = vectors 2u, 2u+1: one 16-byte word per colour
    static __device__ __forceinline__ void load2(const char *s, int cs, int u, cpx<float> a[3], cpx<float> b[3])
    {
        const float4 *p = reinterpret_cast<const float4 *>(s) + u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 q = p[(int64_t)c * (cs >> 1)];
            a[c].re = q.x;
            b[c].re = q.y;
            a[c].im = q.z;
            b[c].im = q.w;
        }
    }
    static __device__ __forceinline__ void store2(char *s, int cs, int u, const cpx<float> a[3], const cpx<float> b[3])
    {
        float4 *p = reinterpret_cast<float4 *>(s) + u;
#pragma unroll
        for (int c = 0; c < 3; ++c) p[(int64_t)c * (cs >> 1)] = make_float4(a[c].re, b[c].re, a[c].im, b[c].im);
    }
    // units 2u2, 2u2+1 = vectors 4u2 .. 4u2+3 of colour c as (re, im) pairs of
    // the vector pairs: re[j] = (re_{4u2+2j}, re_{4u2+2j+1}), im[j] alike.
    // One 32-byte global load.
    static __device__ __forceinline__ void load4g_pairs(const char *s, int cs, int u2, int c, float2 re[2],
                                                        float2 im[2])
    {
        const float *p = reinterpret_cast<const float *>(s) + 2 * ((int64_t)c * cs + 4 * u2);
        asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(re[0].x), "=f"(re[0].y), "=f"(im[0].x), "=f"(im[0].y), "=f"(re[1].x), "=f"(re[1].y),
                       "=f"(im[1].x), "=f"(im[1].y)
                     : "l"(p));
    }
    static __device__ __forceinline__ void store4g_pairs(char *s, int cs, int u2, int c, const float2 re[2],
                                                         const float2 im[2])
    {
        float *p = reinterpret_cast<float *>(s) + 2 * ((int64_t)c * cs + 4 * u2);
        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(re[0].x),
                     "f"(re[0].y), "f"(im[0].x), "f"(im[0].y), "f"(re[1].x), "f"(re[1].y), "f"(im[1].x), "f"(im[1].y)
                     : "memory");
    }
    // units 2u2, 2u2+1 = vectors 4u2 .. 4u2+3: one 32-byte global load / store per colour
    static __device__ __forceinline__ void load4g(const char *s, int cs, int u2, cpx<float> v[4][3])
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 re[2], im[2];
            load4g_pairs(s, cs, u2, c, re, im);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                v[2 * j][c].re = re[j].x;
                v[2 * j + 1][c].re = re[j].y;
                v[2 * j][c].im = im[j].x;
                v[2 * j + 1][c].im = im[j].y;
            }
        }
    }
    static __device__ __forceinline__ void store4g(char *s, int cs, int u2, const cpx<float> v[4][3])
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 re[2], im[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                re[j] = make_float2(v[2 * j][c].re, v[2 * j + 1][c].re);
                im[j] = make_float2(v[2 * j][c].im, v[2 * j + 1][c].im);
            }
            store4g_pairs(s, cs, u2, c, re, im);
        }
    }
};

// 16-bit: vectors 2u and 2u + 1 of a site share one 32-byte record of eight
// 32-bit words: {re_2u, re_2u+1} and {im_2u, im_2u+1} of colours 0, 1, 2 as
// 16-bit pairs, then the FP32 scales s_2u, s_2u+1 (value = stored number
// times s; s = max |re|, |im| over the vector's six reals at that site, s = 0
// storing zeros).  A conversion of one word gives the real or imaginary parts
// of two vectors as an aligned FP32 pair.  A 16-bit record group holds an even
// number of vectors.
template <typename H> struct VRecH {
    typedef float R;
    static constexpr int U = 2;
    static constexpr int SB = 16;
    // quantise one vector: scale and the six 16-bit values (RN), as the planar format does
    static __device__ __forceinline__ float quant(const cpx<float> v[3], float q[6])
    {
        const float m = fmaxf(fmaxf(fmaxf(fabsf(v[0].re), fabsf(v[0].im)), fmaxf(fabsf(v[1].re), fabsf(v[1].im))),
                              fmaxf(fabsf(v[2].re), fabsf(v[2].im)));
        const float inv = m > 0.0f ? 1.0f / m : 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q[2 * c] = __fmul_rn(v[c].re, inv);
            q[2 * c + 1] = __fmul_rn(v[c].im, inv);
        }
        return m;
    }
    static __device__ __forceinline__ void load(const char *s, int, int w, cpx<float> v[3])
    {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(s + (w >> 1) * 32);
        const int l = w & 1;
        const float sc = __uint_as_float(p[6 + l]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 re = H2<H>::to2(p[2 * c]), im = H2<H>::to2(p[2 * c + 1]);
            v[c].re = __fmul_rn(l ? re.y : re.x, sc);
            v[c].im = __fmul_rn(l ? im.y : im.x, sc);
        }
    }
    static __device__ __forceinline__ void store(char *s, int, int w, const cpx<float> v[3])
    {
        float q[6];
        const float m = quant(v, q);
        char *b = s + (w >> 1) * 32 + (w & 1) * 2;  // this vector's half of each 16-bit pair
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const uint32_t h = H2<H>::from2(q[k], 0.0f);
            *reinterpret_cast<unsigned short *>(b + 4 * k) = (unsigned short)(h & 0xffffu);
        }
        reinterpret_cast<float *>(s + (w >> 1) * 32)[6 + (w & 1)] = m;
    }
    // unit u = vectors 2u, 2u+1: the whole 32-byte record
    static __device__ __forceinline__ void load2(const char *s, int, int u, cpx<float> a[3], cpx<float> b[3])
    {
        float2 re[3], im[3];
        load_pairs<false>(s, u, re, im);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c].re = re[c].x;
            b[c].re = re[c].y;
            a[c].im = im[c].x;
            b[c].im = im[c].y;
        }
    }
    static __device__ __forceinline__ void store2(char *s, int, int u, const cpx<float> a[3], const cpx<float> b[3])
    {
        float2 re[3], im[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            re[c] = make_float2(a[c].re, b[c].re);
            im[c] = make_float2(a[c].im, b[c].im);
        }
        store_pairs<false>(s, u, re, im);
    }
    // unit u as FP32 pairs over its two vectors: re[c] = (re_2u, re_2u+1) of colour c, im[c] alike
    // GM: s is global memory (one 32-byte load / store per record)
    template <bool GM = true>
    static __device__ __forceinline__ void load_pairs(const char *s, int u, float2 re[3], float2 im[3])
    {
        uint4 x, y;
        if constexpr (GM) {
            asm volatile("ld.global.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(x.x), "=r"(x.y), "=r"(x.z), "=r"(x.w), "=r"(y.x), "=r"(y.y), "=r"(y.z), "=r"(y.w)
                         : "l"(s + u * 32));
        } else {
            const uint4 *p = reinterpret_cast<const uint4 *>(s + u * 32);
            x = p[0];
            y = p[1];
        }
        const float2 sc = make_float2(__uint_as_float(y.z), __uint_as_float(y.w));
        re[0] = __fmul2_rn(H2<H>::to2(x.x), sc);
        im[0] = __fmul2_rn(H2<H>::to2(x.y), sc);
        re[1] = __fmul2_rn(H2<H>::to2(x.z), sc);
        im[1] = __fmul2_rn(H2<H>::to2(x.w), sc);
        re[2] = __fmul2_rn(H2<H>::to2(y.x), sc);
        im[2] = __fmul2_rn(H2<H>::to2(y.y), sc);
    }
    template <bool GM = true>
    static __device__ __forceinline__ void store_pairs(char *s, int u, const float2 re[3], const float2 im[3])
    {
        cpx<float> a[3], b[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c].re = re[c].x;
            a[c].im = im[c].x;
            b[c].re = re[c].y;
            b[c].im = im[c].y;
        }
        float qa[6], qb[6];
        const float ma = quant(a, qa), mb = quant(b, qb);
        uint4 x, y;
        x.x = H2<H>::from2(qa[0], qb[0]);
        x.y = H2<H>::from2(qa[1], qb[1]);
        x.z = H2<H>::from2(qa[2], qb[2]);
        x.w = H2<H>::from2(qa[3], qb[3]);
        y.x = H2<H>::from2(qa[4], qb[4]);
        y.y = H2<H>::from2(qa[5], qb[5]);
        y.z = __float_as_uint(ma);
        y.w = __float_as_uint(mb);
        if constexpr (GM) {
            asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(s + u * 32), "r"(x.x),
                         "r"(x.y), "r"(x.z), "r"(x.w), "r"(y.x), "r"(y.y), "r"(y.z), "r"(y.w)
                         : "memory");
        } else {
            uint4 *p = reinterpret_cast<uint4 *>(s + u * 32);
            p[0] = x;
            p[1] = y;
        }
    }
};
template <> struct VRec<P_F16> : VRecH<__half> {};
template <> struct VRec<P_BF16> : VRecH<__nv_bfloat16> {};

// Bytes between consecutive sites' records in the interleaved layout, per vector.
__host__ __device__ constexpr int il_site_bytes(int prec) { return prec == P_F64 ? 16 : prec == P_F32 ? 8 : 16; }
// Whether the interleaved layout splits colours into planes.
__host__ __device__ constexpr bool il_planes(int prec) { return prec == P_F64 || prec == P_F32; }

// F32 threads with four or eight vectors own adjacent units (32-byte loads).
template <int VP, int VB> __host__ __device__ constexpr bool il_adj4() { return VP == P_F32 && VB % 4 == 0; }

// Vector index of the k-th of the VB vectors that thread t (of T = nvec / VB
// per site) owns.
template <int VP, int VB> __device__ __forceinline__ int il_vec(int t, int T, int k)
{
    if constexpr (il_adj4<VP, VB>()) {
        return VB * t + k;
    } else {
        constexpr int U = VB % VRec<VP>::U == 0 ? VRec<VP>::U : 1;
        return (t + (k / U) * T) * U + k % U;
    }
}

// The VB vectors of thread t at site pointer s (colour planes cs elements
// apart).  GM: s is global memory (32-byte loads allowed).
template <int VP, int VB, bool GM = true> struct RecGroup {
    typedef typename VRec<VP>::R R;
    static constexpr bool PAIRS = VRec<VP>::U == 2 && VB % 2 == 0;
    static __device__ __forceinline__ void load(const char *s, int cs, int t, int T, cpx<R> v[VB][3])
    {
        if constexpr (il_adj4<VP, VB>()) {
#pragma unroll
            for (int j = 0; j < VB / 4; ++j) {
                const int q = VB / 4 * t + j;  // vectors 4q .. 4q+3
                if constexpr (GM) {
                    VRec<VP>::load4g(s, cs, q, v + 4 * j);
                } else {
                    VRec<VP>::load2(s, cs, 2 * q, v[4 * j], v[4 * j + 1]);
                    VRec<VP>::load2(s, cs, 2 * q + 1, v[4 * j + 2], v[4 * j + 3]);
                }
            }
        } else if constexpr (PAIRS) {
#pragma unroll
            for (int j = 0; j < VB / 2; ++j) VRec<VP>::load2(s, cs, t + j * T, v[2 * j], v[2 * j + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < VB; ++k) VRec<VP>::load(s, cs, t + k * T, v[k]);
        }
    }
    static __device__ __forceinline__ void store(char *s, int cs, int t, int T, const cpx<R> v[VB][3])
    {
        if constexpr (il_adj4<VP, VB>()) {
#pragma unroll
            for (int j = 0; j < VB / 4; ++j) {
                const int q = VB / 4 * t + j;
                if constexpr (GM) {
                    VRec<VP>::store4g(s, cs, q, v + 4 * j);
                } else {
                    VRec<VP>::store2(s, cs, 2 * q, v[4 * j], v[4 * j + 1]);
                    VRec<VP>::store2(s, cs, 2 * q + 1, v[4 * j + 2], v[4 * j + 3]);
                }
            }
        } else if constexpr (PAIRS) {
#pragma unroll
            for (int j = 0; j < VB / 2; ++j) VRec<VP>::store2(s, cs, t + j * T, v[2 * j], v[2 * j + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < VB; ++k) VRec<VP>::store(s, cs, t + k * T, v[k]);
        }
    }
};

// (re, im) -> (im, re): the second operand pair of a packed complex multiply-add.
__device__ __forceinline__ float2 f2swap(float2 a) { return make_float2(a.y, a.x); }

// The six +-1 sublattice neighbours of site i (periodic in h).
__device__ __forceinline__ void sub_neighbours(const SubGeom &g, int i, int fw[3], int bw[3])
{
    int xq = i % g.hx;
    int r = i / g.hx;
    int yq = r % g.hy;
    int zq = r / g.hy;
    int sy = g.hx, sz = g.hx * g.hy;
    fw[0] = xq == g.hx - 1 ? i - (g.hx - 1) : i + 1;
    bw[0] = xq == 0 ? i + (g.hx - 1) : i - 1;
    fw[1] = yq == g.hy - 1 ? i - (g.hy - 1) * sy : i + sy;
    bw[1] = yq == 0 ? i + (g.hy - 1) * sy : i - sy;
    fw[2] = zq == g.hz - 1 ? i - (g.hz - 1) * sz : i + sz;
    bw[2] = zq == 0 ? i + (g.hz - 1) * sz : i - sz;
}

}  // namespace tls
