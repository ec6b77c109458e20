// k_ilt.cuh -- multi-RHS smearing step with the W rows staged by TMA bulk copies.
//
// The step of Sec. 2 (Eq. tlSmear with Eq. tlLapl1) on the interleaved
// (vector-innermost, vector-pair) layout, with the per-vector FMA sequence of
// site_step: results are bitwise equal to every other kernel of the library.
//
// Work decomposition: a CTA owns one whole x'-row of one (slice, sublattice)
// block and one group of the vectors; thread (threadIdx.x, threadIdx.y) takes
// VB vectors of the group at site x' = threadIdx.y.  Because the row is whole
// and periodic in x', the five W rows it needs are plain contiguous segments:
//   set 0  W_x of the row itself   (x forward at x', x backward at x' - 1)
//   set 1  W_y of row y'           (y forward)
//   set 2  W_y of row y' - 1       (y backward)
//   set 3  W_z of row y'           (z forward)
//   set 4  W_z of row y' in z' - 1 (z backward)
// The leader thread initialises one mbarrier, copies the five rows into
// shared memory in their stored format with cp.async.bulk (one copy per
// 16-byte plane segment, completion counted in transaction bytes) and waits;
// the other threads request the records of their first hop and wait at the
// CTA barrier, so the staging takes none of their load/store instructions.
//
// Arithmetic: a record load yields the real parts (re_a, re_b) and the
// imaginary parts (im_a, im_b) of a vector pair.  With W element (wr, wi)
// broadcast as {wr, wr} and {wi, wi}, one complex multiply-add is four
// packed FMAs (fma.rn.f32x2):
//   forward  W(r, c):      R += {wr}*re + {wi}*(-im);  I += {wr}*im + {wi}*re
//   backward conj W(c, r): R += {wr}*re + {wi}*im;     I += {wr}*im + {wi}*(-re)
// with the negated pair formed once per record and colour; lane by lane this
// is the FMA sequence of cmac / cmacc.
//
// Variants (tile[1] of the tune entry): 6 the plain form; 7 the records of
// the next hop requested before the current hop is applied; 8 the row's own
// records copied in with the W rows (the centre and the x neighbours then
// come from shared memory).  tile[2] > 0 (or < 0 for an automatic distance):
// the leader also asks L2 for the W rows and records of the row that many
// planes ahead in launch order, so their first DRAM touch happens before the
// CTA that needs them waits for it.
//
// The wait is bounded: if it runs out the CTA sets DERR_TIMEOUT, waits once
// more (bounded) for its own copies in flight and returns without writing.
#pragma once

#include "tls_dev.cuh"
#include "tls_internal.h"
#include "tma.cuh"

namespace tls {

// Shared-memory bytes of the k_step_ilt CTA: the mbarrier (128 bytes) and the five W rows.
inline int ilt_smem(int hx, int wb) { return 128 + 5 * hx * wb; }

// Whether the TMA staging applies: every plane segment of a W row starts and
// ends on a 16-byte boundary (the remainder plane has 4 or 8 bytes per site).
inline bool ilt_ok(int wfmt, const SubGeom &g)
{
    const int rem = wfmt_bytes(wfmt) % 16;
    return rem == 0 || (g.hx * rem) % 16 == 0;
}

// Issues the bulk copies of the five W rows of row (blk, zq, yq) into the
// sets at ws (one elected thread); completion lands on bar.
template <int WF>
__device__ __forceinline__ void ilt_issue_w(char *ws, const char *__restrict__ W, const SubGeom &g, int blk, int zq,
                                            int yq, uint64_t *bar)
{
    constexpr int WB = wfmt_bytes(WF);
    constexpr int NQ = WB / 16, REM = WB % 16;
    const int hx = g.hx, setB = hx * WB;
    const int sy = hx, sz = hx * g.hy;
    const int row = zq * sz + yq * sy;
    const int ym = yq == 0 ? g.hy - 1 : yq - 1;
    const int zm = zq == 0 ? g.hz - 1 : zq - 1;
    const char *wb = W + (int64_t)blk * 3 * g.Ps * WB;
    const int srow[5] = {row, row, zq * sz + ym * sy, row, zm * sz + yq * sy};
    mbar_expect_tx(bar, 5u * (unsigned)setB);
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const char *wd = wb + (int64_t)((s + 1) >> 1) * g.Ps * WB;  // direction of set s
        char *dst = ws + s * setB;
#pragma unroll
        for (int j = 0; j < NQ; ++j)
            bulk_load(dst + j * hx * 16, wd + ((int64_t)j * g.Ps + srow[s]) * 16, (unsigned)(hx * 16), bar);
        if constexpr (REM > 0)
            bulk_load(dst + NQ * hx * 16, wd + (int64_t)NQ * g.Ps * 16 + (int64_t)srow[s] * REM, (unsigned)(hx * REM),
                      bar);
    }
}

// Requests into L2 the data that the CTA pfd planes (grid z) further on in
// launch order reads first: the W rows of the three directions at its row
// and the records of its row (all vectors).  Every row of the launch is
// requested once, by the CTA pfd planes before it, so the DRAM reads run
// ahead of the CTAs that use them.  Issued by the leader of the CTAs with
// blockIdx.x == 0; a request is a hint and changes no result.
template <int VP, int WF>
__device__ __forceinline__ void ilt_prefetch_ahead(const char *__restrict__ W, const char *__restrict__ in,
                                                   const SubGeom &g, int nvec, int pfd)
{
    const unsigned z2 = blockIdx.z + (unsigned)pfd;
    if (z2 >= gridDim.z) return;
    const int blk = (int)z2 / g.hz, zq = (int)z2 - blk * g.hz;
    const int64_t row = (int64_t)zq * g.hy * g.hx + (int64_t)blockIdx.y * g.hx;
    constexpr int WB = wfmt_bytes(WF), NQ = WB / 16, REM = WB % 16;
    const char *wb = W + (int64_t)blk * 3 * g.Ps * WB;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const char *wd = wb + (int64_t)d * g.Ps * WB;
#pragma unroll
        for (int j = 0; j < NQ; ++j) l2_prefetch(wd + ((int64_t)j * g.Ps + row) * 16, (unsigned)(g.hx * 16));
        if constexpr (REM > 0) l2_prefetch(wd + (int64_t)NQ * g.Ps * 16 + row * REM, (unsigned)(g.hx * REM));
    }
    constexpr int VBY = vfmt_bytes(VP);
    const char *rb = in + (int64_t)blk * g.Ps * nvec * VBY;
    if constexpr (VP == P_F32) {
        if (nvec % 2 == 0)  // 16-byte aligned colour-plane rows
#pragma unroll
            for (int c = 0; c < 3; ++c)
                l2_prefetch(rb + ((int64_t)c * g.Ps + row) * nvec * 8, (unsigned)(g.hx * nvec * 8));
    } else {
        l2_prefetch(rb + row * nvec * VBY, (unsigned)(g.hx * nvec * VBY));
    }
}

// One thread's part of a row: site x' = k of row (blk, zq, yq), vector units
// t of T (VB vectors each), W rows staged at ws.  pl holds the records of the
// first hop (requested before the wait on the copies).
template <int VP, int WF, int VB, bool ACT, bool PF = false> struct IltSite {
    int nb[6];  // the six hops in the order of site_step
    int i;
    const char *rin;
    char *rout;
    unsigned rstride;
    int cs;
    bool on[VB];
    bool any, all;
    // Records as vector pairs, real and imaginary lanes split (the layouts of
    // VRec<P_F32> and VRecH): re[j][c] = (re_a, re_b) of vectors a, b of pair
    // j, im[j][c] alike.  Odd VB: complex records.
    static constexpr bool PAIRS = VB % 2 == 0;
    static constexpr int NP = PAIRS ? VB / 2 : 1;
    float2 pre[NP][3], pim[NP][3];
    cpx<float> pl[PAIRS ? 1 : VB][3];

    // the records of this thread's vectors at site pointer s
    __device__ __forceinline__ void load_rec(const char *s) { load_rec_to(s, pre, pim); }
    __device__ __forceinline__ void load_rec_to(const char *s, float2 (&pre)[NP][3], float2 (&pim)[NP][3])
    {
        if constexpr (PAIRS && VP != P_F32) {  // 16-bit: one 32-byte record per pair, dequantised
#pragma unroll
            for (int j = 0; j < NP; ++j) VRec<VP>::load_pairs(s, tt + j * TT, pre[j], pim[j]);
        } else if constexpr (PAIRS) {
            if constexpr (VB % 4 == 0) {
#pragma unroll
                for (int j = 0; j < VB / 4; ++j)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float2 r2[2], i2[2];
                        VRec<P_F32>::load4g_pairs(s, cs, VB / 4 * tt + j, c, r2, i2);
                        pre[2 * j][c] = r2[0];
                        pre[2 * j + 1][c] = r2[1];
                        pim[2 * j][c] = i2[0];
                        pim[2 * j + 1][c] = i2[1];
                    }
            } else {  // VB = 2: one 16-byte word per colour
                const float4 *p = reinterpret_cast<const float4 *>(s) + tt;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 q = p[(int64_t)c * (cs >> 1)];
                    pre[0][c] = make_float2(q.x, q.y);
                    pim[0][c] = make_float2(q.z, q.w);
                }
            }
        } else {
            RecGroup<VP, VB>::load(s, cs, tt, TT, pl);
        }
    }
    int tt, TT;
    // RB: the records of the site's own row in shared memory (the global
    // layout of the row, colour planes rcs elements apart), for the x
    // neighbours and the centre
    const char *rbuf = nullptr;
    int rcs = 0;
    __device__ __forceinline__ void load_rec_row(int kk, float2 (&pre)[NP][3], float2 (&pim)[NP][3])
    {
        const char *s = rbuf + (unsigned)kk * rstride;
        if constexpr (PAIRS && VP != P_F32) {
#pragma unroll
            for (int j = 0; j < NP; ++j) VRec<VP>::template load_pairs<false>(s, tt + j * TT, pre[j], pim[j]);
        } else if constexpr (PAIRS) {
            if constexpr (VB % 4 == 0) {
#pragma unroll
                for (int j = 0; j < VB / 4; ++j)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float4 *p = reinterpret_cast<const float4 *>(s) + (c * rcs + 4 * (VB / 4 * tt + j)) / 2;
                        const float4 a = p[0], b = p[1];
                        pre[2 * j][c] = make_float2(a.x, a.y);
                        pim[2 * j][c] = make_float2(a.z, a.w);
                        pre[2 * j + 1][c] = make_float2(b.x, b.y);
                        pim[2 * j + 1][c] = make_float2(b.z, b.w);
                    }
            } else {
                const float4 *p = reinterpret_cast<const float4 *>(s) + tt;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float4 q = p[c * (rcs >> 1)];
                    pre[0][c] = make_float2(q.x, q.y);
                    pim[0][c] = make_float2(q.z, q.w);
                }
            }
        }
    }

    __device__ __forceinline__ void setup(const char *__restrict__ in, char *__restrict__ out,
                                          const int *__restrict__ active, const SubGeom &g, int nvec, int blk, int zq,
                                          int yq, int k, int t, int T)
    {
        constexpr int VBY = vfmt_bytes(VP);
        const int hx = g.hx, sy = hx, sz = hx * g.hy;
        i = zq * sz + yq * sy + k;
        nb[0] = k == hx - 1 ? i - (hx - 1) : i + 1;
        nb[1] = k == 0 ? i + (hx - 1) : i - 1;
        nb[2] = yq == g.hy - 1 ? i - (g.hy - 1) * sy : i + sy;
        nb[3] = yq == 0 ? i + (g.hy - 1) * sy : i - sy;
        nb[4] = zq == g.hz - 1 ? i - (g.hz - 1) * sz : i + sz;
        nb[5] = zq == 0 ? i + (g.hz - 1) * sz : i - sz;
        rin = in + (int64_t)blk * g.Ps * nvec * VBY;
        rout = out + (int64_t)blk * g.Ps * nvec * VBY;
        rstride = (unsigned)nvec * VRec<VP>::SB;  // site stride
        cs = g.Ps * nvec;                         // colour planes
        // ACT (serving): vectors whose slot is inactive are not stored
        any = false;
        all = true;
#pragma unroll
        for (int v = 0; v < VB; ++v) {
            on[v] = !ACT || active[il_vec<VP, VB>(t, T, v)] != 0;
            any = any || on[v];
            all = all && on[v];
        }
        tt = t;
        TT = T;
        if (any && !rbuf) {  // RB: the first hops come from the staged row
            if constexpr (COLS)
                load_col(rin + (unsigned)nb[0] * rstride, 0, pre0, pim0);
            else
                load_rec(rin + (unsigned)nb[0] * rstride);
        }
    }

    // FP32 with VB = 8: records are read one colour at a time (two 32-byte
    // loads), so only one colour of the four vector pairs is live.
    static constexpr bool COLS = VP == P_F32 && VB == 8;
    float2 pre0[COLS ? 4 : 1], pim0[COLS ? 4 : 1];  // colour 0 of the first hop
    __device__ __forceinline__ void load_col(const char *s, int c, float2 re[4], float2 im[4])
    {
#pragma unroll
        for (int j = 0; j < 2; ++j) VRec<P_F32>::load4g_pairs(s, cs, 2 * tt + j, c, re + 2 * j, im + 2 * j);
    }

    __device__ __forceinline__ void compute(const char *ws, int hx, int k, int t, int T,
                                            const float *__restrict__ alphaf)
    {
        if constexpr (COLS)
            compute_cols(ws, hx, k, t, T, alphaf);
        else if constexpr (PAIRS)
            compute_pairs(ws, hx, k, t, T, alphaf);
        else
            compute_cpx(ws, hx, k, t, T, alphaf);
    }

    // The element of the stored W matrix the hop uses for row r, column c.
    __device__ __forceinline__ cpx<float> w_elem(const char *wset, int hx, int wk, const cpx<float> *m, bool dag,
                                                 int r, int c)
    {
        cpx<float> w;
        if constexpr (WF == W_F32_18) {
            // element e of a stored f32-18 matrix: one 8-byte word, read when used
            const int e = dag ? c * 3 + r : r * 3 + c;
            const float2 f = e < 8 ? reinterpret_cast<const float2 *>(wset)[((e >> 1) * hx + wk) * 2 + (e & 1)]
                                   : reinterpret_cast<const float2 *>(wset + 4 * hx * 16)[wk];
            w.re = f.x;
            w.im = f.y;
        } else {
            w = dag ? m[c * 3 + r] : m[r * 3 + c];
        }
        return w;
    }

    // compute_pairs for FP32 with VB = 8, one colour of the records at a time.
    __device__ __forceinline__ void compute_cols(const char *ws, int hx, int k, int t, int T,
                                                 const float *__restrict__ alphaf)
    {
        constexpr int WB = wfmt_bytes(WF);
        const int setB = hx * WB;
        float2 accR[4][3], accI[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 3; ++r) accR[j][r] = accI[j][r] = make_float2(0.f, 0.f);
        const int km = k == 0 ? hx - 1 : k - 1;
        const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const bool dag = q & 1;
            const char *rs = rin + (unsigned)nb[q] * rstride;
            const char *wset = ws + (q == 0 ? 0 : q - 1) * setB;
            const int wk = q == 1 ? km : k;
            cpx<float> m[WF == W_F32_18 ? 1 : 9];
            if constexpr (WF != W_F32_18) WFmt<WF>::load(wset, hx, wk, m);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 re[4], im[4], ng[4];
                if (q == 0 && c == 0) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        re[j] = pre0[j];
                        im[j] = pim0[j];
                    }
                } else {
                    load_col(rs, c, re, im);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) ng[j] = __fmul2_rn(dag ? re[j] : im[j], neg1);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const cpx<float> w = w_elem(wset, hx, wk, m, dag, r, c);
                    const float2 wr = make_float2(w.re, w.re), wi = make_float2(w.im, w.im);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        accR[j][r] = __ffma2_rn(wr, re[j], accR[j][r]);
                        accR[j][r] = __ffma2_rn(wi, dag ? im[j] : ng[j], accR[j][r]);
                        accI[j][r] = __ffma2_rn(wr, im[j], accI[j][r]);
                        accI[j][r] = __ffma2_rn(wi, dag ? ng[j] : re[j], accI[j][r]);
                    }
                }
            }
        }
        const float2 m6 = make_float2(-6.f, -6.f);
        float2 a2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a2[j] = *reinterpret_cast<const float2 *>(alphaf + il_vec<VP, VB>(t, T, 2 * j));
        const char *sc = rin + (unsigned)i * rstride;
        char *so = rout + (unsigned)i * rstride;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 re[4], im[4];
            load_col(sc, c, re, im);  // the centre
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                re[j] = __ffma2_rn(a2[j], __ffma2_rn(m6, re[j], accR[j][c]), re[j]);
                im[j] = __ffma2_rn(a2[j], __ffma2_rn(m6, im[j], accI[j][c]), im[j]);
            }
            if (all) {
#pragma unroll
                for (int j = 0; j < 2; ++j) VRec<P_F32>::store4g_pairs(so, cs, 2 * t + j, c, re + 2 * j, im + 2 * j);
            } else {
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    if (on[v]) {
                        float *p = reinterpret_cast<float *>(so) + 2 * ((int64_t)c * cs + (8 * t + (v & ~1))) + (v & 1);
                        p[0] = (v & 1) ? re[v >> 1].y : re[v >> 1].x;
                        p[2] = (v & 1) ? im[v >> 1].y : im[v >> 1].x;
                    }
            }
        }
    }

    // FP32 storage.  Per element w of a hop and vector pair j, with the negated
    // pair of the record (-im for a forward hop, -re for a backward one):
    //   forward  W(r, c):       R += {wr} re;  R += {wi} (-im);  I += {wr} im;  I += {wi} re
    //   backward conj W(c, r):  R += {wr} re;  R += {wi} im;     I += {wr} im;  I += {wi} (-re)
    // ({x} = the pair (x, x)): lane by lane the FMA sequence of cmac / cmacc,
    // products with a negated factor being exact negations.
    // PF: the records of hop q + 1 (the centre after hop 5) are requested
    // before hop q is applied, two record buffers alternating.
    __device__ __forceinline__ void compute_pairs(const char *ws, int hx, int k, int t, int T,
                                                  const float *__restrict__ alphaf)
    {
        constexpr int WB = wfmt_bytes(WF);
        const int setB = hx * WB;
        float2 qre[NP][3], qim[NP][3];  // the other buffer of the prefetch
        float2 accR[NP][3], accI[NP][3];
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int r = 0; r < 3; ++r) accR[j][r] = accI[j][r] = make_float2(0.f, 0.f);
        const int km = k == 0 ? hx - 1 : k - 1;
        const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const bool from_row = rbuf && q < 2;  // RB: x neighbours from the staged row
            if constexpr (PF) {
                const char *nx = rin + (unsigned)(q < 5 ? nb[q + 1] : i) * rstride;
                if (q & 1)
                    load_rec_to(nx, pre, pim);
                else
                    load_rec_to(nx, qre, qim);
            } else if (from_row) {
                load_rec_row(q == 0 ? (k == hx - 1 ? 0 : k + 1) : km, qre, qim);
            } else if (q > 0) {
                load_rec(rin + (unsigned)nb[q] * rstride);
            }
            float2 (&cre)[NP][3] = ((PF && (q & 1)) || from_row) ? qre : pre;
            float2 (&cim)[NP][3] = ((PF && (q & 1)) || from_row) ? qim : pim;
            const bool dag = q & 1;
            const char *wset = ws + (q == 0 ? 0 : q - 1) * setB;
            const int wk = q == 1 ? km : k;
            cpx<float> m[WF == W_F32_18 ? 1 : 9];
            if constexpr (WF != W_F32_18) WFmt<WF>::load(wset, hx, wk, m);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 ng[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) ng[j] = __fmul2_rn(dag ? cre[j][c] : cim[j][c], neg1);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    cpx<float> w;
                    if constexpr (WF == W_F32_18) {
                        // element e of a stored f32-18 matrix: one 8-byte word, read when used
                        const int e = dag ? c * 3 + r : r * 3 + c;
                        const float2 f = e < 8 ? reinterpret_cast<const float2 *>(wset)[((e >> 1) * hx + wk) * 2 + (e & 1)]
                                               : reinterpret_cast<const float2 *>(wset + 4 * hx * 16)[wk];
                        w.re = f.x;
                        w.im = f.y;
                    } else {
                        w = dag ? m[c * 3 + r] : m[r * 3 + c];
                    }
                    const float2 wr = make_float2(w.re, w.re), wi = make_float2(w.im, w.im);
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        accR[j][r] = __ffma2_rn(wr, cre[j][c], accR[j][r]);
                        accR[j][r] = __ffma2_rn(wi, dag ? cim[j][c] : ng[j], accR[j][r]);
                        accI[j][r] = __ffma2_rn(wr, cim[j][c], accI[j][r]);
                        accI[j][r] = __ffma2_rn(wi, dag ? ng[j] : cre[j][c], accI[j][r]);
                    }
                }
            }
        }
        if constexpr (!PF) {  // the centre (PF: loaded during hop 5)
            if (rbuf)
                load_rec_row(k, pre, pim);
            else
                load_rec(rin + (unsigned)i * rstride);
        }
        const float2 m6 = make_float2(-6.f, -6.f);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const int v0 = il_vec<VP, VB>(t, T, 2 * j);  // even: the pair's alphas are one aligned float2
            const float2 a2 = *reinterpret_cast<const float2 *>(alphaf + v0);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                pre[j][r] = __ffma2_rn(a2, __ffma2_rn(m6, pre[j][r], accR[j][r]), pre[j][r]);
                pim[j][r] = __ffma2_rn(a2, __ffma2_rn(m6, pim[j][r], accI[j][r]), pim[j][r]);
            }
        }
        char *so = rout + (unsigned)i * rstride;
        if constexpr (VP != P_F32) {
            if (all) {
#pragma unroll
                for (int j = 0; j < NP; ++j) VRec<VP>::store_pairs(so, t + j * T, pre[j], pim[j]);
                return;
            }
        }
        if (all) {
            if constexpr (VB % 4 == 0) {
#pragma unroll
                for (int j = 0; j < VB / 4; ++j)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 r2[2] = {pre[2 * j][c], pre[2 * j + 1][c]};
                        const float2 i2[2] = {pim[2 * j][c], pim[2 * j + 1][c]};
                        VRec<P_F32>::store4g_pairs(so, cs, VB / 4 * t + j, c, r2, i2);
                    }
            } else {
                float4 *p = reinterpret_cast<float4 *>(so) + t;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    p[(int64_t)c * (cs >> 1)] = make_float4(pre[0][c].x, pre[0][c].y, pim[0][c].x, pim[0][c].y);
            }
        } else {
#pragma unroll
            for (int v = 0; v < VB; ++v)
                if (on[v]) {
                    cpx<float> o[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        o[c].re = (v & 1) ? pre[v >> 1][c].y : pre[v >> 1][c].x;
                        o[c].im = (v & 1) ? pim[v >> 1][c].y : pim[v >> 1][c].x;
                    }
                    VRec<VP>::store(so, cs, il_vec<VP, VB>(t, T, v), o);
                }
        }
    }

    __device__ __forceinline__ void compute_cpx(const char *ws, int hx, int k, int t, int T,
                                                const float *__restrict__ alphaf)
    {
        constexpr int WB = wfmt_bytes(WF);
        const int setB = hx * WB;
        float2 acc[VB][3];
#pragma unroll
        for (int v = 0; v < VB; ++v)
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[v][r] = make_float2(0.f, 0.f);
        const int km = k == 0 ? hx - 1 : k - 1;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            if (q > 0) RecGroup<VP, VB>::load(rin + (unsigned)nb[q] * rstride, cs, t, T, pl);
            const bool dag = q & 1;
            cpx<float> m[9];
            WFmt<WF>::load(ws + (q == 0 ? 0 : q - 1) * setB, hx, q == 1 ? km : k, m);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 p[VB], ps[VB];
#pragma unroll
                for (int v = 0; v < VB; ++v) {
                    p[v] = make_float2(pl[v][c].re, pl[v][c].im);
                    ps[v] = f2swap(p[v]);
                }
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const cpx<float> w = dag ? m[c * 3 + r] : m[r * 3 + c];
                    const float2 wa = make_float2(w.re, w.re);
                    const float2 wc = dag ? make_float2(w.im, -w.im) : make_float2(-w.im, w.im);
#pragma unroll
                    for (int v = 0; v < VB; ++v) {
                        acc[v][r] = __ffma2_rn(wa, p[v], acc[v][r]);
                        acc[v][r] = __ffma2_rn(wc, ps[v], acc[v][r]);
                    }
                }
            }
        }
        cpx<float> cc[VB][3], o[VB][3];
        RecGroup<VP, VB>::load(rin + (unsigned)i * rstride, cs, t, T, cc);
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
            for (int v = 0; v < VB; ++v)
                if (on[v]) VRec<VP>::store(rout + (unsigned)i * rstride, cs, il_vec<VP, VB>(t, T, v), o[v]);
        }
    }
};

// Bounded wait for phase `parity` of bar: each poll may sleep up to 20 us in
// the instruction (a few polls cover the copy latency), at most
// kIltWaitPolls polls (about 2 s).
constexpr long long kIltWaitPolls = 100000;
__device__ __forceinline__ bool ilt_wait(uint64_t *bar, unsigned parity)
{
    for (long long n = 0; !mbar_try_wait_sleep(bar, parity, 20000u);)
        if (++n > kIltWaitPolls) return false;
    return true;
}

// RB (one vector group per row, vector pairs): the row's own records are
// copied into shared memory with the W rows, and the x neighbours and the
// centre are read from there.
template <int VP, int WF, int VB, bool ACT, int MAXT, int MINB, bool PF = false, bool RB = false>
__global__ void __launch_bounds__(MAXT, MINB) k_step_ilt(const char *__restrict__ W, const char *__restrict__ in,
                                                        char *__restrict__ out, const float *__restrict__ alphaf,
                                                        const int *__restrict__ active, SubGeom g, int nvec, int *err,
                                                        int pfd)
{
    static_assert(!RB || (VB % 2 == 0 && !PF), "row staging: vector pairs, no next-hop prefetch");
    static_assert(VP != P_F64, "packed FP32 pairs only");
    extern __shared__ __align__(128) unsigned char ilt_sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(ilt_sm);
    char *ws = reinterpret_cast<char *>(ilt_sm) + 128;
    const int yq = blockIdx.y;
    const int blk = blockIdx.z / g.hz;
    const int zq = blockIdx.z - blk * g.hz;
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    // Only the leader touches the mbarrier (initialises it, issues the copies
    // and waits), so no CTA barrier is needed before the copies start.
    if (leader) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    constexpr int VBY = vfmt_bytes(VP);
    char *rbuf = ws + 5 * g.hx * wfmt_bytes(WF);
    if (leader) {
        if constexpr (RB) {  // the row's records: its bytes join the phase before the W arrival
            const unsigned rowB = (unsigned)(g.hx * nvec * VBY);
            mbar_expect_tx_only(bar, rowB);
            const char *rb = in + (int64_t)blk * g.Ps * nvec * VBY;
            const int64_t row = (int64_t)zq * g.hy * g.hx + (int64_t)yq * g.hx;
            if constexpr (VP == P_F32) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    bulk_load(rbuf + c * (rowB / 3), rb + ((int64_t)c * g.Ps + row) * nvec * 8, rowB / 3, bar);
            } else {
                bulk_load(rbuf, rb + row * nvec * VBY, rowB, bar);
            }
        }
        ilt_issue_w<WF>(ws, W, g, blk, zq, yq, bar);
        if (pfd > 0 && blockIdx.x == 0) ilt_prefetch_ahead<VP, WF>(W, in, g, nvec, pfd);
    }

    const int k = threadIdx.y;                           // x' of this thread's site
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // vector unit over the whole site
    const int T = nvec / VB;
    IltSite<VP, WF, VB, ACT, PF> st;
    if constexpr (RB) {
        st.rbuf = rbuf;
        st.rcs = g.hx * nvec;
    }
    st.setup(in, out, active, g, nvec, blk, zq, yq, k, t, T);
    // The leader waits for the copies; the other threads wait at the CTA
    // barrier without spending issue slots.  The CTA must not retire while its
    // copies are in flight: on a timeout the leader waits once more (bounded).
    __shared__ int w_ok;
    if (leader) {
        const bool okw = ilt_wait(bar, 0u);
        w_ok = okw;
        if (!okw) {
            atomicOr(err, DERR_TIMEOUT);
            ilt_wait(bar, 0u);
        }
    }
    __syncthreads();
    if (!w_ok) return;
    if (st.any) st.compute(ws, g.hx, k, t, T, alphaf);
}

// Vectors per CTA: tile[0] if it is a multiple of VB dividing nvec, else the
// largest such count with (count / VB) * hx <= 256 threads.  0: no fit.
inline int ilt_group(int nvec, int vb, int hx, int want)
{
    auto fits = [&](int n) { return n >= vb && n % vb == 0 && nvec % n == 0 && (n / vb) * hx <= 256; };
    if (want > 0 && fits(want)) return want;
    for (int n = nvec; n >= vb; n -= vb)
        if (fits(n)) return n;
    return 0;
}

// tile[1] = 6: registers capped for 3 CTAs of 256 threads per SM; 7: the next
// hop's records prefetched, registers for 3 CTAs of 192 threads (2 of 256
// when the row needs more threads); 8: the row's own records staged with the
// W rows.  tile[2] > 0: each CTA requests into L2 the row data of the CTA
// tile[2] planes ahead; < 0: the distance that keeps about 12 MB ahead.
template <int VP, int WF, int VB> cudaError_t ilt_launch(const StepArgs &a)
{
    if constexpr (VP == P_F64 || (VB > 4 && !(VP == P_F32 && VB == 8))) {
        return cudaErrorNotSupported;
    } else {
        if (!a.err || !a.alphaf || !ilt_ok(WF, a.g)) return cudaErrorNotSupported;
        const int nvg = ilt_group(a.nvec, VB, a.g.hx, a.tile[0]);
        if (nvg == 0) return cudaErrorNotSupported;
        dim3 block(nvg / VB, a.g.hx);
        dim3 grid(a.nvec / nvg, a.g.hy, (unsigned)a.g.hz * a.nblk);
        if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
        const int smem = ilt_smem(a.g.hx, wfmt_bytes(WF));
        if (smem > (48 << 10)) return cudaErrorNotSupported;
        const bool act = a.active != nullptr;
        const int threads = block.x * block.y;
        // L2 prefetch distance in planes: tile[2] > 0 as given, 0 none, < 0
        // about 12 MB of row data ahead of the CTA that requests it
        int pfd = a.tile[2] > 0 ? a.tile[2] : 0;
        if (a.tile[2] < 0) {
            const int64_t plane =
                (int64_t)a.g.hy * a.g.hx * ((int64_t)a.nvec * vfmt_bytes(VP) + 3 * wfmt_bytes(WF));
            pfd = (int)std::max<int64_t>(1, std::min<int64_t>(1 << 16, (int64_t(12) << 20) / plane));
        }
        if constexpr (VB % 2 == 0) {
            // tile[1] = 8: the row's own records staged with the W rows (one vector group per row)
            const int smem_rb = smem + a.g.hx * a.nvec * vfmt_bytes(VP);
            if (a.tile[1] == 8 && nvg == a.nvec && smem_rb <= (48 << 10)) {
                if (act)
                    k_step_ilt<VP, WF, VB, true, 256, 3, false, true><<<grid, block, smem_rb, a.stream>>>(
                        a.W, a.in, a.out, a.alphaf, a.active, a.g, a.nvec, a.err, pfd);
                else
                    k_step_ilt<VP, WF, VB, false, 256, 3, false, true><<<grid, block, smem_rb, a.stream>>>(
                        a.W, a.in, a.out, a.alphaf, nullptr, a.g, a.nvec, a.err, pfd);
                return cudaGetLastError();
            }
        }
        if (a.tile[1] == 7 && threads <= 192) {  // registers for 3 CTAs of 192 threads per SM
            if (act)
                k_step_ilt<VP, WF, VB, true, 192, 3, true><<<grid, block, smem, a.stream>>>(
                    a.W, a.in, a.out, a.alphaf, a.active, a.g, a.nvec, a.err, pfd);
            else
                k_step_ilt<VP, WF, VB, false, 192, 3, true><<<grid, block, smem, a.stream>>>(
                    a.W, a.in, a.out, a.alphaf, nullptr, a.g, a.nvec, a.err, pfd);
        } else if (a.tile[1] == 7) {  // registers for 2 CTAs of 256 threads per SM
            if (act)
                k_step_ilt<VP, WF, VB, true, 256, 2, true><<<grid, block, smem, a.stream>>>(
                    a.W, a.in, a.out, a.alphaf, a.active, a.g, a.nvec, a.err, pfd);
            else
                k_step_ilt<VP, WF, VB, false, 256, 2, true><<<grid, block, smem, a.stream>>>(
                    a.W, a.in, a.out, a.alphaf, nullptr, a.g, a.nvec, a.err, pfd);
        } else {  // registers for 3 CTAs of 256 threads per SM
            if (act)
                k_step_ilt<VP, WF, VB, true, 256, 3><<<grid, block, smem, a.stream>>>(
                    a.W, a.in, a.out, a.alphaf, a.active, a.g, a.nvec, a.err, pfd);
            else
                k_step_ilt<VP, WF, VB, false, 256, 3><<<grid, block, smem, a.stream>>>(
                    a.W, a.in, a.out, a.alphaf, nullptr, a.g, a.nvec, a.err, pfd);
        }
        return cudaGetLastError();
    }
}

}  // namespace tls
