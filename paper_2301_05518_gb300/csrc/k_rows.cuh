// k_rows.cuh -- multi-RHS smearing step with TMA row staging (sm_100+ bulk copies).
//
// Same step as k_step_il (Sec. 2, Eq. tlSmear with Eq. tlLapl1) on the
// interleaved layout, organised around contiguous rows:
//  * a CTA owns one z'-plane of one (slice, sublattice) block and sweeps its
//    hy rows of hx sites in order;
//  * a row of the interleaved field (hx sites x nvec records) is one
//    contiguous segment, fetched into shared memory by one cp.async.bulk; a W
//    row of one direction is 4-5 plane segments;
//  * for row y the CTA needs psi rows y-1, y, y+1 of its plane (a ring of 4
//    slots, the next row prefetched), rows y of planes z'-1 and z'+1, the W rows
//    of row y (3 directions), W_y of row y-1 (ring of 3) and W_z of row y in
//    plane z'-1;
//  * stage y+1 is issued by one warp before row y is computed, so the copies of
//    the next row overlap the arithmetic of this one; completion is tracked by
//    two mbarriers (transaction bytes), one per stage parity.
// The per-vector FMA sequence is that of site_step, so results are bitwise
// equal to the other kernels.
//
// Waits are bounded: a wait that runs out sets DERR_TIMEOUT, waits once more
// (bounded) for this CTA's copies in flight and returns.
#pragma once

#include "tls_dev.cuh"
#include "tls_internal.h"
#include "tma.cuh"

namespace tls {

// Geometry of one CTA's staging buffers (bytes, all 128-aligned).
struct RowsPlan {
    int rowB;   // one psi row: hx * nvec * record bytes
    int wrowB;  // one W row of one direction: hx * W bytes
    int offY, offZ, offW, offWz, total;
};

inline RowsPlan rows_plan(int hx, int nvec, int vby, int wb)
{
    auto up = [](int n) { return (n + 127) / 128 * 128; };
    RowsPlan p{};
    p.rowB = hx * nvec * vby;
    p.wrowB = hx * wb;
    p.offY = 128;                             // 4 mbarriers at 0 (full[2], empty[2])
    p.offZ = p.offY + 4 * up(p.rowB);         // Y ring of 4
    p.offW = p.offZ + 4 * up(p.rowB);         // Z [parity][minus, plus]
    p.offWz = p.offW + 9 * up(p.wrowB);       // Wc [ring 3][dir 3]
    p.total = p.offWz + 2 * up(p.wrowB);      // Wz [parity]
    return p;
}

template <int WF> struct WPlanes {
    static constexpr int WB = wfmt_bytes(WF);
    static constexpr int NQ = WB / 16;
    static constexpr int REM = WB % 16;
};

// Shared memory allows one or two CTAs per SM, so the launch bound scales
// with VB and leaves the compiler registers to hoist the next loads.
template <int VB> struct RowsBound {
    static constexpr int threads = VB == 1 ? 768 : VB == 2 ? 384 : 256;
};

template <int VP, int WF, int VB>
__global__ void __launch_bounds__(RowsBound<VB>::threads) k_step_rows(const char *__restrict__ W, const char *__restrict__ in,
                                                   char *__restrict__ out, const double *__restrict__ alpha,
                                                   SubGeom g, int nvec, RowsPlan pl, int *err)
{
    typedef typename VRec<VP>::R R;
    constexpr int WB = wfmt_bytes(WF);
    constexpr int VBY = vfmt_bytes(VP);
    constexpr int NQ = WPlanes<WF>::NQ, REM = WPlanes<WF>::REM;
    extern __shared__ __align__(128) unsigned char rows_sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(rows_sm);
    auto up = [](int n) { return (n + 127) / 128 * 128; };
    const int rowS = up(pl.rowB), wS = up(pl.wrowB);
    char *Y = reinterpret_cast<char *>(rows_sm) + pl.offY;
    char *Z = reinterpret_cast<char *>(rows_sm) + pl.offZ;
    char *Wc = reinterpret_cast<char *>(rows_sm) + pl.offW;
    char *Wz = reinterpret_cast<char *>(rows_sm) + pl.offWz;

    // A bounded wait already ran out somewhere: do nothing (no copy issued yet).
    {
        int e0;
        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(e0) : "l"(err) : "memory");
        if (e0 & DERR_TIMEOUT) return;
    }
    const int hx = g.hx, hy = g.hy, hz = g.hz;
    const int zq = blockIdx.x;
    const int blk = blockIdx.y;
    const int zm = zq == 0 ? hz - 1 : zq - 1;
    const int zp = zq == hz - 1 ? 0 : zq + 1;
    const char *wblk = W + (int64_t)blk * 3 * g.Ps * WB;
    const int64_t recB = (int64_t)nvec * VBY;  // bytes of one site's records
    const char *inblk = in + (int64_t)blk * g.Ps * recB;
    char *outblk = out + (int64_t)blk * g.Ps * recB;
    // interleaved layout: site stride nvec * SB; F32 / F64 colour planes cs apart
    constexpr int SB = VRec<VP>::SB;
    constexpr bool PL = il_planes(VP);
    const int64_t sst = (int64_t)nvec * SB;
    const int cs_g = g.Ps * nvec, cs_s = hx * nvec;  // colour stride in global memory / in a staged row

    const int tx = nvec / VB;
    const int tid = threadIdx.x;
    const int xq = tid / tx;
    const int vg = tid - xq * tx;
    const int t = vg, T = tx;  // this thread's vectors: il_vec(t, T, k)
    const bool worker = xq < hx;
    R a_v[VB];  // alpha per vector, converted once (keeps FP64 out of the row loop)
#pragma unroll
    for (int k = 0; k < VB; ++k) a_v[k] = worker ? (R)alpha[il_vec<VP, VB>(t, T, k)] : R(0);

    auto row_of = [&](int z, int y) { return (z * hy + y) * hx; };
    auto ring4 = [](int r) { return (r + 4) & 3; };
    auto ring3 = [](int r) { return (r + 3) % 3; };
    auto wrap_y = [&](int r) { return r < 0 ? r + hy : (r >= hy ? r - hy : r); };

    // W row (direction d, global row r0) into smem slot.
    auto load_wrow = [&](char *dst, int d, int r0, uint64_t *bar) {
        const char *base = wblk + (int64_t)d * g.Ps * WB;
#pragma unroll
        for (int j = 0; j < NQ; ++j) bulk_load(dst + j * hx * 16, base + ((int64_t)j * g.Ps + r0) * 16, hx * 16, bar);
        if (REM) bulk_load(dst + NQ * hx * 16, base + (int64_t)NQ * g.Ps * 16 + (int64_t)r0 * REM, hx * REM, bar);
    };
    const unsigned wrow_bytes = (unsigned)(hx * WB);
    const unsigned row_bytes = (unsigned)pl.rowB;
    // psi row starting at site r0 into a row slot: one segment per colour plane
    auto load_prow = [&](char *dst, int r0, uint64_t *bar) {
        if constexpr (PL) {
            const unsigned segB = (unsigned)(hx * nvec * SB);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                bulk_load(dst + c * segB, inblk + ((int64_t)c * g.Ps + r0) * sst, segB, bar);
        } else {
            bulk_load(dst, inblk + (int64_t)r0 * sst, row_bytes, bar);
        }
    };

    // Stage r (r >= 0): psi row r+1 of this plane, rows r of planes z-1, z+1,
    // W rows r (3 dirs), W_z row r of plane z-1.
    auto issue_stage = [&](int r) {
        uint64_t *bar = &bars[r & 1];
        const int y = r, yn = wrap_y(r + 1);
        mbar_expect_tx(bar, 3 * row_bytes + 4 * wrow_bytes);
        load_prow(Y + ring4(r + 1) * rowS, row_of(zq, yn), bar);
        load_prow(Z + ((r & 1) * 2 + 0) * rowS, row_of(zm, y), bar);
        load_prow(Z + ((r & 1) * 2 + 1) * rowS, row_of(zp, y), bar);
#pragma unroll
        for (int d = 0; d < 3; ++d) load_wrow(Wc + (ring3(r) * 3 + d) * wS, d, row_of(zq, y), bar);
        load_wrow(Wz + (r & 1) * wS, 2, row_of(zm, y), bar);
    };

    // full[b]: the stage of parity b has landed (1 arrival + transaction bytes).
    // empty[b]: every warp has finished the row of parity b (one arrival per warp).
    uint64_t *full = bars, *empty = bars + 2;
    const int nwarps = (blockDim.x + 31) / 32;
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], nwarps);
        mbar_init(&empty[1], nwarps);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Prologue on full[1] (its first phase): psi rows -1 and 0, W rows -1.
    // Then stage 0 on full[0].
    unsigned fph0 = 0u, fph1 = 0u;
    if (tid == 0) {
        uint64_t *bar = &full[1];
        mbar_expect_tx(bar, 2 * row_bytes + 3 * wrow_bytes);
        load_prow(Y + ring4(-1) * rowS, row_of(zq, hy - 1), bar);
        load_prow(Y + ring4(0) * rowS, row_of(zq, 0), bar);
#pragma unroll
        for (int d = 0; d < 3; ++d) load_wrow(Wc + (ring3(-1) * 3 + d) * wS, d, row_of(zq, hy - 1), bar);
        issue_stage(0);
    }
    const long long kLimit = 1LL << 22;
    auto wait_on = [&](uint64_t *bar, unsigned parity) -> bool {
        long long n = 0;
        while (!mbar_try_wait(bar, parity)) {
            if (++n > kLimit) return false;
        }
        return true;
    };
    auto wait_full = [&](int b) -> bool {
        unsigned &ph = b ? fph1 : fph0;
        if (!wait_on(&full[b], ph)) return false;
        ph ^= 1u;
        return true;
    };
    bool ok = wait_full(1);

    for (int y = 0; y < hy && ok; ++y) {
        // Stage y+1 refills the slots row y-1 read: the producer waits until
        // every warp has released row y-1, the other warps run on.
        if (tid == 0 && y + 1 < hy) {
            if (y >= 1) ok = wait_on(&empty[(y - 1) & 1], ((y - 1) >> 1) & 1);
            if (ok) {
                fence_proxy_async_smem();
                issue_stage(y + 1);
            }
        }
        if (ok) ok = wait_full(y & 1);
        if (!ok) break;
        if (worker) {
            const int xp = xq == hx - 1 ? 0 : xq + 1;
            const int xm = xq == 0 ? hx - 1 : xq - 1;
            const char *Yc = Y + ring4(y) * rowS, *Ym = Y + ring4(y - 1) * rowS, *Yp = Y + ring4(y + 1) * rowS;
            const char *Zm = Z + ((y & 1) * 2 + 0) * rowS, *Zp = Z + ((y & 1) * 2 + 1) * rowS;
            const char *Wrow = Wc + ring3(y) * 3 * wS;
            const char *Wym = Wc + (ring3(y - 1) * 3 + 1) * wS;
            const char *Wzm = Wz + (y & 1) * wS;
            const unsigned rs = (unsigned)sst;
            // Operand addresses of the six hops, in the order of site_step:
            // x forward, x backward, y forward, y backward, z forward, z backward.
            const char *wsrc[6] = {Wrow, Wrow, Wrow + wS, Wym, Wrow + 2 * wS, Wzm};
            const int wsite[6] = {xq, xm, xq, xq, xq, xq};
            const char *psrc[6] = {Yc + xp * rs, Yc + xm * rs, Yp + xq * rs,
                                   Ym + xq * rs, Zp + xq * rs, Zm + xq * rs};
            cpx<R> acc[VB][3];
#pragma unroll
            for (int k = 0; k < VB; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[k][c].re = acc[k][c].im = R(0);
            // software pipeline: the operands of hop h+1 are loaded before hop h is applied
            cpx<R> m[2][9], p[2][VB][3];
            WFmt<WF>::load(wsrc[0], hx, wsite[0], m[0]);
            RecGroup<VP, VB, false>::load(psrc[0], cs_s, t, T, p[0]);
#pragma unroll
            for (int h = 0; h < 6; ++h) {
                if (h + 1 < 6) {
                    WFmt<WF>::load(wsrc[h + 1], hx, wsite[h + 1], m[(h + 1) & 1]);
                    RecGroup<VP, VB, false>::load(psrc[h + 1], cs_s, t, T, p[(h + 1) & 1]);
                }
#pragma unroll
                for (int k = 0; k < VB; ++k) {
                    if (h & 1)
                        mdv_add(m[h & 1], p[h & 1][k], acc[k]);
                    else
                        mv_add(m[h & 1], p[h & 1][k], acc[k]);
                }
            }
            cpx<R> c[VB][3], o[VB][3];
            RecGroup<VP, VB, false>::load(Yc + xq * rs, cs_s, t, T, c);
#pragma unroll
            for (int k = 0; k < VB; ++k) {
                const R a = a_v[k];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    o[k][q].re = fma(a, fma(R(-6), c[k][q].re, acc[k][q].re), c[k][q].re);
                    o[k][q].im = fma(a, fma(R(-6), c[k][q].im, acc[k][q].im), c[k][q].im);
                }
            }
            RecGroup<VP, VB>::store(outblk + ((int64_t)row_of(zq, y) + xq) * sst, cs_g, t, T, o);
                }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[y & 1]);
    }
    if (!ok) {
        atomicOr(err, DERR_TIMEOUT);
        // let this CTA's own copies land before shared memory goes away
        long long n = 0;
        while (!mbar_try_wait(&full[0], fph0) && ++n < kLimit) {
        }
        n = 0;
        while (!mbar_try_wait(&full[1], fph1) && ++n < kLimit) {
        }
    }
}

// Host side: whether the row kernel applies, and its launch.
inline bool rows_ok(int wfmt, int prec, const SubGeom &g, int nvec, int vb, int max_smem)
{
    const int wb = wfmt_bytes(wfmt), vby = vfmt_bytes(prec);
    if (g.hx % 4 != 0) return false;  // 16-byte bulk copies of every plane segment
    if (vb < 1 || nvec % vb != 0) return false;
    const int threads = g.hx * (nvec / vb);
    const int bound = vb == 1 ? 768 : vb == 2 ? 384 : 256;
    if (threads > bound || threads < 32) return false;
    if ((g.hx * nvec * vby) % 16 != 0) return false;
    (void)wb;
    RowsPlan p = rows_plan(g.hx, nvec, vby, wb);
    return p.total <= max_smem;
}

template <int VP, int WF, int VB> cudaError_t rows_launch(const StepArgs &a, int *err)
{
    const RowsPlan pl = rows_plan(a.g.hx, a.nvec, vfmt_bytes(VP), wfmt_bytes(WF));
    // per launch: the attribute belongs to the current device
    cudaError_t e = cudaFuncSetAttribute(k_step_rows<VP, WF, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         pl.total);
    if (e != cudaSuccess) return e;
    const int threads = (a.g.hx * (a.nvec / VB) + 31) / 32 * 32;
    dim3 grid(a.g.hz, a.nblk);
    k_step_rows<VP, WF, VB><<<grid, threads, pl.total, a.stream>>>(a.W, a.in, a.out, a.alpha, a.g, a.nvec, pl,
                                                                       err);
    return cudaGetLastError();
}

template <int VP, int WF> cudaError_t rows_w(const StepArgs &a, int *err)
{
    if constexpr (!combo_ok<VP, WF>() || VP == P_F64) {
        return cudaErrorNotSupported;
    } else {
        int vb = a.vb > 0 ? a.vb : 1;
        if (a.nvec % vb != 0) vb = 1;
        if constexpr (VP == P_F32) {
            switch (vb) {
            case 2: return rows_launch<VP, WF, 2>(a, err);
            case 4: return rows_launch<VP, WF, 4>(a, err);
            default: return rows_launch<VP, WF, 1>(a, err);
            }
        } else {
            switch (vb) {
            case 2: return rows_launch<VP, WF, 2>(a, err);
            case 4: return rows_launch<VP, WF, 4>(a, err);
            default: return rows_launch<VP, WF, 1>(a, err);
            }
        }
    }
}

template <int VP> cudaError_t rows_dispatch(const StepArgs &a, int *err)
{
    const int wf = a.wfmt;
    TLS_WFMT_SWITCH(rows_w, VP, (a, err), cudaErrorNotSupported)
}

}  // namespace tls
