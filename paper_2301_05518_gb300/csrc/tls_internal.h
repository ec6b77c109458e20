// tls_internal.h -- host-side launch interface between the C ABI and the kernels.
#pragma once

#include <algorithm>

#include <cuda_runtime.h>
#include <stdint.h>

#include "tls_types.h"

namespace tls {

// One smearing-step launch over nblk (slice, sublattice) blocks and nvec vectors.
struct StepArgs {
    const char *W;         // W of the first selected block
    const char *in;        // packed vectors: vector v at in + v * vstride_in
    char *out;
    const double *alpha;   // device, per vector: width / (4 N)
    const float *alphaf;   // device (nullable): alpha rounded to FP32, for the FP32-arithmetic kernels
    const int *active;     // device, per vector (nullable): 0 = leave this vector alone
    SubGeom g;
    int nblk;
    int nvec;
    int64_t vstride_in;    // bytes between vectors
    int64_t vstride_out;
    int wfmt;
    int prec_in;           // vector storage of `in`
    int prec_out;          // vector storage of `out`
    int vb;                // vectors per thread
    int threads;           // threads per CTA (multiple of 32)
    int tile[3];           // interleaved kernel: sites per CTA along x', y', z' (0 = a strip along x')
    int *err;              // device error word (kernels with bounded waits); nullable for the others
    cudaStream_t stream;
};

// Persistent multi-step launch: all N steps, group by group.
struct PersistArgs {
    const char *W;
    const char *in;        // storage prec (read at step 0)
    char *out;             // storage prec (written at step N-1)
    char *scr[2];          // scratch ping-pong, scratch prec, sized for one group
    const double *alpha;
    SubGeom g;
    int nblk, nvec, N;
    int group_blocks;      // blocks per group
    int64_t vstride;       // bytes between vectors of in/out
    int64_t sstride;       // bytes between vectors of scratch
    int wfmt, prec, sprec, vb, threads;
    unsigned *bar;         // 2 words: arrival count, generation (zeroed)
    int *err;              // device error word
    long long budget;      // polls per barrier
    int grid;              // CTAs (co-resident)
    int onchip;            // 1: one CTA per (block, vector group) keeps W and the iterates in shared memory
    int nvg;               // on-chip form: vectors per CTA
    int smem;              // on-chip form: dynamic shared memory bytes
    cudaStream_t stream;
};

// On-chip persistent form: whether one (slice, sublattice) block's W and two
// scratch copies of nvg vectors fit in max_smem bytes; fills nvg (<= nvec)
// and the shared-memory bytes.  Host-only arithmetic.
inline bool onchip_plan(const SubGeom &g, int wfmt_bytes_, int scratch_bytes, int nvec, int max_smem, int *nvg,
                        int *smem)
{
    const int64_t Pss = (g.Vs + 3) / 4 * 4;
    const int64_t wbytes = 3 * Pss * wfmt_bytes_;
    const int64_t per_vec = 2 * Pss * scratch_bytes;
    if (wbytes + per_vec > max_smem) return false;
    const int64_t n = std::min<int64_t>(nvec, (max_smem - wbytes) / per_vec);
    *nvg = (int)n;
    *smem = (int)(wbytes + n * per_vec);
    return true;
}

// Returns cudaErrorNotSupported for combinations without a kernel.
cudaError_t launch_step(const StepArgs &a);
// Interleaved-layout multi-RHS step (nvec <= 256 vectors per record group).
cudaError_t launch_step_il(const StepArgs &a);
// The same step marching along z' with a register window (interleaved layout, active unused).
cudaError_t launch_step_zm(const StepArgs &a);
// One-link Gaussian smearing step psi + alpha H psi (interleaved layout; W = the link field).
cudaError_t launch_hop(const StepArgs &a);
// The same step with TMA row staging in shared memory (k_rows.cuh); err gets
// DERR_TIMEOUT if a bounded wait runs out.  rows_applicable says whether the
// shape and formats allow it (16-byte bulk copies, CTA size, shared memory).
cudaError_t launch_step_rows(const StepArgs &a, int *err);
bool rows_applicable(int wfmt, int prec, const SubGeom &g, int nvec, int vb, int max_smem);
cudaError_t launch_persistent(const PersistArgs &a);
// Co-resident CTAs per SM of the persistent kernel for this combination (0: none).
int persistent_occupancy(int wfmt, int prec, int sprec, int vb, int threads);

// Per-precision entry points (one translation unit each).
cudaError_t launch_step_f64(const StepArgs &a);
cudaError_t launch_step_f32(const StepArgs &a);
cudaError_t launch_step_f16(const StepArgs &a);
cudaError_t launch_step_bf16(const StepArgs &a);
cudaError_t launch_step_il_f64(const StepArgs &a);
cudaError_t launch_step_il_f32(const StepArgs &a);
cudaError_t launch_step_il_f16(const StepArgs &a);
cudaError_t launch_step_il_bf16(const StepArgs &a);
cudaError_t launch_step_zm_f64(const StepArgs &a);
cudaError_t launch_hop_f64(const StepArgs &a);
cudaError_t launch_hop_f32(const StepArgs &a);
cudaError_t launch_hop_f16(const StepArgs &a);
cudaError_t launch_hop_bf16(const StepArgs &a);
cudaError_t launch_step_zm_f32(const StepArgs &a);
cudaError_t launch_step_zm_f16(const StepArgs &a);
cudaError_t launch_step_zm_bf16(const StepArgs &a);
cudaError_t launch_step_rows_f64(const StepArgs &a, int *err);
cudaError_t launch_step_rows_f32(const StepArgs &a, int *err);
cudaError_t launch_step_rows_f16(const StepArgs &a, int *err);
cudaError_t launch_step_rows_bf16(const StepArgs &a, int *err);
cudaError_t launch_persistent_f64(const PersistArgs &a);
cudaError_t launch_persistent_f32(const PersistArgs &a);
cudaError_t launch_persistent_f16(const PersistArgs &a);
cudaError_t launch_persistent_bf16(const PersistArgs &a);
int persistent_occupancy_f64(int wfmt, int vb, int threads);
int persistent_occupancy_f32(int wfmt, int vb, int threads);
int persistent_occupancy_f16(int wfmt, int vb, int threads);
int persistent_occupancy_bf16(int wfmt, int vb, int threads);

// Layout kernels (k_layout.cu).
cudaError_t launch_ingest_gauge(const double *U, int nd, double *Up, const SubGeom &g, const int L[4],
                                cudaStream_t s);
cudaError_t launch_export_gauge(const double *Up, double *out, const SubGeom &g, const int L[4], cudaStream_t s);
cudaError_t launch_build_twolink(const double *Up, char *W, int wfmt, const SubGeom &g, int nblk, int *err,
                                 cudaStream_t s);
// The one-link field: U itself rounded into a W format (same planes as W).
cudaError_t launch_build_links(const double *Up, char *L1, int wfmt, const SubGeom &g, int nblk, cudaStream_t s);
// One APE step on the packed spatial links: out = P((1-a) U + (a/4) staples) (k_ape.cu).
cudaError_t launch_ape_step(const double *U, double *out, const SubGeom &g, int nblk, double a, int *err,
                            cudaStream_t s);
cudaError_t launch_export_twolink(const char *W, int wfmt, double *out, const SubGeom &g, const int L[4],
                                  cudaStream_t s);
// Whether the interleaved pack/unpack use the row transposes (contiguous canonical rows).
bool rows_transpose_ok(const SubGeom &g, int rec_n, int prec, const int L[4]);
// Interleaved layout: rec_n <= 256 records per site, record (block, i, r).  Caller vector v
// (0 <= v < nvec) goes to / comes from record rec_v0 + v.
cudaError_t launch_pack_il(const void *src, int io_prec, int64_t src_vstride_sites, char *dst, int prec,
                           const SubGeom &g, const int L[4], int t_first, int nsl, int nvec, int rec_n, int rec_v0,
                           cudaStream_t s);
cudaError_t launch_unpack_il(const char *src, int prec, void *dst, int io_prec, int64_t dst_vstride_sites,
                             const SubGeom &g, const int L[4], int t_first, int nsl, int nvec, int rec_n, int rec_v0,
                             cudaStream_t s);
// FP64 |psi|^2 partial sums of nvec canonical vectors (vector v at base + v * vstride
// sites), kNormPartsPerSlice per (vector, slice) over nsl slices of slice_sites sites:
// partial (v, s, p) at partials[v * part_stride + part_off + s * kNormPartsPerSlice + p].
// A partial depends only on its slice, so slices may be summed in separate launches;
// launch_reduce_norms(partials, part_stride, ...) then adds each vector's partials in order.
const int kNormPartsPerSlice = 16;
cudaError_t launch_norm_partials(const void *base, int io_prec, int64_t vstride_sites, int64_t slice_sites, int nsl,
                                 int nvec, double *partials, int64_t part_stride, int64_t part_off, cudaStream_t s);
// Canonical caller vectors (io_prec F64/F32, slices [t_first, t_first + nsl)) -> packed storage.
cudaError_t launch_pack_vectors(const void *src, int io_prec, int64_t src_vstride_sites, char *dst, int prec,
                                int64_t dst_vstride, const SubGeom &g, const int L[4], int t_first, int nsl,
                                int nvec, cudaStream_t s);
// Packed storage -> canonical; partials (nullable) gets one FP64 sum of |psi|^2 per (vector, CTA).
cudaError_t launch_unpack_vectors(const char *src, int prec, int64_t src_vstride, void *dst, int io_prec,
                                  int64_t dst_vstride_sites, const SubGeom &g, const int L[4], int t_first,
                                  int nsl, int nvec, double *partials, int *nparts, cudaStream_t s);
cudaError_t launch_reduce_norms(const double *partials, int nparts, int nvec, double *norms, cudaStream_t s);
int unpack_parts(const SubGeom &g, int nsl);

}  // namespace tls
