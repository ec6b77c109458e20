// k_step_bf16.cu -- stencil and persistent kernels for bf16 vector storage.
#include "k_stencil.cuh"
#include "k_rows.cuh"
#include "k_hop.cuh"

namespace tls {

cudaError_t launch_step_bf16(const StepArgs &a) { return step_dispatch<P_BF16>(a); }
cudaError_t launch_step_il_bf16(const StepArgs &a) { return step_il_dispatch<P_BF16>(a); }
cudaError_t launch_step_zm_bf16(const StepArgs &a) { return step_zm_dispatch<P_BF16>(a); }
cudaError_t launch_hop_bf16(const StepArgs &a) { return hop_dispatch<P_BF16>(a); }
cudaError_t launch_step_rows_bf16(const StepArgs &a, int *err) { return rows_dispatch<P_BF16>(a, err); }
cudaError_t launch_persistent_bf16(const PersistArgs &a) { return persist_dispatch<P_BF16>(a); }
int persistent_occupancy_bf16(int wfmt, int vb, int threads) { return occ_dispatch<P_BF16>(wfmt, vb, threads); }

}  // namespace tls
