// k_step_f64.cu -- stencil and persistent kernels for f64 vector storage.
#include "k_stencil.cuh"
#include "k_rows.cuh"
#include "k_hop.cuh"

namespace tls {

cudaError_t launch_step_f64(const StepArgs &a) { return step_dispatch<P_F64>(a); }
cudaError_t launch_step_il_f64(const StepArgs &a) { return step_il_dispatch<P_F64>(a); }
cudaError_t launch_step_zm_f64(const StepArgs &a) { return step_zm_dispatch<P_F64>(a); }
cudaError_t launch_hop_f64(const StepArgs &a) { return hop_dispatch<P_F64>(a); }
cudaError_t launch_step_rows_f64(const StepArgs &a, int *err) { return rows_dispatch<P_F64>(a, err); }
cudaError_t launch_persistent_f64(const PersistArgs &a) { return persist_dispatch<P_F64>(a); }
int persistent_occupancy_f64(int wfmt, int vb, int threads) { return occ_dispatch<P_F64>(wfmt, vb, threads); }

}  // namespace tls
