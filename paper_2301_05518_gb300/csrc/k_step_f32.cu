// k_step_f32.cu -- stencil and persistent kernels for f32 vector storage.
#include "k_stencil.cuh"
#include "k_rows.cuh"
#include "k_hop.cuh"

namespace tls {

cudaError_t launch_step_f32(const StepArgs &a) { return step_dispatch<P_F32>(a); }
cudaError_t launch_step_il_f32(const StepArgs &a) { return step_il_dispatch<P_F32>(a); }
cudaError_t launch_step_zm_f32(const StepArgs &a) { return step_zm_dispatch<P_F32>(a); }
cudaError_t launch_hop_f32(const StepArgs &a) { return hop_dispatch<P_F32>(a); }
cudaError_t launch_step_rows_f32(const StepArgs &a, int *err) { return rows_dispatch<P_F32>(a, err); }
cudaError_t launch_persistent_f32(const PersistArgs &a) { return persist_dispatch<P_F32>(a); }
int persistent_occupancy_f32(int wfmt, int vb, int threads) { return occ_dispatch<P_F32>(wfmt, vb, threads); }

bool rows_applicable(int wfmt, int prec, const SubGeom &g, int nvec, int vb, int max_smem)
{
    if (prec == P_F64) return false;
    return rows_ok(wfmt, prec, g, nvec, vb, max_smem);
}

}  // namespace tls
