// Deterministic fit module: compiled as its own unit with -fmad=false
// -prec-div=true -prec-sqrt=true -ftz=false (the compile-time part of the
// deterministic mode, Sec. 2), so that its operation sequence equals the
// strict-FP32 host reference bit for bit.
#define TPCFIT_DET 1
#define TPCFIT_NS det
#include "fit_core.cuh"
#include "fit_lanes.cuh"
#include "adjoint_core.cuh"
#include "smooth_core.cuh"

namespace tpcfit {
cudaError_t launch_fit_det(const FitArgs& a, int lanes_per_track, int rows_per_stage, int warps, cudaStream_t s) {
  // several lanes per track: uniform field without material layers only
  if (lanes_per_track != 1 && !a.mat && !a.field) return det::launch_lanes(a, lanes_per_track, s);
  return det::launch(a, 1, rows_per_stage, warps, s);
}
cudaError_t launch_backward_det(const BwdArgs& a, int warps, cudaStream_t s) {
  return det::launch_backward(a, warps, s);
}
cudaError_t launch_smooth_det(const SmoothArgs& a, cudaStream_t s) { return det::launch_smooth(a, s); }
cudaError_t smooth_store_det(int64_t& float4s) { return det::smooth_store(float4s); }
}  // namespace tpcfit
