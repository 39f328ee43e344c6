// Fast FP32 fit module: compiled with FMA contraction, approximate division and
// square root, flush-to-zero.
#define TPCFIT_DET 0
#define TPCFIT_NS fast
#include "fit_core.cuh"
#include "fit_lanes.cuh"
#include "adjoint_core.cuh"
#include "smooth_core.cuh"

namespace tpcfit {
cudaError_t launch_fit_fast(const FitArgs& a, int lanes_per_track, int rows_per_stage, int warps, cudaStream_t s) {
  // several lanes per track: uniform field without material layers only
  if (lanes_per_track != 1 && !a.mat && !a.field) return fast::launch_lanes(a, lanes_per_track, s);
  return fast::launch(a, 1, rows_per_stage, warps, s);
}
cudaError_t launch_backward_fast(const BwdArgs& a, int warps, cudaStream_t s) {
  return fast::launch_backward(a, warps, s);
}
cudaError_t backward_store_fast(int warps, int phys, int form, int64_t& float4s) {
  return fast::backward_store(warps, phys, form, float4s);
}
int64_t backward_tape_float4s(int64_t n_tracks) { return fast::tape_float4s(n_tracks); }
cudaError_t launch_smooth_fast(const SmoothArgs& a, cudaStream_t s) { return fast::launch_smooth(a, s); }
cudaError_t smooth_store_fast(int64_t& float4s) { return fast::smooth_store(float4s); }
}  // namespace tpcfit
