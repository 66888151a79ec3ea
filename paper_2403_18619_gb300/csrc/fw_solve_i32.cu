// int32 instantiation of the solver (packed-key DPX kernels + generic fallback).
#include "fw_solve_impl.cuh"

namespace fwh {
cudaError_t launch_solve_i32(int32_t* D, int32_t* P, int64_t n, int64_t ld, const SolveWs& ws,
                             const LaunchCfg& cfg, cudaStream_t s) {
  return fwk::launch_any<int32_t>(D, P, n, ld, ws, cfg, s);
}
}  // namespace fwh
