// fp64 instantiation of the solver (generic kernels).
#include "fw_solve_impl.cuh"

namespace fwh {
cudaError_t launch_solve_f64(double* D, int32_t* P, int64_t n, int64_t ld, const SolveWs& ws,
                             const LaunchCfg& cfg, cudaStream_t s) {
  return fwk::launch_any<double>(D, P, n, ld, ws, cfg, s);
}
}  // namespace fwh
