// Solver kernels (phased and persistent drivers) and their host launcher,
// templated on the element type; instantiated in fw_solve_i32.cu / _f32.cu.
#pragma once

#include "fw_device.cuh"
#include "fw_internal.h"
#include "fw_ws.cuh"

namespace fwk {

// -------------------------------------------------------- phased driver ----

template <typename T, int BS>
__global__ void __launch_bounds__(kThreads, 1) k_phase_pivot(Args<T> a, int r) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ CtaScratch cs;
  task_pivot<T, BS>(a, r, smem, &cs);
}

template <typename T, int BS>
__global__ void __launch_bounds__(kThreads, 1) k_phase_panel(Args<T> a, int r) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ CtaScratch cs;
  const fwh::Task k = fwh::task_panel(a.R, r, blockIdx.x);
  task_panel<T, BS>(a, r, k.type == 1 ? k.tj : k.ti, k.type == 1, smem, &cs);
}

template <typename T, int BS>
__global__ void __launch_bounds__(kThreads, 1) k_phase_rest(Args<T> a, int r) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ CtaScratch cs;
  if (threadIdx.x == 0) {
    mbar_init(&cs.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int w = a.R - 1;
  int i = blockIdx.x / w, j = blockIdx.x % w;
  i = i < r ? i : i + 1;
  j = j < r ? j : j + 1;
  unsigned phase = 0;
  task_minplus<T, BS>(a, r, i, j, smem, &cs, phase);
}

// ---------------------------------------------------------------- host ----

// Tensor-map element type of T.
template <typename T> struct TmapType;
template <> struct TmapType<int32_t> { static constexpr CUtensorMapDataType kType = CU_TENSOR_MAP_DATA_TYPE_INT32; };
template <> struct TmapType<float> { static constexpr CUtensorMapDataType kType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };
template <> struct TmapType<int64_t> { static constexpr CUtensorMapDataType kType = CU_TENSOR_MAP_DATA_TYPE_INT64; };
template <> struct TmapType<double> { static constexpr CUtensorMapDataType kType = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; };

template <typename T, int BS>
cudaError_t launch_bs(T* D, int32_t* P, int64_t n, int64_t ld, const fwh::SolveWs& ws,
                      const fwh::LaunchCfg& cfg, cudaStream_t s) {
  Args<T> a{};
  a.D = D; a.P = P; a.n = n; a.ld = ld; a.R = ws.R; a.slot_tiles = ws.slot_tiles;
  a.ver = ws.ver; a.done = ws.done; a.ctr = ws.ctr; a.abort_flag = ws.abort_flag; a.status = ws.status;
  a.stage_off = ws.stage_off; a.lookahead = (int)cfg.lookahead; a.skip_task = cfg.skip_task;
  a.timeout_ns = cfg.timeout_ns; a.packed = cfg.packed;
  a.piv = reinterpret_cast<T*>(ws.piv); a.pivP = ws.pivP;
  a.colK = ws.colK; a.colR = reinterpret_cast<T*>(ws.colR); a.colB = ws.colB;
  a.rowK = ws.rowK; a.rowR = reinterpret_cast<T*>(ws.rowR); a.rowP = ws.rowP; a.rowB = ws.rowB;
  a.trace = cfg.trace; a.trace_cap = (int)cfg.trace_cap; a.trace_stride = cfg.trace_stride;
  const int R = ws.R;
  const size_t smem = Smem<BS, T>::bytes();
  cudaError_t e;

  if (P) {  // null: distance-only
    int64_t blocks = (n * n + 255) / 256;
    const int cap = fwh::num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_init_pred<T><<<(int)blocks, 256, 0, s>>>(D, P, n, ld);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (cfg.ev_start) cudaEventRecord(cfg.ev_start, s);
  if (cfg.driver == 2) {
    if (fwh::kernel_setup(reinterpret_cast<const void*>(k_phase_pivot<T, BS>), smem, kThreads) < 1 ||
        fwh::kernel_setup(reinterpret_cast<const void*>(k_phase_panel<T, BS>), smem, kThreads) < 1 ||
        fwh::kernel_setup(reinterpret_cast<const void*>(k_phase_rest<T, BS>), smem, kThreads) < 1)
      return cudaErrorInvalidConfiguration;
    for (int r = 0; r < R; ++r) {
      k_phase_pivot<T, BS><<<1, kThreads, smem, s>>>(a, r);
      if (R > 1) {
        k_phase_panel<T, BS><<<2 * (R - 1), kThreads, smem, s>>>(a, r);
        k_phase_rest<T, BS><<<(R - 1) * (R - 1), kThreads, smem, s>>>(a, r);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  } else {
    auto kern = k_persistent_ws<T, BS>;
    const size_t wsmem = WsLayout<BS, T>::bytes();
    const int occ = fwh::kernel_setup(reinterpret_cast<const void*>(kern), wsmem, kWsThreads);
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t grid = cfg.grid > 0 ? cfg.grid : (int64_t)occ * fwh::num_sms();
    if (grid > (int64_t)occ * fwh::num_sms()) grid = (int64_t)occ * fwh::num_sms();
    const int64_t total = (int64_t)R * R * R;
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kWsThreads);
    lc.dynamicSmemBytes = wsmem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    CUtensorMap tmD{}, tmP{};
    int use_tmap = 0;
    if (cfg.tile_tma) {
      if (fwh::encode_tile_map(&tmD, D, n, ld, BS, TmapType<T>::kType, (int)sizeof(T)))
        use_tmap |= 1;
      if (P && fwh::encode_tile_map(&tmP, P, n, ld, BS, CU_TENSOR_MAP_DATA_TYPE_INT32, 4))
        use_tmap |= 2;
    }
    if ((e = cudaLaunchKernelEx(&lc, kern, a, tmD, tmP, use_tmap)) != cudaSuccess) return e;
  }
  if (cfg.ev_stop) cudaEventRecord(cfg.ev_stop, s);
  if (ViaPred<T>::kOn && P) {
    int64_t blocks = (n * n + 255) / 256;
    const int cap = fwh::num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_resolve_pred<<<(int)blocks, 256, 0, s>>>(P, n, ld);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_any(T* D, int32_t* P, int64_t n, int64_t ld, const fwh::SolveWs& ws,
                       const fwh::LaunchCfg& cfg, cudaStream_t s) {
  switch (cfg.BS) {
    case 32: return launch_bs<T, 32>(D, P, n, ld, ws, cfg, s);
    case 64: return launch_bs<T, 64>(D, P, n, ld, ws, cfg, s);
    case 128:
      // three 128 x 128 tiles of 64-bit elements do not fit in shared memory
      if constexpr (sizeof(T) == 4) return launch_bs<T, 128>(D, P, n, ld, ws, cfg, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fwk
