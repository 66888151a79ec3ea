// Solver kernels (phased and persistent drivers) and their host launcher,
// templated on the element type; instantiated in fw_solve_i32.cu / _f32.cu.
#pragma once

#include "fw_device.cuh"
#include "fw_internal.h"

namespace fwk {

// ----------------------------------------------------- persistent driver ----

// Bounded wait until *p >= target (thread 0 only).  Gives up when another CTA
// has aborted or when the wait exceeds timeout_ns; then records the timeout
// and raises the abort flag so that every other CTA stops too.
__device__ __forceinline__ bool wait_ge(const int* p, int target, int* abort_flag, int* status,
                                        int64_t timeout_ns) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = globaltimer();
  // iteration cap as well as the clock: each iteration sleeps >= 32 ns
  const int64_t max_it = timeout_ns / 32 + 1024;
  unsigned ns = 32;
  for (int64_t it = 0;; ++it) {
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
    if (ld_acquire(p) >= target) return true;
    if (ld_relaxed(abort_flag)) return false;
    if (globaltimer() - t0 > (uint64_t)timeout_ns || it > max_it) {
      atomicOr(status, kStTimeout);
      atomicExch(abort_flag, 1);
      return false;
    }
  }
}

template <typename T>
__device__ bool wait_deps(const Args<T>& a, const fwh::Task& k) {
  const int R = a.R;
  const int* ver = a.ver;
  auto w = [&](const int* p, int target) {
    return wait_ge(p, target, a.abort_flag, a.status, a.timeout_ns);
  };
  const int* done2 = reinterpret_cast<const int*>(a.ctr + 1);
  const int* done3 = reinterpret_cast<const int*>(a.ctr + 2);
  switch (k.type) {
    case 0:  // pivot: its tile after round r-1; pivot slot free (panels of r-2 done)
      if (!w(ver + (size_t)k.r * R + k.r, k.r)) return false;
      if (k.r >= 2 && !w(done2, 2 * (R - 1) * (k.r - 1))) return false;
      return true;
    case 1:
    case 2:  // panel: its tile after round r-1, the pivot of r, snapshot slot free
      if (!w(ver + (size_t)k.ti * R + k.tj, k.r)) return false;
      if (!w(ver + (size_t)k.r * R + k.r, k.r + 1)) return false;
      if (k.r >= 2 && !w(done3, (R - 1) * (R - 1) * (k.r - 1))) return false;
      return true;
    default:  // remaining tile: itself after r-1, both panels of round r
      if (!w(ver + (size_t)k.ti * R + k.tj, k.r)) return false;
      if (!w(ver + (size_t)k.ti * R + k.r, k.r + 1)) return false;
      if (!w(ver + (size_t)k.r * R + k.tj, k.r + 1)) return false;
      return true;
  }
}

template <typename T>
__device__ __forceinline__ void publish(const Args<T>& a, const fwh::Task& k) {
  st_release(a.ver + (size_t)k.ti * a.R + k.tj, k.r + 1);
  if (k.type == 1 || k.type == 2) red_release_add(a.ctr + 1, 1u);
  if (k.type == 3) red_release_add(a.ctr + 2, 1u);
}

template <typename T, int BS>
__global__ void __launch_bounds__(kThreads, 1) k_persistent(Args<T> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ CtaScratch cs;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&cs.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned phase = 0;
  const int64_t total = a.stage_off[a.R + 1];
  for (;;) {
    if (tid == 0) {
      const int64_t t = atomicAdd(a.ctr, 1u);
      int ok = t < total && !ld_relaxed(a.abort_flag);
      if (ok) ok = wait_deps(a, fwh::decode_task(t, a.R, a.lookahead, a.stage_off));
      if (ok) fence_proxy_async();
      cs.task = ok ? (int)t : -1;
    }
    __syncthreads();
    const int t = cs.task;
    if (t < 0) break;
    const fwh::Task k = fwh::decode_task(t, a.R, a.lookahead, a.stage_off);
    if (k.type == 0) {
      task_pivot<T, BS>(a, k.r, smem, &cs);
    } else if (k.type == 3) {
      task_minplus<T, BS>(a, k.r, k.ti, k.tj, smem, &cs, phase);
    } else {
      task_panel<T, BS>(a, k.r, k.type == 1 ? k.tj : k.ti, k.type == 1, smem, &cs);
    }
    __syncthreads();
    if (tid == 0 && t != a.skip_task) publish(a, k);
  }
}

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

template <typename T, int BS>
cudaError_t launch_bs(T* D, int32_t* P, int64_t n, int64_t ld, const fwh::SolveWs& ws,
                      const fwh::LaunchCfg& cfg, cudaStream_t s) {
  Args<T> a{};
  a.D = D; a.P = P; a.n = n; a.ld = ld; a.R = ws.R; a.slot_tiles = ws.slot_tiles;
  a.ver = ws.ver; a.ctr = ws.ctr; a.abort_flag = ws.abort_flag; a.status = ws.status;
  a.stage_off = ws.stage_off; a.lookahead = (int)cfg.lookahead; a.skip_task = cfg.skip_task;
  a.timeout_ns = cfg.timeout_ns; a.packed = cfg.packed;
  a.piv = reinterpret_cast<T*>(ws.piv); a.pivP = ws.pivP;
  a.colK = ws.colK; a.colR = reinterpret_cast<T*>(ws.colR); a.colB = ws.colB;
  a.rowK = ws.rowK; a.rowR = reinterpret_cast<T*>(ws.rowR); a.rowP = ws.rowP; a.rowB = ws.rowB;
  const int R = ws.R;
  const size_t smem = Smem<BS>::bytes();
  cudaError_t e;

  {
    int64_t blocks = (n * n + 255) / 256;
    const int cap = fwh::num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_init_pred<T><<<(int)blocks, 256, 0, s>>>(D, P, n, ld);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (cfg.ev_start) cudaEventRecord(cfg.ev_start, s);
  if (cfg.driver == 2) {
    static bool attr_done = false;
    if (!attr_done) {
      cudaFuncSetAttribute(k_phase_pivot<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_phase_panel<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_phase_rest<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr_done = true;
    }
    for (int r = 0; r < R; ++r) {
      k_phase_pivot<T, BS><<<1, kThreads, smem, s>>>(a, r);
      if (R > 1) {
        k_phase_panel<T, BS><<<2 * (R - 1), kThreads, smem, s>>>(a, r);
        k_phase_rest<T, BS><<<(R - 1) * (R - 1), kThreads, smem, s>>>(a, r);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  } else {
    auto kern = k_persistent<T, BS>;
    static int occ = -1;
    if (occ < 0) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      int o = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kThreads, smem);
      occ = o > 0 ? o : 1;
    }
    int64_t grid = cfg.grid > 0 ? cfg.grid : (int64_t)occ * fwh::num_sms();
    if (grid > (int64_t)occ * fwh::num_sms()) grid = (int64_t)occ * fwh::num_sms();
    const int64_t total = (int64_t)R * R * R;
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kThreads);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    if ((e = cudaLaunchKernelEx(&lc, kern, a)) != cudaSuccess) return e;
  }
  if (cfg.ev_stop) cudaEventRecord(cfg.ev_stop, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_any(T* D, int32_t* P, int64_t n, int64_t ld, const fwh::SolveWs& ws,
                       const fwh::LaunchCfg& cfg, cudaStream_t s) {
  switch (cfg.BS) {
    case 32: return launch_bs<T, 32>(D, P, n, ld, ws, cfg, s);
    case 64: return launch_bs<T, 64>(D, P, n, ld, ws, cfg, s);
    case 128: return launch_bs<T, 128>(D, P, n, ld, ws, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fwk
