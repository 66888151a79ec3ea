// fw_solve_noalloc: the persistent solve for callers that cannot allocate
// device memory.
//
// fw_solve keeps a per-stream workspace that it obtains with cudaMalloc the
// first time a stream solves a problem of a given size.  Some callers cannot
// let a library do that: code running under a fixed device-memory budget
// managed by another allocator (a framework's caching pool, a serving process
// that has reserved all free memory up front), code that must not hit
// cudaMalloc's implicit device-wide synchronisation in a latency-critical
// loop, or hosts whose policy forbids allocations outside their own pool.  This
// entry point runs the same persistent kernel with its workspace placed in one
// file-scope __device__ array of fixed size instead.
//
// The array is part of the library's device image: every GPU on which the
// library's kernels are loaded holds kScratchBytes for it until the process
// exits, whether or not this entry point is ever called.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "fw_solve_impl.cuh"

namespace {

// Largest graph this entry point accepts, and the scratch that covers it
// (flags, queue offsets and the panel snapshots of a solve with BS = 64 and
// R = 64 tiles per side, about 10.6 MB, plus the status word).
constexpr int64_t kMaxN = 4096;
constexpr size_t kScratchBytes = (size_t)12 << 20;
constexpr size_t kStatusBytes = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side cache of the device address of g_scratch, one per device.  Host
// code must never pass `g_scratch` itself to a kernel: on the host that name is
// only a stand-in for the symbol, not a device address.  The address is looked
// up once per device and kept for the life of the process; after a
// cudaDeviceReset the library's module is loaded again and the kept address is
// stale, so calls after a device reset are not supported.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mu;

__global__ void k_stage_offsets(unsigned* off, int R, int64_t look) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t acc = 0;
    for (int s = 0; s <= R; ++s) {
      off[s] = (unsigned)acc;
      acc += fwh::stage_size(R, s, look);
    }
    off[R + 1] = (unsigned)acc;
  }
}

template <typename T, int BS>
cudaError_t run(T* D, int32_t* P, int64_t n, int64_t ld, unsigned char* base, int sms,
                cudaStream_t s) {
  using namespace fwk;
  const int R = (int)((n + BS - 1) / BS);
  const int64_t look = fwh::auto_lookahead(R, sms);
  int* status = reinterpret_cast<int*>(base);
  fwh::SolveWs ws = fwh::carve_solve_ws(base + kStatusBytes, R, BS);
  cudaError_t e;
  // everything a solve expects to start at zero: status, tile flags, counters
  if ((e = cudaMemsetAsync(status, 0, sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.ver, 0, ws.flags_bytes, s)) != cudaSuccess) return e;
  k_stage_offsets<<<1, 1, 0, s>>>(ws.stage_off, R, look);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  Args<T> a{};
  a.D = D; a.P = P; a.n = n; a.ld = ld; a.R = R; a.slot_tiles = ws.slot_tiles;
  a.ver = ws.ver; a.done = ws.done; a.ctr = ws.ctr; a.abort_flag = ws.abort_flag; a.status = status;
  a.stage_off = ws.stage_off; a.lookahead = (int)look; a.skip_task = -1;
  a.timeout_ns = 2000000000LL; a.packed = 1;
  a.piv = reinterpret_cast<T*>(ws.piv); a.pivP = ws.pivP;
  a.colK = ws.colK; a.colR = reinterpret_cast<T*>(ws.colR); a.colB = ws.colB;
  a.rowK = ws.rowK; a.rowR = reinterpret_cast<T*>(ws.rowR); a.rowP = ws.rowP; a.rowB = ws.rowB;

  int64_t blocks = (n * n + 255) / 256;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (P) {
    k_init_pred<T><<<(int)blocks, 256, 0, s>>>(D, P, n, ld);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }

  const size_t smem = WsLayout<BS, T>::bytes();
  auto kern = k_persistent_ws<T, BS>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWsThreads, smem)) !=
      cudaSuccess)
    return e;
  int64_t grid = (int64_t)(occ > 0 ? occ : 1) * sms;
  const int64_t total = (int64_t)R * R * R;
  if (grid > total) grid = total;
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3((unsigned)grid);
  lc.blockDim = dim3(kWsThreads);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  // the tensor map would be a second copy of the caller's layout per call;
  // this entry point keeps the per-row tile copies
  CUtensorMap tm{};
  if ((e = cudaLaunchKernelEx(&lc, kern, a, tm, tm, 0)) != cudaSuccess) return e;
  if (ViaPred<T>::kOn && P) {
    k_resolve_pred<<<(int)blocks, 256, 0, s>>>(P, n, ld);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" fw_status fw_solve_noalloc(void* dist, int32_t* pred, int64_t n, int64_t ld,
                                      fw_dtype dtype, void* stream) {
  if (!dist || dist == (void*)pred) return FW_ERR_ARG;  // pred null: distance-only
  if (n <= 0 || ld < n || (ld % 4) != 0) return FW_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(dist) & 15) || (reinterpret_cast<uintptr_t>(pred) & 15))
    return FW_ERR_ARG;
  if (dtype == FW_I64 || dtype == FW_F64) return FW_ERR_UNSUPPORTED;  // 32-bit types only
  if (dtype != FW_I32 && dtype != FW_F32) return FW_ERR_ARG;
  if (n > kMaxN) return FW_ERR_UNSUPPORTED;  // larger graphs need fw_solve's workspace
  const int BS = n <= 512 ? 32 : 64;
  const int R = (int)((n + BS - 1) / BS);
  if (fwh::solve_ws_bytes(R, BS) + kStatusBytes > kScratchBytes) return FW_ERR_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FW_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    // one-time set-up on this device (the device is current): the address of
    // the scratch array as the kernels must see it
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return FW_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = reinterpret_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return FW_ERR_CUDA;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (dtype == FW_I32) {
    e = BS == 32 ? run<int32_t, 32>(reinterpret_cast<int32_t*>(dist), pred, n, ld, base, sms, s)
                 : run<int32_t, 64>(reinterpret_cast<int32_t*>(dist), pred, n, ld, base, sms, s);
  } else {
    e = BS == 32 ? run<float, 32>(reinterpret_cast<float*>(dist), pred, n, ld, base, sms, s)
                 : run<float, 64>(reinterpret_cast<float*>(dist), pred, n, ld, base, sms, s);
  }
  if (e != cudaSuccess) return FW_ERR_CUDA;
  // synchronous: the status word comes back on the caller's stream, behind
  // the solve, and only that stream is waited for (no device-wide sync)
  int st = 0;
  if (cudaMemcpyAsync(&st, base, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FW_ERR_CUDA;
  if (st & fwk::kStTimeout) return FW_ERR_TIMEOUT;
  if (st & fwk::kStNegCycle) return FW_ERR_NEG_CYCLE;
  return FW_OK;
}
