// Host side of the C ABI (include/fw.h): argument checks, workspace cache and
// dispatch to the solver launchers.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "fw_internal.h"

namespace fwh {

namespace {

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct StreamWs {
  void* base = nullptr;
  size_t bytes = 0;
  int cached_R = -1, cached_BS = -1;
  int64_t cached_look = -1;
  // host-buffer path (fw_solve_host)
  void* hd = nullptr;
  void* hp = nullptr;
  size_t hbytes = 0;
  cudaStream_t side = nullptr;     // copies dist back while pred is still resolved
  cudaEvent_t ev_solved = nullptr, ev_side = nullptr;
  int* status = nullptr;  // sticky status word of this stream (lives in `sbase`)
  void* sbase = nullptr;
  void* bwd = nullptr;    // backward scratch (subtree sums)
  size_t bwd_bytes = 0;
  std::mutex mu;          // guards this entry; taken after g_mu, never the other way round
};

std::mutex g_mu;       // guards the map g_ws (entries are guarded by their own mutex)
std::mutex g_sms_mu;   // guards g_sms (taken on its own, also while g_mu is held)
std::map<std::pair<int, cudaStream_t>, StreamWs> g_ws;
std::map<int, int> g_sms;
std::mutex g_ksetup_mu;  // guards g_ksetup (taken on its own, also while g_mu is held)
std::map<std::pair<int, const void*>, int> g_ksetup;  // (device, kernel) -> CTAs per SM

}  // namespace

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}
}  // namespace

bool encode_tile_map(CUtensorMap* map, const void* base, int64_t n, int64_t ld, int box,
                     CUtensorMapDataType dt, int esize) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || n <= 0 || box <= 0 || box > 256 || (esize != 4 && esize != 8)) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * esize) & 15)) return false;
  if (((int64_t)box * esize) & 15) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  const cuuint32_t boxd[2] = {(cuuint32_t)box, (cuuint32_t)box};
  const cuuint32_t estr[2] = {1, 1};
  // elements outside [0, n) read as zero; the kernels mask them
  return fn(map, dt, 2,
            const_cast<void*>(base), dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_sms_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  if (v <= 0) v = 1;
  g_sms[dev] = v;
  return v;
}

int kernel_setup(const void* fn, size_t smem, int threads) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lk(g_ksetup_mu);
  auto it = g_ksetup.find({dev, fn});
  if (it != g_ksetup.end()) return it->second;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return -1;
  }
  g_ksetup[{dev, fn}] = occ;
  return occ;
}

size_t solve_ws_bytes(int R, int BS, int esize) {
  const size_t t = (size_t)BS * BS;
  const size_t keys = esize == 4 ? 2 : 0;  // packed-key snapshots (32-bit elements only)
  size_t b = 0;
  b += up(((size_t)R * R + 2 * (size_t)R) * 4 + 4 * 4 + 4);  // ver + done + ctr + abort
  b += up((size_t)(R + 2) * 4);              // stage offsets
  b += up(2 * t * esize) + up(2 * t * 4);    // piv, pivP
  b += up(2 * (size_t)R * t * 4) * keys;     // colK, rowK
  b += up(2 * (size_t)R * t * esize) * 2;    // colR, rowR
  b += up(2 * (size_t)R * t * 4);            // rowP
  b += up(2 * (size_t)R * 4) * 2;            // colB, rowB
  return b + kAlign;
}

SolveWs carve_solve_ws(void* base, int R, int BS, int esize) {
  SolveWs w;
  char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(base) + kAlign - 1) / kAlign * kAlign);
  const size_t t = (size_t)BS * BS;
  w.ver = reinterpret_cast<int*>(p);
  w.done = w.ver + (size_t)R * R;
  w.ctr = reinterpret_cast<unsigned*>(w.done + 2 * (size_t)R);
  w.abort_flag = reinterpret_cast<int*>(w.ctr + 4);
  w.flags_bytes = ((size_t)R * R + 2 * (size_t)R) * 4 + 4 * 4 + 4;
  p += up(w.flags_bytes);
  w.stage_off = reinterpret_cast<unsigned*>(p);  p += up((size_t)(R + 2) * 4);
  w.piv = p;                                     p += up(2 * t * esize);
  w.pivP = reinterpret_cast<int32_t*>(p);        p += up(2 * t * 4);
  if (esize == 4) {
    w.colK = reinterpret_cast<uint32_t*>(p);     p += up(2 * (size_t)R * t * 4);
    w.rowK = reinterpret_cast<uint32_t*>(p);     p += up(2 * (size_t)R * t * 4);
  }
  w.colR = p;                                    p += up(2 * (size_t)R * t * esize);
  w.rowR = p;                                    p += up(2 * (size_t)R * t * esize);
  w.rowP = reinterpret_cast<int32_t*>(p);        p += up(2 * (size_t)R * t * 4);
  w.colB = reinterpret_cast<int32_t*>(p);        p += up(2 * (size_t)R * 4);
  w.rowB = reinterpret_cast<int32_t*>(p);        p += up(2 * (size_t)R * 4);
  w.R = R; w.BS = BS; w.slot_tiles = R;
  return w;
}

// Automatic BS of a single solve.  Larger blocks relax faster (BS = 128 runs
// the DPX loop at ~84 % of peak, BS = 64 at ~50 %) but make R = n / BS rounds
// whose pivot -> panel chain is longer; measured on GB300 (int32, persistent
// driver): n = 2048 BS 64 1.27 ms vs BS 128 2.16 ms; n = 4096 BS 64 7.70 ms vs
// BS 128 5.91 ms.  The two costs cross near n = 3072.
int pick_bs(int64_t n, fw_dtype dtype = FW_I32) {
  if (n <= 512) return 32;
  if (n <= 3072 || dtype == FW_I64 || dtype == FW_F64) return 64;
  return 128;
}

int dtype_size(fw_dtype dtype) { return (dtype == FW_I64 || dtype == FW_F64) ? 8 : 4; }
bool dtype_valid(fw_dtype dtype) {
  return dtype == FW_I32 || dtype == FW_F32 || dtype == FW_I64 || dtype == FW_F64;
}

// The workspace entry of (current device, stream), created if missing, locked
// for the caller.  Host threads working on different streams hold different
// entries and do not wait for each other.
static std::unique_lock<std::mutex> lock_entry(cudaStream_t s, StreamWs** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *out = nullptr;
    return std::unique_lock<std::mutex>();
  }
  std::lock_guard<std::mutex> g(g_mu);
  StreamWs& w = g_ws[{dev, s}];
  std::unique_lock<std::mutex> lk(w.mu);
  *out = &w;
  return lk;
}

// Grows the locked entry w of stream s to `need` bytes of solve workspace
// (and creates its status word).
static fw_status get_ws(StreamWs& w, cudaStream_t s, size_t need) {
  if (!w.sbase) {
    if (cudaMalloc(&w.sbase, 256) != cudaSuccess) return FW_ERR_NOMEM;
    if (cudaMemset(w.sbase, 0, 256) != cudaSuccess) return FW_ERR_CUDA;
    w.status = reinterpret_cast<int*>(w.sbase);
  }
  if (w.bytes < need) {
    if (w.base) {
      cudaStreamSynchronize(s);
      cudaFree(w.base);
      w.base = nullptr;
      w.bytes = 0;
    }
    if (cudaMalloc(&w.base, need) != cudaSuccess) {
      cudaGetLastError();
      return FW_ERR_NOMEM;
    }
    w.bytes = need;
    w.cached_R = -1;
  }
  return FW_OK;
}

// pred may be null: a distance-only solve.
fw_status check_matrix_args(const void* dist, const void* pred, int64_t n, int64_t ld) {
  if (!dist) return FW_ERR_ARG;
  if (n <= 0 || n > 131072 || ld < n || (ld % 4) != 0) return FW_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(dist) & 15) || (reinterpret_cast<uintptr_t>(pred) & 15))
    return FW_ERR_ARG;
  if (dist == (const void*)pred) return FW_ERR_ARG;
  return FW_OK;
}

fw_status check_options(const fw_options& o) {
  if (o.bs != 0 && o.bs != 32 && o.bs != 64 && o.bs != 128) return FW_ERR_ARG;
  if (o.driver < 0 || o.driver > 2) return FW_ERR_ARG;
  if (o.grid < 0 || o.timeout_ns < 0) return FW_ERR_ARG;
  if (o.trace && (o.trace_cap <= 0 || o.trace_cap > (1 << 30) || o.trace_stride <= 0)) return FW_ERR_ARG;
  if (o.tile_tma != 0 && o.tile_tma != 1) return FW_ERR_ARG;
  return FW_OK;
}

fw_status solve_device(void* dist, int32_t* pred, int64_t n, int64_t ld, fw_dtype dtype,
                       const fw_options& o, cudaStream_t s) {
  const int esize = dtype_size(dtype);
  const int BS = o.bs ? o.bs : pick_bs(n, dtype);
  if (esize == 8 && BS > 64) return FW_ERR_UNSUPPORTED;
  const int64_t R64 = (n + BS - 1) / BS;
  if (R64 > 1024) return FW_ERR_UNSUPPORTED;
  const int R = (int)R64;
  int64_t look = o.lookahead;
  if (look < 0) look = auto_lookahead(R, num_sms());

  StreamWs* w = nullptr;
  auto lk = lock_entry(s, &w);
  if (!w) return FW_ERR_CUDA;
  fw_status st = get_ws(*w, s, solve_ws_bytes(R, BS, esize));
  if (st != FW_OK) return st;
  SolveWs ws = carve_solve_ws(w->base, R, BS, esize);
  ws.status = w->status;
  if (w->cached_R != R || w->cached_BS != BS || w->cached_look != look) {
    std::vector<unsigned> off(R + 2);
    fill_stage_offsets(R, look, off.data());
    if (cudaMemcpyAsync(ws.stage_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return FW_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FW_ERR_CUDA;
    w->cached_R = R; w->cached_BS = BS; w->cached_look = look;
  }
  if (cudaMemsetAsync(ws.ver, 0, ws.flags_bytes, s) != cudaSuccess) return FW_ERR_CUDA;
  LaunchCfg cfg;
  cfg.BS = BS;
  cfg.driver = o.driver == FW_DRIVER_PHASED ? 2 : 1;
  cfg.lookahead = look;
  cfg.grid = o.grid;
  cfg.timeout_ns = o.timeout_ns > 0 ? o.timeout_ns : 2000000000LL;
  cfg.packed = o.packed_keys ? 1 : 0;
  cfg.skip_task = o.debug_skip_release;
  cfg.ev_start = reinterpret_cast<cudaEvent_t>(o.ev_start);
  cfg.ev_stop = reinterpret_cast<cudaEvent_t>(o.ev_stop);
  cfg.trace = o.trace;
  cfg.trace_cap = o.trace_cap;
  cfg.trace_stride = o.trace_stride;
  cfg.tile_tma = o.tile_tma != 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (dtype) {
    case FW_I32: e = launch_solve_i32(reinterpret_cast<int32_t*>(dist), pred, n, ld, ws, cfg, s); break;
    case FW_F32: e = launch_solve_f32(reinterpret_cast<float*>(dist), pred, n, ld, ws, cfg, s); break;
    case FW_I64: e = launch_solve_i64(reinterpret_cast<int64_t*>(dist), pred, n, ld, ws, cfg, s); break;
    case FW_F64: e = launch_solve_f64(reinterpret_cast<double*>(dist), pred, n, ld, ws, cfg, s); break;
  }
  return e == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

// Backward scratch of (current device, stream), grown to `bytes`.
void* backward_scratch(cudaStream_t s, size_t bytes) {
  StreamWs* wp = nullptr;
  auto lk = lock_entry(s, &wp);
  if (!wp) return nullptr;
  StreamWs& w = *wp;
  if (w.bwd_bytes < bytes) {
    if (w.bwd) {
      cudaStreamSynchronize(s);
      cudaFree(w.bwd);
      w.bwd = nullptr;
      w.bwd_bytes = 0;
    }
    if (cudaMalloc(&w.bwd, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    w.bwd_bytes = bytes;
  }
  return w.bwd;
}

// Status word of (current device, stream), created if the stream has none yet.
int* status_word_for(cudaStream_t s) {
  StreamWs* w = nullptr;
  auto lk = lock_entry(s, &w);
  if (!w || get_ws(*w, s, 0) != FW_OK) return nullptr;
  return w->status;
}

// Status word of (current device, stream); nullptr if the stream never solved.
int* stream_status(cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_ws.find({dev, s});
  if (it == g_ws.end()) return nullptr;
  std::lock_guard<std::mutex> lk2(it->second.mu);
  return it->second.status;
}

}  // namespace fwh

using namespace fwh;

extern "C" {

void fw_options_default(fw_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->bs = 0;
  o->driver = FW_DRIVER_AUTO;
  o->lookahead = -1;
  o->grid = 0;
  o->timeout_ns = 0;
  o->packed_keys = 1;
  o->debug_skip_release = -1;
  o->ev_start = nullptr;
  o->ev_stop = nullptr;
  o->trace = nullptr;
  o->trace_cap = 0;
  o->trace_stride = 0;
  o->tile_tma = 1;
  o->debug_shuffle = 0;
}

const char* fw_status_string(fw_status s) {
  switch (s) {
    case FW_OK: return "ok";
    case FW_ERR_ARG: return "invalid argument";
    case FW_ERR_CUDA: return "CUDA error";
    case FW_ERR_TIMEOUT: return "device dependency wait timed out";
    case FW_ERR_NEG_CYCLE: return "negative cycle (a diagonal distance is negative)";
    case FW_ERR_NOMEM: return "out of memory";
    case FW_ERR_UNSUPPORTED: return "unsupported dtype or size";
  }
  return "unknown status";
}

fw_status fw_solve_ex(void* dist, int32_t* pred, int64_t n, int64_t ld, fw_dtype dtype,
                      const fw_options* opt, void* stream) {
  fw_options o;
  fw_options_default(&o);
  if (opt) o = *opt;
  fw_status st = check_matrix_args(dist, pred, n, ld);
  if (st != FW_OK) return st;
  if (!dtype_valid(dtype)) return FW_ERR_ARG;
  if ((st = check_options(o)) != FW_OK) return st;
  return solve_device(dist, pred, n, ld, dtype, o, reinterpret_cast<cudaStream_t>(stream));
}

fw_status fw_solve(void* dist, int32_t* pred, int64_t n, int64_t ld, fw_dtype dtype,
                   void* stream) {
  return fw_solve_ex(dist, pred, n, ld, dtype, nullptr, stream);
}

fw_status fw_sync_status(void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return FW_ERR_CUDA;
  int* st = stream_status(s);
  if (!st) return FW_OK;
  int v = 0;
  if (cudaMemcpy(&v, st, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return FW_ERR_CUDA;
  if (v) cudaMemset(st, 0, 4);
  if (v & 1) return FW_ERR_TIMEOUT;
  if (v & 2) return FW_ERR_NEG_CYCLE;
  return FW_OK;
}

fw_status fw_solve_host(void* dist_host, int32_t* pred_host, int64_t n, int64_t ld,
                        fw_dtype dtype, const fw_options* opt, void* stream) {
  return fw_solve_host_io(dist_host, dist_host, pred_host, n, ld, dtype, opt, stream);
}

fw_status fw_solve_host_io(const void* w_host, void* dist_host, int32_t* pred_host, int64_t n,
                           int64_t ld, fw_dtype dtype, const fw_options* opt, void* stream) {
  if (!w_host || !dist_host) return FW_ERR_ARG;
  if (n <= 0 || n > 131072 || ld < n || (ld % 4) != 0) return FW_ERR_ARG;
  if (!dtype_valid(dtype)) return FW_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)n * ld * dtype_size(dtype);  // dist (pred needs no more)
  void* dd = nullptr;
  void* dp = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_side = nullptr;
  fw_options o;
  if (opt) o = *opt;
  else fw_options_default(&o);
  {
    StreamWs* wp = nullptr;
    auto lk = lock_entry(s, &wp);
    if (!wp) return FW_ERR_CUDA;
    StreamWs& w = *wp;
    if (w.hbytes < bytes) {
      if (w.hd) { cudaStreamSynchronize(s); cudaFree(w.hd); cudaFree(w.hp); w.hd = w.hp = nullptr; }
      if (cudaMalloc(&w.hd, bytes) != cudaSuccess || cudaMalloc(&w.hp, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (w.hd) cudaFree(w.hd);
        w.hd = w.hp = nullptr;
        w.hbytes = 0;
        return FW_ERR_NOMEM;
      }
      w.hbytes = bytes;
    }
    if (!w.side) {
      if (cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&w.ev_solved, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&w.ev_side, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return FW_ERR_CUDA;
      }
    }
    dd = w.hd;
    dp = w.hp;
    side = w.side;
    ev_side = w.ev_side;
    o.ev_stop = o.ev_stop ? o.ev_stop : reinterpret_cast<void*>(w.ev_solved);
  }
  // the n x n block only (rows ld apart): the caller's padding columns are
  // neither read nor written (one plain copy when there are none)
  const size_t pitch = (size_t)ld * dtype_size(dtype), width = (size_t)n * dtype_size(dtype);
  const size_t ppitch = (size_t)ld * 4, pwidth = (size_t)n * 4;
  auto copy_block = [&](void* dst, const void* src, size_t p, size_t w, cudaMemcpyKind kind,
                        cudaStream_t st) {
    return p == w ? cudaMemcpyAsync(dst, src, w * (size_t)n, kind, st)
                  : cudaMemcpy2DAsync(dst, p, src, p, w, (size_t)n, kind, st);
  };
  if (copy_block(dd, w_host, pitch, width, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FW_ERR_CUDA;
  fw_status st = fw_solve_ex(dd, pred_host ? reinterpret_cast<int32_t*>(dp) : nullptr, n, ld,
                             dtype, &o, stream);
  if (st != FW_OK) return st;
  // The distances are final at ev_stop (the int32 solve's last pass rewrites
  // only pred): they leave on the side stream while that pass runs.
  if (cudaStreamWaitEvent(side, reinterpret_cast<cudaEvent_t>(o.ev_stop), 0) != cudaSuccess ||
      copy_block(dist_host, dd, pitch, width, cudaMemcpyDeviceToHost, side) != cudaSuccess ||
      cudaEventRecord(ev_side, side) != cudaSuccess ||
      (pred_host &&
       copy_block(pred_host, dp, ppitch, pwidth, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
      cudaStreamWaitEvent(s, ev_side, 0) != cudaSuccess)
    return FW_ERR_CUDA;
  return fw_sync_status(stream);
}

fw_status fw_release_workspace(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FW_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return FW_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->first.first == dev) {
      StreamWs& w = it->second;
      { std::lock_guard<std::mutex> wait_for_user(w.mu); }  // no other thread is inside this entry
      if (w.base) cudaFree(w.base);
      if (w.hd) cudaFree(w.hd);
      if (w.hp) cudaFree(w.hp);
      if (w.side) cudaStreamDestroy(w.side);
      if (w.ev_solved) cudaEventDestroy(w.ev_solved);
      if (w.ev_side) cudaEventDestroy(w.ev_side);
      if (w.sbase) cudaFree(w.sbase);
      if (w.bwd) cudaFree(w.bwd);
      it = g_ws.erase(it);
    } else {
      ++it;
    }
  }
  return FW_OK;
}

fw_status fw_solve_plan(int64_t n, fw_dtype dtype, const fw_options* opt, int32_t sms,
                        int32_t* bs, int32_t* rounds, int64_t* lookahead,
                        int64_t* workspace_bytes) {
  fw_options o;
  if (opt) o = *opt;
  else fw_options_default(&o);
  if (n <= 0 || n > 131072 || sms < 1 || !dtype_valid(dtype)) return FW_ERR_ARG;
  if (check_options(o) != FW_OK) return FW_ERR_ARG;
  const bool wide = dtype_size(dtype) == 8;
  if (wide && o.bs == 128) return FW_ERR_UNSUPPORTED;  // 64-bit types take BS 32 or 64
  const int BS = o.bs ? o.bs : pick_bs(n, dtype);
  const int64_t R64 = (n + BS - 1) / BS;
  if (R64 > 1024) return FW_ERR_UNSUPPORTED;
  const int R = (int)R64;
  if (bs) *bs = BS;
  if (rounds) *rounds = R;
  if (lookahead) *lookahead = o.lookahead < 0 ? auto_lookahead(R, sms) : o.lookahead;
  if (workspace_bytes) *workspace_bytes = (int64_t)solve_ws_bytes(R, BS, dtype_size(dtype));
  return FW_OK;
}

fw_status fw_queue_tasks(int32_t R, int64_t lookahead, int64_t first, int64_t count,
                         int32_t* out) {
  if (R < 1 || R > 1024 || lookahead < 0 || first < 0 || count < 0 || !out) return FW_ERR_ARG;
  const int64_t total = (int64_t)R * R * R;
  if (first + count > total) return FW_ERR_ARG;
  std::vector<unsigned> off(R + 2);
  fill_stage_offsets(R, lookahead, off.data());
  if ((int64_t)off[R + 1] != total) return FW_ERR_CUDA;
  for (int64_t t = 0; t < count; ++t) {
    const Task k = decode_task(first + t, R, lookahead, off.data());
    out[4 * t + 0] = k.type;
    out[4 * t + 1] = k.r;
    out[4 * t + 2] = k.ti;
    out[4 * t + 3] = k.tj;
  }
  return FW_OK;
}

}  // extern "C"
