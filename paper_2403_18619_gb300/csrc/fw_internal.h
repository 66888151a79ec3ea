// Host-side internals shared by the translation units of libfw.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fw.h"

namespace fwh {

// Queue layout of the persistent driver, shared by host and device.
//
// Tasks: 0 pivot (r,r); 1 row panel (r,t); 2 column panel (t,r); 3 remaining
// tile (ti,tj).  Round r has R^2 tasks.  The queue is cut into R+1 stages:
//   stage 0        : P1(0), P2(0) x 2(R-1), L(0)
//   stage s (1..R-1): P1(s), Rest(s-1)[0:g], P2(s) x 2(R-1), Rest(s-1)[g:], L(s)
//   stage R        : Rest(R-1)
// where L(r) are round r's remaining tiles in tile row / column r+1 (the
// inputs of round r+1's pivot and panels) and Rest(r) the other remaining
// tiles of round r; g = min(lookahead, |Rest(s-1)|).  Every task's inputs are
// produced by tasks earlier in the queue, so claiming tasks in queue order
// with all CTAs co-resident cannot deadlock.
struct Task {
  int type, r, ti, tj;
};

__host__ __device__ inline int64_t size_L(int R, int r) { return (r + 1 < R) ? 2 * (int64_t)R - 3 : 0; }
__host__ __device__ inline int64_t size_rest(int R, int r) {
  return (int64_t)(R - 1) * (R - 1) - size_L(R, r);
}
// Automatic lookahead g for `sms` co-resident CTAs: enough remaining tiles
// of round s-1 ahead of the panels of round s that the panels are claimed as
// the pivot finishes (its inputs' wait plus the pivot itself last about six
// BS = 128 remaining-tile tasks; claimed earlier, a panel task idles its SM
// until then), while leaving at least three tasks per CTA behind the panels
// to cover their own latency before round s's remaining tiles need them.
__host__ __device__ inline int64_t auto_lookahead(int R, int sms) {
  const int64_t nrest = size_rest(R, 0);
  int64_t g = nrest - 3 * (int64_t)sms;
  if (g > 6 * (int64_t)sms) g = 6 * (int64_t)sms;
  if (g < 2 * (int64_t)sms) g = 2 * (int64_t)sms;
  return g;
}
__host__ __device__ inline int64_t stage_size(int R, int s, int64_t look) {
  if (s == 0) return 1 + 2 * (int64_t)(R - 1) + size_L(R, 0);
  if (s == R) return size_rest(R, R - 1);
  return 1 + 2 * (int64_t)(R - 1) + size_rest(R, s - 1) + size_L(R, s);
}

__host__ __device__ inline Task task_L(int R, int r, int64_t l) {
  if (l == 0) return Task{3, r, r + 1, r + 1};
  const int k = (int)((l - 1) >> 1);
  const int jj = (r + 2 + k) % R;
  return ((l - 1) & 1) ? Task{3, r, jj, r + 1} : Task{3, r, r + 1, jj};
}
__host__ __device__ inline Task task_rest(int R, int r, int64_t u) {
  // u < R^2 <= 2^20: 32-bit arithmetic
  const unsigned uu = (unsigned)u;
  if (r + 1 < R) {
    const unsigned w = (unsigned)(R - 2);
    int i = (int)(uu / w), j = (int)(uu - (unsigned)i * w);
    i = i < r ? i : i + 2;
    j = j < r ? j : j + 2;
    return Task{3, r, i, j};
  }
  const unsigned w = (unsigned)(R - 1);
  int i = (int)(uu / w), j = (int)(uu - (unsigned)i * w);
  i = i < r ? i : i + 1;
  j = j < r ? j : j + 1;
  return Task{3, r, i, j};
}
__host__ __device__ inline Task task_panel(int R, int r, int64_t q) {
  const int k = (int)(q >> 1);
  const int jj = (r + 1 + k) % R;
  return (q & 1) ? Task{2, r, jj, r} : Task{1, r, r, jj};
}

// off: R+2 stage starts (off[R+1] = total = R^3).
__host__ __device__ inline Task decode_task(int64_t t, int R, int64_t look, const unsigned* off) {
  int lo = 0, hi = R;  // find s with off[s] <= t < off[s+1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)off[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int s = lo;
  int64_t u = t - (int64_t)off[s];
  if (s == R) return task_rest(R, R - 1, u);
  if (u == 0) return Task{0, s, s, s};
  u -= 1;
  const int64_t np = 2 * (int64_t)(R - 1);
  if (s == 0) {
    if (u < np) return task_panel(R, 0, u);
    return task_L(R, 0, u - np);
  }
  const int64_t nrest = size_rest(R, s - 1);
  const int64_t g = look < nrest ? look : nrest;
  if (u < g) return task_rest(R, s - 1, u);
  u -= g;
  if (u < np) return task_panel(R, s, u);
  u -= np;
  if (u < nrest - g) return task_rest(R, s - 1, g + u);
  u -= nrest - g;
  return task_L(R, s, u);
}

inline void fill_stage_offsets(int R, int64_t look, unsigned* off) {
  int64_t acc = 0;
  for (int s = 0; s <= R; ++s) {
    off[s] = (unsigned)acc;
    acc += stage_size(R, s, look);
  }
  off[R + 1] = (unsigned)acc;
}

// Device workspace of one solve (carved from one allocation).
struct SolveWs {
  int* ver = nullptr;
  int* done = nullptr;  // [2R]: panel tasks done per round, then remaining tiles done per round
  unsigned* ctr = nullptr;
  int* abort_flag = nullptr;
  int* status = nullptr;
  unsigned* stage_off = nullptr;
  void* piv = nullptr;
  int32_t* pivP = nullptr;
  uint32_t* colK = nullptr;
  void* colR = nullptr;
  int32_t* colB = nullptr;
  uint32_t* rowK = nullptr;
  void* rowR = nullptr;
  int32_t* rowP = nullptr;
  int32_t* rowB = nullptr;
  int R = 0, BS = 0, slot_tiles = 0;
  size_t flags_bytes = 0;  // ver + done + ctr + abort (zeroed before each solve)
};

// Bytes needed by a solve of R tiles of BS with esize-byte elements (4: int32
// or fp32, with the packed-key snapshots; 8: int64 or fp64, without them).
size_t solve_ws_bytes(int R, int BS, int esize = 4);
// Carve a workspace out of `base` (cudaMalloc'd, >= solve_ws_bytes).
SolveWs carve_solve_ws(void* base, int R, int BS, int esize = 4);

struct LaunchCfg {
  int BS;
  int driver;        // 1 persistent, 2 phased
  int64_t lookahead;
  int grid;
  int64_t timeout_ns;
  int packed;
  int skip_task;
  cudaEvent_t ev_start, ev_stop;
  uint64_t* trace = nullptr;
  int64_t trace_cap = 0;
  int trace_stride = 0;
  bool tile_tma = true;
};

// Enqueue one solve (init + driver).  Returns a cudaError_t.
cudaError_t launch_solve_i32(int32_t* D, int32_t* P, int64_t n, int64_t ld, const SolveWs& ws,
                             const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_solve_f32(float* D, int32_t* P, int64_t n, int64_t ld, const SolveWs& ws,
                             const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_solve_i64(int64_t* D, int32_t* P, int64_t n, int64_t ld, const SolveWs& ws,
                             const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_solve_f64(double* D, int32_t* P, int64_t n, int64_t ld, const SolveWs& ws,
                             const LaunchCfg& cfg, cudaStream_t s);

int num_sms();

// Dynamic shared-memory opt-in (smem bytes) and the number of co-resident CTAs
// of `threads` threads per SM for kernel `fn` on the CURRENT device.  The
// opt-in belongs to a device's context, so it is applied once per (device,
// kernel) under a lock and cached there.  Returns <= 0 on failure.
int kernel_setup(const void* fn, size_t smem, int threads);

// Tensor map of a row-major n x n matrix of `dt` elements (esize bytes each)
// with leading dimension ld (elements), read in box x box tiles (2-D TMA).
// False when the driver offers no encoder or rejects the layout; callers then
// copy by rows.
bool encode_tile_map(CUtensorMap* map, const void* base, int64_t n, int64_t ld, int box,
                     CUtensorMapDataType dt, int esize);

}  // namespace fwh
