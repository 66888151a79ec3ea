// Warp-specialised persistent driver (the GPU form of Opt-9's intra-round
// concurrency, Sec. 3.2, extended across rounds as the paper's future work
// proposes, Sec. 5).
//
// A CTA has 8 compute warps, 1 producer warp and 1 publisher warp.
//   * The producer claims tasks from a global queue in order, waits (bounded)
//     on the tiles' ready flags, and streams the operands of remaining-tile
//     tasks into shared memory with TMA copies while the compute warps work
//     on the previous task:
//       - the tile's own D block (one 2-D tensor copy, or one copy per row) -> Dbuf
//       - the A and B panel snapshots, 64 (fp32: 32) k-steps per chunk -> 2-stage ring
//       - the predecessor tile of the B panel (fp32 epilogue)          -> Pbuf
//     and, for int32 panel tasks, the tile and the closed pivot (ws_panel).
//   * The compute warps relax (min-plus over the chunks) and store improved
//     entries; pivot tasks (and the panels of the other element types) are
//     run by them alone, using the shared buffer as scratch (the producer
//     waits until such a task is published).  The task that finishes tile
//     (r+1, r+1) of round r runs the pivot of round r+1 right after it.
//   * The publisher sleeps on the compute warps' task-done barrier and
//     publishes each finished tile (the GPU-scope release), so that neither the
//     compute warps nor the producer wait on that fence.
// mbarriers carry "full" (transaction bytes landed) and "empty" (compute warps
// done reading) signals.
//
// The same engine runs one graph (fw_solve) or a batch of graphs with
// different sizes and block sizes in one launch (fw_solve_batched): a "task
// source" maps a global queue index to (graph, task).
#pragma once

#include "fw_device.cuh"
#include "fw_internal.h"

namespace fwk {

// 10 warps: 8 compute, 1 producer, 1 publisher.  Three of them share one SM
// sub-partition, whose 16K registers then cap the kernel at 168 registers per
// thread (ptxas derives this from the launch bounds).
constexpr int kWsThreads = kThreads + 64;
constexpr int kPubDepth = 4;  // tasks handed to the compute warps but not yet published
// Internal task type: remaining tile (r+1, r+1) of round r followed, on the
// same CTA and without a publication in between, by the pivot of round r+1
// (whose own queue entry is then skipped).  That tile is the pivot's only
// input, so the pivot starts as soon as the tile is relaxed: one hand-off
// less on the chain that bounds small solves (pivot -> panels -> tile ->
// next pivot).
constexpr int kFusedTask = 4;

// Operand chunks of a task with block size BS: CK k-steps of A and of B.
// int32 streams 64-step chunks (2 per task at BS = 128: fewer ring hand-offs);
// fp32 keeps 32-step chunks and spends the saved space on the predecessor
// snapshot tile of its epilogue.
// 64-bit elements stream 32-step chunks (BS is at most 64 for them).
template <int BS, typename T>
struct WsChunk {
  static constexpr int kCKmax = (ViaPred<T>::kOn && sizeof(T) == 4) ? 64 : 32;
  static constexpr int CK = BS < kCKmax ? BS : kCKmax;                    // k-steps per chunk
  static constexpr int NC = BS / CK;                                      // chunks per task
  static constexpr size_t kChunkBytes = (size_t)CK * BS * sizeof(T);      // one operand chunk
  static constexpr size_t kTile = (size_t)BS * BS * sizeof(T);            // a tile of elements
  static constexpr size_t kPTile = (size_t)BS * BS * 4;                   // a tile of int32 pred
};

// Shared-memory layout sized for the largest block size LBS a launch runs:
// the 2-stage operand ring, the tile's own D (Dbuf) and, for the floating
// types, the row-panel predecessor snapshot (Pbuf); 192 KB for LBS = 128 with
// 32-bit elements, 112 KB (fp64) or 96 KB (int64) for LBS = 64.
template <int LBS, typename T>
struct WsLayout {
  static constexpr size_t kStage = 2 * WsChunk<LBS, T>::kChunkBytes;  // A chunk + B chunk
  static constexpr size_t kRing = 2 * kStage;
  static constexpr size_t kTile = WsChunk<LBS, T>::kTile;
  static constexpr size_t kPTile = WsChunk<LBS, T>::kPTile;
  __host__ __device__ static constexpr size_t ring_off() { return 0; }
  __host__ __device__ static constexpr size_t d_off() { return kRing; }
  __host__ __device__ static constexpr size_t p_off() { return kRing + kTile; }
  __host__ __device__ static constexpr size_t bytes() {
    return kRing + kTile + (ViaPred<T>::kOn ? 0 : kPTile);
  }
  // pivot and panel tasks use the buffer from offset 0 as scratch (As, Bs of
  // elements and Ps of int32)
  static_assert(bytes() >= 2 * kTile + kPTile, "scratch of pivot / panel tasks");
  static_assert(bytes() <= 227 * 1024, "shared memory of one CTA");
};

struct WsBars {
  uint64_t desc_full[2], desc_empty[2];
  uint64_t chunk_full[2], chunk_empty[2];
  uint64_t d_full, d_empty, p_full, p_empty, task_done;
  uint64_t pub_full[kPubDepth], pub_empty[kPubDepth];
  int desc[2][8];           // t, type, r, ti, tj, fast, graph, key operands
  int pubq[kPubDepth][6];   // t, type, r, ti, tj, graph of tasks awaiting publication
};

// Bounded wait on an mbarrier phase; false (and the timeout status) on expiry.
// With poll_abort, a wait that has already lasted over a millisecond (normal
// waits take microseconds) also gives up, without recording anything, once
// another CTA has raised the abort flag, so that one failure does not make
// every pending wait of every CTA run out its own limit in turn.  Polling the
// flag from the start cost the compute warps' operand waits about 1 % of the
// n = 32768 solve.
constexpr uint64_t kAbortPollAfterNs = 1000000;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* status,
                                          int* abort_flag, int64_t timeout_ns,
                                          bool poll_abort = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (int64_t it = 0; it < ((int64_t)1 << 26); ++it) {
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
    if ((it & 15) == 15) {
      const uint64_t waited = globaltimer() - t0;
      if (waited > (uint64_t)timeout_ns) break;
      if (poll_abort && waited > kAbortPollAfterNs && ld_relaxed(abort_flag)) return false;
    }
  }
  atomicOr(status, kStTimeout);
  atomicExch(abort_flag, 1);
  return false;
}

// A cycle count clamped to 20 bits (three of them share a trace word).
__device__ __forceinline__ uint64_t cyc20(long long c) {
  return (uint64_t)(c < 0 ? 0 : c > 0xfffff ? 0xfffff : c);
}

// Scalars the compute warps need, passed by value (kept in registers).
template <typename T>
struct TileCtx {
  T* D;
  int32_t* P;
  int64_t n, ld;
  int r;                // round
  int* status;
  int* abort_flag;
  int64_t timeout_ns;
};

// Counters of the shared-memory pipelines (each side keeps its own copy).
// The producer also records, per full barrier, 1 + the last phase it armed
// with a copy (0: none), and stops arming once a wait has given up: arming a
// phase whose predecessor has not completed would add its bytes to the wrong
// phase.
// (The drain waits on the LAST phase of each barrier: a parity wait can only
// tell the latest two phases apart.)
struct PipeCnt {
  unsigned d = 0, chunk = 0, p = 0;
  unsigned d_armed = 0, p_armed = 0, chunk_armed[2] = {0, 0};
  bool stop = false;
};

// ------------------------------------------------------------ compute side ----

// In-place decode of `count` packed keys (int32 path) back to values, for a
// remaining tile relaxed with compare and select whose panel wrote its key
// snapshot only (exact: every finite value was below CAP).  Compute warps
// only; the caller synchronises them before reading the buffer.
template <int BS>
__device__ __forceinline__ void decode_keys(uint32_t* buf, int count) {
  using K = Keys<BS>;
  for (int i = (int)threadIdx.x * 4; i < count; i += kThreads * 4) {
    uint4 v = *reinterpret_cast<uint4*>(buf + i);
    auto d = [](uint32_t k) -> uint32_t {
      const uint32_t x = k >> K::KB;
      return x == (uint32_t)K::CAP ? (uint32_t)Num<int32_t>::inf() : x;
    };
    v.x = d(v.x);
    v.y = d(v.y);
    v.z = d(v.z);
    v.w = d(v.w);
    *reinterpret_cast<uint4*>(buf + i) = v;
  }
}

// Operands of a compare-and-select remaining tile that arrive as keys: decode
// them in the ring stage (bit 0: A, bit 1: B; every warp has waited for the
// stage to fill, so no warp still reads its previous contents) and
// synchronise the compute warps.
template <typename T, int BS, int CK>
__device__ __forceinline__ void decode_chunk(unsigned char* stage, int dec) {
  if constexpr (Num<T>::kPacked) {
    if (!dec) return;
    uint32_t* As = reinterpret_cast<uint32_t*>(stage);
    if (dec & 1) decode_keys<BS>(As, CK * BS);
    if (dec & 2) decode_keys<BS>(As + CK * BS, CK * BS);
    fence_proxy_async_shared();  // generic writes before the stage's next TMA fill
    bar_compute();
  }
}

// Distance-only remaining-tile task (no predecessors, generic kernel): add +
// min over the streamed chunks, then the whole tile written back (unchanged
// entries rewrite their own value).  A function of its own, so that the
// packed kernel's register allocation does not see it.
template <typename T, int BS, int LBS>
__device__ __noinline__ bool ws_minplus_dist(TileCtx<T> c, int ti, int tj, int dec,
                                             unsigned char* smem, WsBars* wb, PipeCnt& pc,
                                             uint64_t* tr) {
  using Gm = Geo<BS>;
  using L = WsLayout<LBS, T>;
  using C = WsChunk<BS, T>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31;
  const T* Dbuf = reinterpret_cast<const T*>(smem + L::d_off());
  unsigned char* ring = smem + L::ring_off();
  const int64_t row0 = (int64_t)ti * BS, col0 = (int64_t)tj * BS;
  const int nrow = (int)(c.n - row0 < BS ? c.n - row0 : BS);
  const int ncol = (int)(c.n - col0 < BS ? c.n - col0 : BS);
  const bool full = nrow == BS && ncol == BS;
  const long long t_a = tr ? clock64() : 0;
  long long cw = 0;
  if (!mbar_wait(&wb->d_full, pc.d & 1, c.status, c.abort_flag, c.timeout_ns)) return false;
  const long long t_b = tr ? clock64() : 0;
  T acc[TM][TM];
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int lr = Gm::idx(ty, m);
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      const int lc0 = g * Gm::SPAN + tx * G;
      T tmp[G];
      vload_s<G>(tmp, Dbuf + lr * BS + lc0);
#pragma unroll
      for (int e = 0; e < G; ++e)
        acc[m][g * G + e] = (lr < nrow && lc0 + e < ncol) ? tmp[e] : Num<T>::inf();
    }
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&wb->d_empty);
  ++pc.d;
  for (int ch = 0; ch < C::NC; ++ch) {
    const unsigned st = pc.chunk & 1;
    const long long w0 = tr ? clock64() : 0;
    if (!mbar_wait(&wb->chunk_full[st], (pc.chunk >> 1) & 1, c.status, c.abort_flag,
                   c.timeout_ns))
      return false;
    if (tr) cw += clock64() - w0;
    decode_chunk<T, BS, C::CK>(ring + st * L::kStage, dec);
    const T* As = reinterpret_cast<const T*>(ring + st * L::kStage);
    const T* Bs = As + C::CK * BS;
    core_min<BS, T, C::CK>(As, Bs, acc, tx, ty);
    __syncwarp();
    if (lane == 0) mbar_arrive(&wb->chunk_empty[st]);
    ++pc.chunk;
  }
  if (tr) {
    tr[7] = cyc20(t_b - t_a) | (cyc20(cw) << 20);
    tr[8] = (uint64_t)(clock64() - t_a);
  }
  T* Drow = c.D + row0 * c.ld + col0;
  bool neg = false;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int lr = Gm::idx(ty, m);
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      const int lc0 = g * Gm::SPAN + tx * G;
      T v[G];
#pragma unroll
      for (int e = 0; e < G; ++e) {
        v[e] = acc[m][g * G + e];
        neg |= (row0 + lr == col0 + lc0 + e) && v[e] < T(0);
      }
      if (full) {
        vstore<G>(Drow + lr * c.ld + lc0, v);
      } else if (lr < nrow) {
#pragma unroll
        for (int e = 0; e < G; ++e)
          if (lc0 + e < ncol) Drow[lr * c.ld + lc0 + e] = v[e];
      }
    }
  }
  if (tr) tr[8] |= (uint64_t)(clock64() - t_a) << 32;
  if (neg) atomicOr(c.status, kStNegCycle);
  return true;
}

// Remaining-tile task (phase 4 of round r, tile ti,tj).  Returns false if an
// operand never arrived (the kernel then stops).
template <typename T, int BS, int LBS>
__device__ __forceinline__ bool ws_minplus(TileCtx<T> c, int ti, int tj, bool fast, int dec,
                                        unsigned char* smem, WsBars* wb, PipeCnt& pc,
                                        uint64_t* tr) {
  if (!fast && !c.P) return ws_minplus_dist<T, BS, LBS>(c, ti, tj, dec, smem, wb, pc, tr);
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  using L = WsLayout<LBS, T>;
  using C = WsChunk<BS, T>;
  constexpr int TM = Gm::TM, G = Gm::G;
  constexpr bool kPacked = Num<T>::kPacked;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31;
  const T* Dbuf = reinterpret_cast<const T*>(smem + L::d_off());
  const int32_t* Pbuf = reinterpret_cast<const int32_t*>(smem + L::p_off());
  unsigned char* ring = smem + L::ring_off();
  const int64_t row0 = (int64_t)ti * BS, col0 = (int64_t)tj * BS;
  const int nrow = (int)(c.n - row0 < BS ? c.n - row0 : BS);  // valid rows / columns of the tile
  const int ncol = (int)(c.n - col0 < BS ? c.n - col0 : BS);
  const bool full = nrow == BS && ncol == BS;

  // optional per-phase SM-cycle counts (trace): Dbuf wait, operand-chunk
  // waits, predecessor-tile wait; start to end of the relaxation, whole task
  const long long t_a = tr ? clock64() : 0;
  long long cw = 0;
  // 1. the tile's current values (rows/columns beyond n read as INF)
  if (!mbar_wait(&wb->d_full, pc.d & 1, c.status, c.abort_flag, c.timeout_ns)) return false;
  const long long t_b = tr ? clock64() : 0;
  T old[TM][TM];
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int lr = Gm::idx(ty, m);
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      const int lc0 = g * Gm::SPAN + tx * G;
      T tmp[G];
      vload_s<G>(tmp, Dbuf + lr * BS + lc0);
#pragma unroll
      for (int e = 0; e < G; ++e)
        old[m][g * G + e] = (lr < nrow && lc0 + e < ncol) ? tmp[e] : Num<T>::inf();
    }
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&wb->d_empty);
  ++pc.d;

  T* Drow = c.D + row0 * c.ld + col0;
  int32_t* Prow = c.P + row0 * c.ld + col0;
  bool neg = false;
  if (kPacked && fast) {  // (packed keys: int32 only)
    uint32_t acc[TM][TM];
    int32_t omax = 0;
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        acc[m][nn] = kPacked ? key_of<BS>((int32_t)old[m][nn]) : 0u;
        omax = max(omax, (int32_t)old[m][nn]);
      }
    const bool clamped = omax >= K::CAP;  // some old value's key is the clamp
    for (int ch = 0; ch < C::NC; ++ch) {
      const unsigned st = pc.chunk & 1;
      const long long w0 = tr ? clock64() : 0;
      if (!mbar_wait(&wb->chunk_full[st], (pc.chunk >> 1) & 1, c.status, c.abort_flag,
                     c.timeout_ns))
        return false;
      if (tr) cw += clock64() - w0;
      const uint32_t* As = reinterpret_cast<const uint32_t*>(ring + st * L::kStage);
      const uint32_t* Bs = As + C::CK * BS;
      core_packed<BS, C::CK>(As, Bs, acc, tx, ty);
      __syncwarp();
      if (lane == 0) mbar_arrive(&wb->chunk_empty[st]);
      ++pc.chunk;
    }
    const long long t_c = tr ? clock64() : 0;
    if (tr) {
      tr[7] = cyc20(t_b - t_a) | (cyc20(cw) << 20);
      tr[8] = (uint64_t)(t_c - t_a);
    }
    // predecessors as "via k" codes: k = r*BS + code - 1
    const int32_t via0 = via_code((int64_t)c.r * BS - 1);  // via_code(k) = via0 - code
    // most tasks of later rounds improve nothing in a warp's 16 x 128 rows:
    // one OR over the codes and a vote skip the epilogue
    uint32_t any = 0;
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) any |= acc[m][nn];
    if (__any_sync(0xffffffffu, (any & K::MASK) != 0)) {
      if (full && !__any_sync(0xffffffffu, clamped)) {
        // no clamped key in the warp: every key decodes exactly; a group of
        // G entries with an improvement is stored as one 16-byte vector
#pragma unroll
        for (int m = 0; m < TM; ++m) {
          const int lr = Gm::idx(ty, m);
#pragma unroll
          for (int g = 0; g < Gm::NG; ++g) {
            const int lc0 = g * Gm::SPAN + tx * G;
            uint32_t cg = 0;
            T dv[G];
#pragma unroll
            for (int e = 0; e < G; ++e) {
              const uint32_t kv = acc[m][g * G + e];
              cg |= kv & K::MASK;
              dv[e] = (T)(int32_t)(kv >> K::KB);
            }
            if (cg) vstore<G>(Drow + lr * c.ld + lc0, dv);
            if (c.P) {
#pragma unroll
              for (int e = 0; e < G; ++e) {
                const int code = (int)(acc[m][g * G + e] & K::MASK);
                if (code) Prow[lr * c.ld + lc0 + e] = via0 - code;
              }
            }
          }
        }
      } else {
        // improved entries one by one (a clamped key -- old value CAP or
        // more, INF or a large finite one -- keeps its old value)
#pragma unroll
        for (int m = 0; m < TM; ++m) {
          const int lr = Gm::idx(ty, m);
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            const int code = (int)(acc[m][nn] & K::MASK);
            const int lc = Gm::idx(tx, nn);
            if (code && lr < nrow && lc < ncol) {
              Drow[lr * c.ld + lc] = (T)(int32_t)(acc[m][nn] >> K::KB);
              if (c.P) Prow[lr * c.ld + lc] = via0 - code;
            }
          }
        }
      }
    }
  } else {
    int arg[TM][TM];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) arg[m][nn] = 0;
    for (int ch = 0; ch < C::NC; ++ch) {
      const unsigned st = pc.chunk & 1;
      const long long w0 = tr ? clock64() : 0;
      if (!mbar_wait(&wb->chunk_full[st], (pc.chunk >> 1) & 1, c.status, c.abort_flag,
                     c.timeout_ns))
        return false;
      if (tr) cw += clock64() - w0;
      decode_chunk<T, BS, C::CK>(ring + st * L::kStage, dec);
      const T* As = reinterpret_cast<const T*>(ring + st * L::kStage);
      const T* Bs = As + C::CK * BS;
      core_generic<BS, T, C::CK, false>(As, Bs, old, arg, tx, ty, ch * C::CK);
      __syncwarp();
      if (lane == 0) mbar_arrive(&wb->chunk_empty[st]);
      ++pc.chunk;
    }
    argmin_finish<T>(arg);
    const long long t_c = tr ? clock64() : 0;
    if constexpr (!ViaPred<T>::kOn) {
      // (this branch always has predecessors)
      if (!mbar_wait(&wb->p_full, pc.p & 1, c.status, c.abort_flag, c.timeout_ns)) return false;
    }
    if (tr) {
      tr[7] = cyc20(t_b - t_a) | (cyc20(cw) << 20) | (cyc20(clock64() - t_c) << 40);
      tr[8] = (uint64_t)(t_c - t_a);
    }
    const int32_t via0 = via_code((int64_t)c.r * BS - 1);
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      const int lr = Gm::idx(ty, m);
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const int lc = Gm::idx(tx, nn);
        if (arg[m][nn] && lr < nrow && lc < ncol) {
          Drow[lr * c.ld + lc] = old[m][nn];
          Prow[lr * c.ld + lc] =
              ViaPred<T>::kOn ? via0 - arg[m][nn] : Pbuf[(arg[m][nn] - 1) * BS + lc];
          neg |= (row0 + lr == col0 + lc) && old[m][nn] < T(0);
        }
      }
    }
  }
  if (tr) tr[8] |= (uint64_t)(clock64() - t_a) << 32;  // whole task
  if constexpr (!ViaPred<T>::kOn) {
    if (c.P) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&wb->p_empty);
      ++pc.p;
    }
  }
  if (neg) atomicOr(c.status, kStNegCycle);
  return true;
}

// Relaxation and epilogue of a producer-fed panel task (ws_panel) whose
// operands are staged: packed keys (kFast) or raw values, A transposed in the
// scratch stage, B in natural layout (Dbuf for a row tile, the pivot stage
// for a column tile).  The accumulators start from the tile's own values as
// staged there.  A function of its own per path, so that the two register
// sets are never live together.
template <typename T, int BS, int LBS, bool is_row, bool kFast>
__device__ __noinline__ bool ws_panel_finish(const Args<T>& a, int r, int t, T* Dbuf, T* Piv,
                                             unsigned char* scratch, WsBars* wb, CtaScratch* cs,
                                             PipeCnt& pc) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  using U = std::conditional_t<kFast, uint32_t, T>;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31;
  const U* As = reinterpret_cast<const U*>(scratch);
  const U* Bs = reinterpret_cast<const U*>(is_row ? Dbuf : Piv);
  U acc[TM][TM];
  if constexpr (is_row) {
    // own values: B-form in Dbuf
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        U v[G];
        vload_s<G>(v, Bs + Gm::idx(ty, m) * BS + g * Gm::SPAN + tx * G);
#pragma unroll
        for (int e = 0; e < G; ++e) acc[m][g * G + e] = v[e];
      }
  } else {
    // own values: A-form in the scratch stage (keys with their column's code)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn)
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        U v[G];
        vload_s<G>(v, As + Gm::idx(tx, nn) * BS + g * Gm::SPAN + ty * G);
#pragma unroll
        for (int e = 0; e < G; ++e) {
          if constexpr (kFast) acc[g * G + e][nn] = v[e] & ~K::MASK;
          else acc[g * G + e][nn] = v[e];
        }
      }
  }
  int code[kFast ? 1 : TM][kFast ? 1 : TM];
  if constexpr (kFast) {
    core_packed<BS>(As, Bs, acc, tx, ty);
  } else {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) code[m][nn] = 0;
    core_generic<BS, T>(As, Bs, acc, code, tx, ty);
  }
  // operands consumed: order this warp's shared-memory writes before the
  // copies that will overwrite the buffers, then release them
  fence_proxy_async_shared();
  __syncwarp();
  if (lane == 0) {
    const unsigned s0 = pc.chunk & 1;
    mbar_arrive(&wb->d_empty);
    mbar_arrive(&wb->chunk_empty[s0]);
    mbar_arrive(&wb->chunk_empty[s0 ^ 1]);
  }
  ++pc.d;
  pc.chunk += 2;
  stamp(2);

  // new values: their bound (the remaining tiles' packed-key test)
  auto value = [&](int m, int nn) -> T {
    if constexpr (kFast) {
      const int32_t v = (int32_t)(acc[m][nn] >> K::KB);
      return v == K::CAP ? Num<T>::inf() : (T)v;
    } else {
      return acc[m][nn];
    }
  };
  auto codeof = [&](int m, int nn) -> int {
    if constexpr (kFast) return (int)(acc[m][nn] & K::MASK);
    else return code[m][nn];
  };
  // (fast path: the accumulator without its code is the value's key)
  auto key = [&](int m, int nn) -> uint32_t {
    if constexpr (kFast) return acc[m][nn] & ~K::MASK;
    else return key_of<BS>((int32_t)acc[m][nn]);
  };
  int nb = 0;
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) nb = max(nb, bound_of<BS>(value(m, nn)));
  int dummy = 0;
  block_max2(nb, dummy, cs);
  // keys are exact while every finite value is below CAP; otherwise (or
  // without packed keys) the raw snapshot is written as well
  const bool keys = a.packed != 0;
  const bool raw = !keys || nb >= K::CAP;
  const int slot = r & 1;
  const size_t tile_off = ((size_t)slot * a.slot_tiles + t) * BS * BS;
  // the pointers and sizes in registers: through the reference every access
  // would be a load, repeated after each store (which might alias it)
  T* const D = a.D;
  int32_t* const P = a.P;
  const int64_t n = a.n, ld = a.ld;
  uint32_t* const snapK = (is_row ? a.rowK : a.colK) + tile_off;
  T* const snapR = (is_row ? a.rowR : a.colR) + tile_off;
  int32_t* const bnd = (is_row ? a.rowB : a.colB) + (size_t)slot * a.slot_tiles + t;

  // the live tile (values, and via codes k = r*BS + code - 1 where improved);
  // a row tile's snapshots in the same (B-form) order
  const int32_t via0 = via_code((int64_t)r * BS - 1);
  const int ti = is_row ? r : t, tj = is_row ? t : r;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int lr = Gm::idx(ty, m);
    const int64_t gi = (int64_t)ti * BS + lr;
#pragma unroll
    for (int gg = 0; gg < Gm::NG; ++gg) {
      const int lc0 = gg * Gm::SPAN + tx * G;
      const int64_t gj0 = (int64_t)tj * BS + lc0;
      T vs[G];
      int32_t vp[G];
      bool all = true;
      int cq[G];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        vs[q] = value(m, gg * G + q);
        cq[q] = codeof(m, gg * G + q);
        vp[q] = via0 - cq[q];
        all &= cq[q] != 0;
      }
      if (gi < n) {
        if (gj0 + G <= n) {
          vstore<G>(D + gi * ld + gj0, vs);
          if (P) {
            if (all) {
              vstore<G>(P + gi * ld + gj0, vp);  // (early rounds: most groups)
            } else {
#pragma unroll
              for (int q = 0; q < G; ++q)
                if (cq[q]) P[gi * ld + gj0 + q] = vp[q];
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < G; ++q)
            if (gj0 + q < n) {
              D[gi * ld + gj0 + q] = vs[q];
              if (P && cq[q]) P[gi * ld + gj0 + q] = vp[q];
            }
        }
      }
      if constexpr (is_row) {
        if (keys) {
          uint32_t kq[G];
#pragma unroll
          for (int q = 0; q < G; ++q) kq[q] = key(m, gg * G + q);
          vstore<G>(snapK + lr * BS + lc0, kq);
        }
        if (raw) vstore<G>(snapR + lr * BS + lc0, vs);
      }
    }
  }
  if constexpr (!is_row) {
    // a column tile's snapshots: A-form (transposed), keys with code = column + 1
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) {
      const int lc = Gm::idx(tx, nn);
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        const size_t off = (size_t)lc * BS + g * Gm::SPAN + ty * G;
        if (keys) {
          uint32_t kq[G];
#pragma unroll
          for (int e = 0; e < G; ++e) kq[e] = key(g * G + e, nn) + (uint32_t)lc + 1u;
          vstore<G>(snapK + off, kq);
        }
        if (raw) {
          T vs[G];
#pragma unroll
          for (int e = 0; e < G; ++e) vs[e] = value(g * G + e, nn);
          vstore<G>(snapR + off, vs);
        }
      }
    }
  }
  if (tid == 0) *bnd = nb;
  stamp(3);
  return true;
}

// Panel task of round r (int32), fed by the producer like a remaining tile:
// Dbuf holds the tile's own values, ring stage s0 the closed pivot (snapshot
// of slot r&1, natural layout) and stage s1 is scratch for the transposed A
// operand.  Row tile (r, t):    A = pivot (transposed), B = own old values.
// Column tile (t, r): A = own old values (transposed), B = pivot.
// The product with the closed pivot equals the in-place sequential phases 2
// and 3 (Sec. 2.3).  Predecessors are recorded as via codes (ViaPred), so the
// task needs no predecessor tile.  The operand buffers are released right
// after the relaxation: the producer streams the next task's operands while
// this one stores its results.
template <typename T, int BS, int LBS, bool is_row>
__device__ __noinline__ bool ws_panel(const Args<T>& a, const fwh::Task& k, unsigned char* smem,
                                      WsBars* wb, CtaScratch* cs, PipeCnt& pc) {
  static_assert(Num<T>::kPacked, "producer-fed panels are the int32 path");
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  using L = WsLayout<LBS, T>;
  static_assert(WsChunk<BS, T>::kTile <= L::kStage, "a tile per ring stage");
  constexpr int TM = Gm::TM, G = Gm::G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r = k.r, t = is_row ? k.tj : k.ti;
  const int64_t row0 = (int64_t)k.ti * BS, col0 = (int64_t)k.tj * BS;
  const int nrow = (int)(a.n - row0 < BS ? a.n - row0 : BS);
  const int ncol = (int)(a.n - col0 < BS ? a.n - col0 : BS);
  T* Dbuf = reinterpret_cast<T*>(smem + L::d_off());
  const unsigned s0 = pc.chunk & 1, s1 = s0 ^ 1;
  T* Piv = reinterpret_cast<T*>(smem + L::ring_off() + s0 * L::kStage);
  unsigned char* scratch = smem + L::ring_off() + s1 * L::kStage;
  stamp(0);
  if (!mbar_wait(&wb->d_full, pc.d & 1, a.status, a.abort_flag, a.timeout_ns) ||
      !mbar_wait(&wb->chunk_full[s0], (pc.chunk >> 1) & 1, a.status, a.abort_flag,
                 a.timeout_ns) ||
      !mbar_wait(&wb->chunk_full[s1], ((pc.chunk + 1) >> 1) & 1, a.status, a.abort_flag,
                 a.timeout_ns))
    return false;

  // micro-tiles of the tile (entries beyond n read as INF) and of the pivot
  T s[TM][TM], pv[TM][TM];
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int lr = Gm::idx(ty, m);
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      const int lc0 = g * Gm::SPAN + tx * G;
      T ts[G], tp[G];
      vload_s<G>(ts, Dbuf + lr * BS + lc0);
      vload_s<G>(tp, Piv + lr * BS + lc0);
#pragma unroll
      for (int e = 0; e < G; ++e) {
        s[m][g * G + e] = (lr < nrow && lc0 + e < ncol) ? ts[e] : Num<T>::inf();
        pv[m][g * G + e] = tp[e];
      }
    }
  }
  int bs_ = 0, bp_ = 0;
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) {
      bs_ = max(bs_, bound_of<BS>(s[m][nn]));
      bp_ = max(bp_, bound_of<BS>(pv[m][nn]));
    }
  block_max2(bs_, bp_, cs);  // (its barriers also end every read of the raw buffers)
  const bool fast = a.packed && (bs_ + bp_ < K::CAP);

  // operands: A (transposed) into the scratch stage, B in place (natural
  // layout: the own tile in Dbuf for a row tile, the pivot for a column
  // tile).  Keys are formed in the registers of s and pv (int32), so that the
  // accumulators are only loaded once those are dead.
  uint32_t* Bk = reinterpret_cast<uint32_t*>(is_row ? (void*)Dbuf : (void*)Piv);
  if (fast) {
    uint32_t (&ka)[TM][TM] = reinterpret_cast<uint32_t(&)[TM][TM]>(is_row ? pv : s);
    uint32_t (&kb)[TM][TM] = reinterpret_cast<uint32_t(&)[TM][TM]>(is_row ? s : pv);
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const uint32_t cc = (uint32_t)Gm::idx(tx, nn) + 1u;  // the A entry's kk + 1
        ka[m][nn] = key_of<BS>((int32_t)ka[m][nn]) + cc;
        kb[m][nn] = key_of<BS>((int32_t)kb[m][nn]);
      }
    put_tile<BS, true>(reinterpret_cast<uint32_t*>(scratch), ka, tx, ty);
    put_tile<BS, false>(Bk, kb, tx, ty);
  } else {
    if constexpr (is_row) {
      put_tile<BS, true>(reinterpret_cast<T*>(scratch), pv, tx, ty);
      put_tile<BS, false>(Dbuf, s, tx, ty);  // (entries beyond n as INF)
    } else {
      put_tile<BS, true>(reinterpret_cast<T*>(scratch), s, tx, ty);
    }
  }
  bar_compute();
  stamp(1);
  return fast ? ws_panel_finish<T, BS, LBS, is_row, true>(a, r, t, Dbuf, Piv, scratch, wb, cs, pc)
              : ws_panel_finish<T, BS, LBS, is_row, false>(a, r, t, Dbuf, Piv, scratch, wb, cs,
                                                           pc);
}

// Any task, compute-warp side.
template <typename T, int BS, int LBS>
__device__ bool compute_task(const Args<T>& a, const fwh::Task& k, bool fast, int dec,
                             unsigned char* smem, WsBars* wb, CtaScratch* cs, PipeCnt& pc,
                             uint64_t* tr) {
  using L = WsLayout<LBS, T>;
  if (k.type == 3 || k.type == kFusedTask) {
    const TileCtx<T> ctx{a.D, a.P, a.n, a.ld, k.r, a.status, a.abort_flag, a.timeout_ns};
    const bool ok = ws_minplus<T, BS, LBS>(ctx, k.ti, k.tj, fast, dec, smem, wb, pc, tr);
    if (!ok || k.type == 3) return ok;
    // fused: the tile's stores precede the pivot's loads of it (same CTA),
    // and every warp has left the tile's operand buffers before the pivot
    // reuses them
    bar_compute();
    task_pivot<T, BS>(a, k.r + 1, smem + L::ring_off(), cs);
    bar_compute();
    return true;
  }
  if constexpr (Num<T>::kPacked) {
    if (k.type != 0) {
      const bool ok = k.type == 1 ? ws_panel<T, BS, LBS, true>(a, k, smem, wb, cs, pc)
                                  : ws_panel<T, BS, LBS, false>(a, k, smem, wb, cs, pc);
      if (ok && tr) {
        const long long t0 = t_stamp[0], t_end = clock64();
        tr[7] = (uint64_t)(t_stamp[1] - t0) | ((uint64_t)(t_stamp[2] - t0) << 32);
        tr[8] = (uint64_t)(t_stamp[3] - t0) | ((uint64_t)(t_end - t0) << 32);
      }
      return ok;
    }
  }
  // Pivot (and, for the other types, panel) tasks overwrite the ring and Dbuf
  // from their first instructions: every compute warp must have left the
  // previous task (a slow warp may still be reading its last operand chunk)
  // before any warp starts.
  bar_compute();
  if (k.type == 0) {
    task_pivot<T, BS>(a, k.r, smem + L::ring_off(), cs);
  } else {
    task_panel<T, BS>(a, k.r, k.type == 1 ? k.tj : k.ti, k.type == 1, smem + L::ring_off(), cs);
  }
  bar_compute();
  if (tr) {
    // pivot: loads | steps ; predecessors resolved | end.  panel: operands
    // staged | relaxed ; stored | end (SM cycles from the task's start)
    const long long t0 = t_stamp[0], t_end = clock64();
    tr[7] = (uint64_t)(t_stamp[1] - t0) | ((uint64_t)(t_stamp[2] - t0) << 32);
    tr[8] = (uint64_t)(t_stamp[3] - t0) | ((uint64_t)(t_end - t0) << 32);
  }
  return true;
}

// ----------------------------------------------------------- producer side ----

// Bounded wait until *p >= target (producer lane only).  Gives up when another
// CTA has aborted or when the wait exceeds timeout_ns; then records the
// timeout and raises the abort flag so that every CTA stops.
__device__ __forceinline__ bool wait_ge(const int* p, int target, int* abort_flag, int* status,
                                        int64_t timeout_ns) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = globaltimer();
  // iteration cap as well as the clock: each iteration sleeps >= 32 ns
  const int64_t max_it = timeout_ns / 32 + 1024;
  // sleeps back off to 64 ns at most: a flag is polled soon after it is
  // published (n = 1024 at BS = 32: 0.610 -> 0.606 ms against 256 ns; the
  // large solves and the batched workload unchanged)
  unsigned ns = 32;
  for (int64_t it = 0;; ++it) {
    __nanosleep(ns);
    if (ns < 64) ns <<= 1;
    if (ld_acquire(p) >= target) return true;
    if (ld_relaxed(abort_flag)) return false;
    if (globaltimer() - t0 > (uint64_t)timeout_ns || it > max_it) {
      atomicOr(status, kStTimeout);
      atomicExch(abort_flag, 1);
      return false;
    }
  }
}

// Inputs of task k (Sec. 2.3 blocked-FW phase order, Opt-9's per-block dependencies of
// Sec. 3.2, and the slot reuse of the double-buffered snapshots): dependency
// `lane` (0..2) as a counter and the value it must reach; false when the task
// has fewer.
template <typename T>
__device__ __forceinline__ bool dep_of(const Args<T>& a, const fwh::Task& k, int lane,
                                       const int*& p, int& target) {
  const int R = a.R;
  const int* ver = a.ver;
  // Slot reuse is guarded by per-round counts: tasks of different rounds may
  // finish out of order, so a running total could reach its target while a
  // task of round r-2 still reads the slot.
  switch (k.type) {
    case 0:  // pivot: its tile after round r-1; pivot slot free (all panels of r-2 done)
      if (lane == 0) { p = ver + (size_t)k.r * R + k.r; target = k.r; return true; }
      if (lane == 1 && k.r >= 2) { p = a.done + (k.r - 2); target = 2 * (R - 1); return true; }
      return false;
    case 1:
    case 2:  // panel: its tile after round r-1, the pivot of r, snapshot slot free
      if (lane == 0) { p = ver + (size_t)k.ti * R + k.tj; target = k.r; return true; }
      if (lane == 1) { p = ver + (size_t)k.r * R + k.r; target = k.r + 1; return true; }
      if (lane == 2 && k.r >= 2) {
        p = a.done + R + (k.r - 2);
        target = (R - 1) * (R - 1);
        return true;
      }
      return false;
    default:  // remaining tile: itself after r-1, both panels of round r
      if (lane == 0) { p = ver + (size_t)k.ti * R + k.tj; target = k.r; return true; }
      if (lane == 1) { p = ver + (size_t)k.ti * R + k.r; target = k.r + 1; return true; }
      if (lane == 2) { p = ver + (size_t)k.r * R + k.tj; target = k.r + 1; return true; }
      // tile (r+1, r+1) fused with the pivot of round r+1: that pivot's
      // snapshot slot is free once every panel of round r-1 is done
      if (lane == 3 && k.type == kFusedTask && k.r >= 1) {
        p = a.done + (k.r - 1);
        target = 2 * (R - 1);
        return true;
      }
      return false;
  }
}

// Wait (bounded) until every input of task k exists: lane i of the producer
// warp acquires dependency i, so the waits overlap; the warp barrier then
// orders those acquires before the copies lane 0 issues.  Whole warp.
template <typename T>
__device__ bool wait_deps(const Args<T>& a, const fwh::Task& k, int lane) {
  const int* p = nullptr;
  int target = 0;
  bool ok = true;
  if (lane < 4 && dep_of(a, k, lane, p, target))
    ok = wait_ge(p, target, a.abort_flag, a.status, a.timeout_ns);
  return __all_sync(0xffffffffu, ok);
}

// Completion of task k: the tile's version, and the per-phase counters that
// guard snapshot slot reuse.  Release semantics make every store of the task
// (made by the compute warps and ordered before this thread through the
// task_done mbarrier) visible to whoever acquires the flag.
template <typename T>
__device__ __forceinline__ void publish(const Args<T>& a, const fwh::Task& k) {
  // (a fused task publishes its tile after round r+1's pivot: version r+2)
  st_release(a.ver + (size_t)k.ti * a.R + k.tj, k.type == kFusedTask ? k.r + 2 : k.r + 1);
  if (k.type == 1 || k.type == 2) red_release_add(reinterpret_cast<unsigned*>(a.done + k.r), 1u);
  if (k.type == 3 || k.type == kFusedTask)
    red_release_add(reinterpret_cast<unsigned*>(a.done + a.R + k.r), 1u);
}

// Whether a remaining-tile task may relax packed keys (int32, bounded panels).
template <typename T, int BS>
__device__ __forceinline__ bool packed_ok(const Args<T>& a, const fwh::Task& k) {
  if (!(Num<T>::kPacked && a.packed && (k.type == 3 || k.type == kFusedTask))) return false;
  const int slot = k.r & 1;
  const int ba = __ldcg(a.colB + (size_t)slot * a.slot_tiles + k.ti);
  const int bb = __ldcg(a.rowB + (size_t)slot * a.slot_tiles + k.tj);
  return ba + bb < Keys<BS>::CAP;
}

// Copy the tile (k.ti, k.tj) of D into Dbuf (whole producer warp): one 2-D
// tensor copy, or one bulk copy per valid row.
template <typename T, int BS, int LBS>
__device__ __forceinline__ void issue_tile_load(const Args<T>& a, const fwh::Task& k,
                                                unsigned char* smem, WsBars* wb, PipeCnt& pc,
                                                int lane) {
  using L = WsLayout<LBS, T>;
  // the tile's own D block, one bulk copy per valid row
  const int64_t row0 = (int64_t)k.ti * BS, col0 = (int64_t)k.tj * BS;
  const int nrows = (int)(a.n - row0 < (int64_t)BS ? a.n - row0 : (int64_t)BS);
  const int ncols = (int)(a.n - col0 < (int64_t)BS ? a.n - col0 : (int64_t)BS);
  // whole 16-byte granules (rows are 16-byte aligned and ld % 4 == 0, so the
  // rounded row stays inside the caller's row)
  const unsigned rowbytes = (unsigned)(((size_t)ncols * sizeof(T) + 15) / 16 * 16);
  unsigned char* dbuf = smem + L::d_off();
  if (a.tmapD) {
    // one tensor copy of the whole box (elements beyond n arrive as zeros and
    // are masked by the compute warps); a single instruction keeps the
    // producer's issue slots, shared with two compute warps, free
    if (lane == 0) {
      if (!pc.stop && mbar_wait(&wb->d_empty, (pc.d & 1) ^ 1, a.status, a.abort_flag, a.timeout_ns)) {
        mbar_expect_tx(&wb->d_full, (unsigned)(BS * BS * sizeof(T)));
        tma_load_2d(dbuf, a.tmapD, (int)col0, (int)row0, &wb->d_full);
        pc.d_armed = pc.d + 1;
      } else {
        pc.stop = true;
      }
    }
  } else {
    bool ok = false;
    if (lane == 0) {
      ok = !pc.stop && mbar_wait(&wb->d_empty, (pc.d & 1) ^ 1, a.status, a.abort_flag, a.timeout_ns);
      if (ok) {
        mbar_expect_tx(&wb->d_full, rowbytes * (unsigned)nrows);
        pc.d_armed = pc.d + 1;
      } else {
        pc.stop = true;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok)
      for (int rr = lane; rr < nrows; rr += 32)
        bulk_g2s(dbuf + (size_t)rr * BS * sizeof(T), a.D + (row0 + rr) * a.ld + col0, rowbytes,
                 &wb->d_full);
  }
  ++pc.d;
}

// Operand forms of a compare-and-select remaining tile (int32): the panel
// snapshots it reads as keys (bit 0: A, bit 1: B) because their panels wrote
// the exact keys only (bound below CAP, packed keys in use).
template <typename T, int BS>
__device__ __forceinline__ int key_operands(const Args<T>& a, const fwh::Task& k, bool fast) {
  if (!(Num<T>::kPacked && a.packed && (k.type == 3 || k.type == kFusedTask)) || fast) return 0;
  const int slot = k.r & 1;
  const int ba = __ldcg(a.colB + (size_t)slot * a.slot_tiles + k.ti);
  const int bb = __ldcg(a.rowB + (size_t)slot * a.slot_tiles + k.tj);
  return (ba < Keys<BS>::CAP ? 1 : 0) | (bb < Keys<BS>::CAP ? 2 : 0);
}

// Issue the operand copies of remaining-tile task k (whole producer warp).
template <typename T, int BS, int LBS>
__device__ void issue_operands(const Args<T>& a, const fwh::Task& k, bool fast, int dec,
                               unsigned char* smem, WsBars* wb, PipeCnt& pc, int lane) {
  using L = WsLayout<LBS, T>;
  using C = WsChunk<BS, T>;
  fence_proxy_async();  // global data published by other CTAs, read by TMA below
  const int slot = k.r & 1;
  issue_tile_load<T, BS, LBS>(a, k, smem, wb, pc, lane);
  // operand chunks
  const size_t toffA = ((size_t)slot * a.slot_tiles + k.ti) * BS * BS;
  const size_t toffB = ((size_t)slot * a.slot_tiles + k.tj) * BS * BS;
  const unsigned char* srcA = (fast || (dec & 1)) ? (const unsigned char*)(a.colK + toffA)
                                                 : (const unsigned char*)(a.colR + toffA);
  const unsigned char* srcB = (fast || (dec & 2)) ? (const unsigned char*)(a.rowK + toffB)
                                                 : (const unsigned char*)(a.rowR + toffB);
  for (int c = 0; c < C::NC; ++c) {
    if (lane == 0) {
      const unsigned st = pc.chunk & 1;
      if (!pc.stop && mbar_wait(&wb->chunk_empty[st], ((pc.chunk >> 1) & 1) ^ 1, a.status,
                                a.abort_flag, a.timeout_ns)) {
        mbar_expect_tx(&wb->chunk_full[st], 2 * (unsigned)C::kChunkBytes);
        unsigned char* dst = smem + L::ring_off() + st * L::kStage;
        bulk_g2s(dst, srcA + c * C::kChunkBytes, (unsigned)C::kChunkBytes, &wb->chunk_full[st]);
        bulk_g2s(dst + C::kChunkBytes, srcB + c * C::kChunkBytes, (unsigned)C::kChunkBytes,
                 &wb->chunk_full[st]);
        pc.chunk_armed[st] = pc.chunk + 1;
      } else {
        pc.stop = true;
      }
    }
    ++pc.chunk;
  }
  // predecessor tile of the row panel snapshot (fp32; int32 records "via" codes)
  if (!ViaPred<T>::kOn && a.P) {
    if (lane == 0) {
      if (!pc.stop && mbar_wait(&wb->p_empty, (pc.p & 1) ^ 1, a.status, a.abort_flag, a.timeout_ns)) {
        mbar_expect_tx(&wb->p_full, (unsigned)C::kPTile);
        bulk_g2s(smem + L::p_off(), a.rowP + toffB, (unsigned)C::kPTile, &wb->p_full);
        pc.p_armed = pc.p + 1;
      } else {
        pc.stop = true;
      }
    }
    ++pc.p;
  }
}

// Issue the operands of panel task k (int32, whole producer warp): the tile
// into Dbuf, the closed pivot of round k.r into the next ring stage, and the
// stage after it handed over empty as the task's scratch (ws_panel).
template <typename T, int BS, int LBS>
__device__ void issue_panel_operands(const Args<T>& a, const fwh::Task& k, unsigned char* smem,
                                     WsBars* wb, PipeCnt& pc, int lane) {
  using L = WsLayout<LBS, T>;
  using C = WsChunk<BS, T>;
  fence_proxy_async();  // global data published by other CTAs, read by TMA below
  issue_tile_load<T, BS, LBS>(a, k, smem, wb, pc, lane);
  if (lane == 0) {
    const unsigned st = pc.chunk & 1;
    if (!pc.stop && mbar_wait(&wb->chunk_empty[st], ((pc.chunk >> 1) & 1) ^ 1, a.status,
                              a.abort_flag, a.timeout_ns)) {
      mbar_expect_tx(&wb->chunk_full[st], (unsigned)C::kTile);
      bulk_g2s(smem + L::ring_off() + st * L::kStage, a.piv + (size_t)(k.r & 1) * BS * BS,
               (unsigned)C::kTile, &wb->chunk_full[st]);
      pc.chunk_armed[st] = pc.chunk + 1;
    } else {
      pc.stop = true;
    }
    const unsigned st1 = (pc.chunk + 1) & 1;
    if (!pc.stop && mbar_wait(&wb->chunk_empty[st1], (((pc.chunk + 1) >> 1) & 1) ^ 1, a.status,
                              a.abort_flag, a.timeout_ns)) {
      mbar_arrive(&wb->chunk_full[st1]);  // no copy: the stage is scratch
      // (recorded all the same: the final drain waits on the latest phase of
      // each barrier, and a parity wait on an older one would never succeed
      // once the barrier is two phases further)
      pc.chunk_armed[st1] = pc.chunk + 2;
    } else {
      pc.stop = true;
    }
  }
  pc.chunk += 2;
}

// Optional per-task trace (sampled tasks): 10 words per entry.
//   [0] task | type << 32 | graph << 40   [1] SM id
//   producer: [2] claimed  [3] inputs ready  [4] copies issued  [5] published
//   compute : [6] descriptor seen  [9] task finished (stores issued)
//   min-plus tasks: [7], [8] SM-cycle counts of the task's phases
__device__ __forceinline__ uint64_t* trace_slot(uint64_t* tr, int cap, int stride, int64_t t) {
  if (!tr || t < 0 || stride <= 0 || t % stride) return nullptr;
  const int64_t s = t / stride;
  return s < cap ? tr + (size_t)s * 10 : nullptr;
}
__device__ __forceinline__ unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// Runs f(std::integral_constant<int, BS>) for the block size of the task.
// kFixedBS > 0: that block size only (single-graph kernels).
template <int kFixedBS, int LBS, typename F>
__device__ __forceinline__ auto with_bs(int bs, F&& f) {
  if constexpr (kFixedBS > 0) {
    return f(std::integral_constant<int, kFixedBS>{});
  } else {
    if (bs == 32) return f(std::integral_constant<int, 32>{});
    if constexpr (LBS >= 64)
      if (bs == 64) return f(std::integral_constant<int, 64>{});
    return f(std::integral_constant<int, LBS>{});
  }
}

// ------------------------------------------------------------------ engine ----

// Src supplies: total(), next (claim counter), status / abort / timeout, trace,
// resolve(t, &g) -> local task, args(g) -> const Args<T>&, bs(g).
template <typename T, int kFixedBS, int LBS, class Src>
__device__ void ws_engine(const Src& src, unsigned char* smem, WsBars& wb, CtaScratch& cs) {
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&wb.desc_full[i], 1);
      mbar_init(&wb.desc_empty[i], kThreads / 32);
      mbar_init(&wb.chunk_full[i], 1);
      mbar_init(&wb.chunk_empty[i], kThreads / 32);
    }
    mbar_init(&wb.d_full, 1);
    mbar_init(&wb.d_empty, kThreads / 32);
    mbar_init(&wb.p_full, 1);
    mbar_init(&wb.p_empty, kThreads / 32);
    mbar_init(&wb.task_done, kThreads / 32);
    for (int i = 0; i < kPubDepth; ++i) {
      mbar_init(&wb.pub_full[i], 1);
      mbar_init(&wb.pub_empty[i], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kThreads / 32 + 1) {
    // ----------------------------------------------------------- publisher
    if (lane == 0) {
      for (unsigned i = 0;; ++i) {
        const unsigned q = i % kPubDepth, ph = (i / kPubDepth) & 1;
        if (!mbar_wait(&wb.pub_full[q], ph, src.status, src.abort_flag, src.timeout_ns)) break;
        const int t = wb.pubq[q][0];
        const fwh::Task k{wb.pubq[q][1], wb.pubq[q][2], wb.pubq[q][3], wb.pubq[q][4]};
        const int g = wb.pubq[q][5];
        if (t < 0) break;
        // tasks finish in hand-off order: the i-th completion is this task
        if (!mbar_wait(&wb.task_done, i & 1, src.status, src.abort_flag, src.timeout_ns)) break;
        if (t != src.skip_task) publish(src.args(g), k);
        if (uint64_t* tr = trace_slot(src.trace, src.trace_cap, src.trace_stride, t))
          tr[5] = globaltimer();
        mbar_arrive(&wb.pub_empty[q]);
      }
    }
    return;
  }

  if (warp == kThreads / 32) {
    // ------------------------------------------------------------ producer
    const int64_t total = src.total();
    unsigned idesc = 0, ipub = 0;
    PipeCnt pc;
    for (;;) {
      int t = -1, g = 0;
      uint64_t t_claim = 0;
      if (lane == 0) {
        t_claim = globaltimer();
        const int64_t tt = atomicAdd(src.next, 1u);
        if (tt < total && !ld_relaxed(src.abort_flag)) t = (int)tt;
      }
      // lane 0 decodes the task; the others take it by shuffle
      fwh::Task k{0, 0, 0, 0};
      if (lane == 0 && t >= 0) k = src.resolve(t, g);
      t = __shfl_sync(0xffffffffu, t, 0);
      g = __shfl_sync(0xffffffffu, g, 0);
      k.type = __shfl_sync(0xffffffffu, k.type, 0);
      k.r = __shfl_sync(0xffffffffu, k.r, 0);
      k.ti = __shfl_sync(0xffffffffu, k.ti, 0);
      k.tj = __shfl_sync(0xffffffffu, k.tj, 0);
      if (t >= 0) {
        // tile (r+1, r+1) of round r takes the pivot of round r+1 along, and
        // that pivot's own queue entry is skipped
        if (k.type == 0 && k.r >= 1) continue;
        if (k.type == 3 && k.ti == k.r + 1 && k.tj == k.r + 1) k.type = kFusedTask;
        if (!wait_deps(src.args(g), k, lane)) t = -1;
      }
      if (lane == 0) {
        if (uint64_t* tr = trace_slot(src.trace, src.trace_cap, src.trace_stride, t)) {
          tr[1] = smid();
          tr[2] = t_claim;
          tr[3] = globaltimer();
        }
      }
      bool fast = false;
      int dec = 0;
      int bs = 0;
      if (t >= 0) {
        bs = src.bs(g);
        fast = with_bs<kFixedBS, LBS>(bs, [&](auto B) {
          return packed_ok<T, decltype(B)::value>(src.args(g), k);
        });
        dec = with_bs<kFixedBS, LBS>(bs, [&](auto B) {
          return key_operands<T, decltype(B)::value>(src.args(g), k, fast);
        });
      }
      unsigned pq = 0;
      if (lane == 0) {
        // queue the task for publication, then hand it to the compute warps
        pq = ipub % kPubDepth;
        mbar_wait(&wb.pub_empty[pq], ((ipub / kPubDepth) & 1) ^ 1, src.status, src.abort_flag,
                  src.timeout_ns);
        wb.pubq[pq][0] = t;
        wb.pubq[pq][1] = k.type;
        wb.pubq[pq][2] = k.r;
        wb.pubq[pq][3] = k.ti;
        wb.pubq[pq][4] = k.tj;
        wb.pubq[pq][5] = g;
        mbar_arrive(&wb.pub_full[pq]);
        const unsigned ds = idesc & 1;
        mbar_wait(&wb.desc_empty[ds], ((idesc >> 1) & 1) ^ 1, src.status, src.abort_flag,
                  src.timeout_ns);
        wb.desc[ds][0] = t;
        wb.desc[ds][1] = k.type;
        wb.desc[ds][2] = k.r;
        wb.desc[ds][3] = k.ti;
        wb.desc[ds][4] = k.tj;
        wb.desc[ds][5] = fast ? 1 : 0;
        wb.desc[ds][6] = g;
        wb.desc[ds][7] = dec;
        mbar_arrive(&wb.desc_full[ds]);
      }
      ++idesc;
      ++ipub;
      if (t < 0) break;
      if (k.type == 3 || k.type == kFusedTask) {
        with_bs<kFixedBS, LBS>(bs, [&](auto B) {
          issue_operands<T, decltype(B)::value, LBS>(src.args(g), k, fast, dec, smem, &wb, pc,
                                                     lane);
          return 0;
        });
        if (k.type == kFusedTask && lane == 0) {
          // its pivot uses the shared buffer as scratch: wait until the task
          // has been published (its publication-queue slot frees up)
          mbar_wait(&wb.pub_empty[pq], (((ipub - 1) / kPubDepth) & 1), src.status,
                    src.abort_flag, src.timeout_ns);
        }
      } else if (Num<T>::kPacked && k.type != 0) {
        with_bs<kFixedBS, LBS>(bs, [&](auto B) {
          issue_panel_operands<T, decltype(B)::value, LBS>(src.args(g), k, smem, &wb, pc, lane);
          return 0;
        });
      } else {
        if (lane == 0) {
          // pivot / panel tasks use the shared buffer as scratch: wait until
          // this task has been published (its publication-queue slot frees up)
          mbar_wait(&wb.pub_empty[pq], (((ipub - 1) / kPubDepth) & 1), src.status,
                    src.abort_flag, src.timeout_ns);
        }
      }
      if (lane == 0) {
        if (uint64_t* tr = trace_slot(src.trace, src.trace_cap, src.trace_stride, t)) {
          tr[0] = (uint64_t)(unsigned)t | ((uint64_t)k.type << 32) | ((uint64_t)(unsigned)g << 40);
          tr[4] = globaltimer();
        }
      }
      if (k.type == 0 || k.type == kFusedTask || (!Num<T>::kPacked && k.type != 3))
        fence_proxy_async();
      __syncwarp();
    }
    // leave no bulk copy in flight: wait (bounded, whatever the abort flag
    // says) for the last phase armed with a copy on every full barrier
    if (lane == 0) {
      if (pc.d_armed)
        mbar_wait(&wb.d_full, (pc.d_armed - 1) & 1, src.status, src.abort_flag, src.timeout_ns,
                  false);
      if (pc.p_armed)
        mbar_wait(&wb.p_full, (pc.p_armed - 1) & 1, src.status, src.abort_flag, src.timeout_ns,
                  false);
      for (int st = 0; st < 2; ++st)
        if (pc.chunk_armed[st])
          mbar_wait(&wb.chunk_full[st], ((pc.chunk_armed[st] - 1) >> 1) & 1, src.status,
                    src.abort_flag, src.timeout_ns, false);
    }
    return;
  }

  // -------------------------------------------------------------- compute
  unsigned idesc = 0;
  PipeCnt pc;
  for (;;) {
    const unsigned ds = idesc & 1;
    if (!mbar_wait(&wb.desc_full[ds], (idesc >> 1) & 1, src.status, src.abort_flag,
                   src.timeout_ns))
      break;
    const int t = wb.desc[ds][0];
    const fwh::Task k{wb.desc[ds][1], wb.desc[ds][2], wb.desc[ds][3], wb.desc[ds][4]};
    const bool fast = wb.desc[ds][5] != 0;
    const int g = wb.desc[ds][6];
    const int dec = wb.desc[ds][7];
    __syncwarp();
    if (lane == 0) mbar_arrive(&wb.desc_empty[ds]);
    ++idesc;
    if (t < 0) break;
    uint64_t* tr = tid == 0 ? trace_slot(src.trace, src.trace_cap, src.trace_stride, t) : nullptr;
    if (tr) tr[6] = globaltimer();
    const bool ok = with_bs<kFixedBS, LBS>(src.bs(g), [&](auto B) {
      return compute_task<T, decltype(B)::value, LBS>(src.args(g), k, fast, dec, smem, &wb, &cs,
                                                      pc, tr);
    });
    if (tr) tr[9] = globaltimer();
    if (!ok) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(&wb.task_done);
  }
}

// One graph: the queue of decode_task, block size BS.
template <typename T, int BS>
struct SingleSrc {
  Args<T> a;
  unsigned* next;
  int* status;
  int* abort_flag;
  int64_t timeout_ns;
  int skip_task;
  uint64_t* trace;
  int trace_cap, trace_stride;
  __device__ SingleSrc(const Args<T>& x, const void* tmapD, const void* tmapP)
      : a(x), next(x.ctr), status(x.status), abort_flag(x.abort_flag), timeout_ns(x.timeout_ns),
        skip_task(x.skip_task), trace(x.trace), trace_cap(x.trace_cap),
        trace_stride(x.trace_stride) {
    a.tmapD = tmapD;
    a.tmapP = tmapP;
  }
  __device__ int64_t total() const { return a.stage_off[a.R + 1]; }
  __device__ fwh::Task resolve(int64_t t, int& g) const {
    g = 0;
    return fwh::decode_task(t, a.R, a.lookahead, a.stage_off);
  }
  __device__ const Args<T>& args(int) const { return a; }
  __device__ int bs(int) const { return BS; }
};

template <typename T, int BS>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_persistent_ws(Args<T> a, const __grid_constant__ CUtensorMap tmD,
                    const __grid_constant__ CUtensorMap tmP, int use_tmap) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ WsBars wb;
  __shared__ CtaScratch cs;
  // use_tmap: bit 0 the D map, bit 1 the P map
  const SingleSrc<T, BS> src(a, (use_tmap & 1) ? &tmD : nullptr, (use_tmap & 2) ? &tmP : nullptr);
  ws_engine<T, BS, BS>(src, smem, wb, cs);
}

}  // namespace fwk
