// Device-side building blocks of the blocked Floyd-Warshall solver.
//
// Blocked FW (Sec. 2.3, "Blocked FW Algorithm", Fig. 2): the matrix is cut into BS x BS tiles, R = ceil(n/BS)
// rounds; round r runs
//   phase 1  the pivot tile (r,r): in-place FW over the BS vertices of block r,
//   phase 2/3 the pivot row tiles (r,j) and column tiles (i,r), each relaxed
//            through the closed pivot tile,
//   phase 4  every other tile (i,j): D_ij = min(D_ij, D_ir (x) D_rj), a min-plus
//            product with inner dimension BS.
// Phases 2 and 3 are independent of each other and run as one "panel" step.
//
// GPU design (not the paper's x86 code):
//   * One task = one tile, processed by a 256-thread CTA; each thread owns a
//     register micro-tile of (BS/16) x (BS/16) outputs.
//   * Phase-4 and panel tasks are min-plus products: the left operand A is
//     stored k-major ("A-form", As[kk][a]) and the right operand B row-major
//     ("B-form", Bs[kk][b]) in shared memory, so that each k step reads two
//     vectors per thread.
//   * Predecessors (last hop, strict "<", see fw.h) are tracked without extra
//     instructions in the int32 inner loop by relaxing packed keys
//         key = (min(d, CAP) << KB) | code,   code = kk + 1 (0 = unchanged)
//     with one __viaddmin_u32 per relaxation.  The minimum key gives both the
//     new distance and the first minimising kk.  This is exact whenever every
//     finite entry of the two operand tiles is bounded so that their sums stay
//     below CAP; each panel tile carries that bound, and a task whose operands
//     exceed it falls back to the generic kernel (distance compare + argmin
//     select per relaxation), which is also the fp32 kernel.
//   * Panel outputs are copied into double-buffered "snapshots" (already in
//     A-form / B-form and in packed-key encoding) that phase-4 tasks stream
//     into shared memory with cp.async.bulk (TMA), so that the next round may
//     overwrite the live panel tiles while this round's phase-4 tasks still
//     read them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

namespace fwk {

constexpr int kThreads = 256;

// Status bits of the sticky device status word.
constexpr int kStTimeout = 1;
constexpr int kStNegCycle = 2;

// ------------------------------------------------------------------ PTX ----

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 2-D tiled tensor copy global -> shared (box of the tensor map at element
// coordinates x = column, y = row), completing on `bar`.  x * 4 bytes must be
// a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], "
      "[%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Bulk stores shared -> global through the TMA unit (bulk-group completion:
// the issuing thread commits and waits for its own groups).  Addresses
// 16-byte aligned, sizes multiples of 16 bytes.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
// 2-D tiled tensor store (box at element coordinates x = column, y = row;
// elements outside the tensor are not written).
__device__ __forceinline__ void tma_store_2d(const void* tmap, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::
                   "l"(tmap),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit_wait_all() {
  asm volatile("cp.async.bulk.commit_group;\n cp.async.bulk.wait_group 0;" ::: "memory");
}
// Commit this thread's bulk stores and wait until their shared-memory source
// has been read (the buffer may be reused; the writes may still be in flight).
__device__ __forceinline__ void bulk_commit_wait_read() {
  asm volatile("cp.async.bulk.commit_group;\n cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// Wait until every bulk store this thread committed has been performed.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Order this thread's earlier generic shared-memory accesses before its
// following async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 1-D bulk copy global -> shared through the TMA unit, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, "
      "p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// The same with a suspend-time hint (ns): a waiting thread sleeps until the
// phase completes or the hint expires instead of re-polling at the hardware's
// own, shorter interval.  Re-polling is not free: the producer warp shares an
// SM sub-partition's issue slots and ALU pipe with two compute warps, and its
// polls measurably slowed them.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, unsigned phase,
                                                    unsigned hint_ns) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Barrier over the 256 compute threads (warps 0-7).  In kernels that add a
// producer warp, that warp does not take part; in 256-thread kernels this is
// the whole CTA.
__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// SM-cycle stamps of the phases of the current pivot / panel task (thread 0
// writes them; the persistent driver's optional trace reads them).
static __shared__ long long t_stamp[4];
__device__ __forceinline__ void stamp(int i) {
  if (threadIdx.x == 0) t_stamp[i] = clock64();
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ------------------------------------------------------------- geometry ----

// Thread micro-tile layout for a BS x BS tile and 256 threads (16 x 16):
// a thread (ty, tx) owns TM rows and TM columns, in NG groups of G consecutive
// indices, groups SPAN apart.  BS=128: rows ty*4+{0..3} and 64+ty*4+{0..3}.
template <int BS>
struct Geo {
  static constexpr int TM = BS / 16;
  static constexpr int G = TM < 4 ? TM : 4;
  static constexpr int NG = TM / G;
  static constexpr int SPAN = BS / NG;
  static_assert(TM * 16 == BS && SPAN == 16 * G, "bad tile geometry");
  __device__ __forceinline__ static int idx(int t, int m) { return (m / G) * SPAN + t * G + (m % G); }
};

// Calls f(std::integral_constant<int, I>{}) for I = 0 .. N-1 (compile-time
// loop indices, e.g. register indices of a micro-tile).
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Packed-key parameters: KB bits hold the code kk+1 (1..BS), CAP bounds the
// distance part so that key(A) + key(B) never wraps a uint32.
template <int BS>
struct Keys {
  static constexpr int KB = (BS == 128) ? 8 : (BS == 64) ? 7 : 6;
  static constexpr uint32_t MASK = (1u << KB) - 1u;
  static constexpr int CAP = (1 << (31 - KB)) - 1;
  static_assert((1 << (KB - 1)) == BS, "BS must be 32, 64 or 128");
};

// Element types: int32 and fp32 (the relaxation of the hot path), int64 and
// fp64 (the paper's double-precision runs, Sec. 4).  kInt: sums are exact, so
// the "via" predecessor encoding holds; kPacked: the DPX packed-key kernels
// apply (int32 only).  Missing edges: 2^29 (int32), 2^61 (int64), +inf.
template <typename T>
struct Num;
template <>
struct Num<int32_t> {
  static constexpr bool kInt = true;
  static constexpr bool kPacked = true;
  __device__ __forceinline__ static int32_t inf() { return 1 << 29; }
  __device__ __forceinline__ static bool finite(int32_t v) { return v < (1 << 29); }
};
template <>
struct Num<float> {
  static constexpr bool kInt = false;
  static constexpr bool kPacked = false;
  __device__ __forceinline__ static float inf() { return __int_as_float(0x7f800000); }
  __device__ __forceinline__ static bool finite(float v) { return v < __int_as_float(0x7f800000); }
};
template <>
struct Num<int64_t> {
  static constexpr bool kInt = true;
  static constexpr bool kPacked = false;
  __device__ __forceinline__ static int64_t inf() { return (int64_t)1 << 61; }
  __device__ __forceinline__ static bool finite(int64_t v) { return v < ((int64_t)1 << 61); }
};
template <>
struct Num<double> {
  static constexpr bool kInt = false;
  static constexpr bool kPacked = false;
  __device__ __forceinline__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
  __device__ __forceinline__ static bool finite(double v) {
    return v < __longlong_as_double(0x7ff0000000000000ll);
  }
};

// a < b in the relaxations.  fp64 values are compared as signed 64-bit
// integers of their bit patterns: that orders every non-negative double and
// +inf like the values themselves and keeps every negative value below every
// non-negative one (all a negative-cycle check needs).  The integer compare
// runs on the ALU pipe; a DSETP or DMNMX would share GB300's narrow FP64 pipe
// with the add, halving the fp64 relaxation rate (measured: 0.83 vs 1.63
// relaxations per SM clock).
template <typename T>
__device__ __forceinline__ bool relax_lt(T a, T b) {
  if constexpr (std::is_same<T, double>::value) return __double_as_longlong(a) < __double_as_longlong(b);
  else return a < b;
}

// min of two elements (fminf for fp32: no NaN occurs; fp64 as relax_lt).
template <typename T>
__device__ __forceinline__ T vmin(T a, T b) {
  if constexpr (std::is_same<T, float>::value) return fminf(a, b);
  else return relax_lt<T>(a, b) ? a : b;
}

// Raw vector of NB bytes and G elements viewed as one value (8-byte elements).
template <int NB> struct RawVec;
template <> struct RawVec<16> { int4 a; };
template <> struct RawVec<32> { int4 a, b; };
template <int G, typename T> struct ValVec { T v[G]; };

// Vector load / store of G consecutive elements (32-bit elements: one 16- or
// 8-byte access; 64-bit elements: one or two 16-byte accesses).
template <int G, typename T>
__device__ __forceinline__ void vload_cg(T (&dst)[G], const T* src) {
  if constexpr (sizeof(T) == 8) {
    RawVec<G * 8> r;
    r.a = __ldcg(reinterpret_cast<const int4*>(src));
    if constexpr (G == 4) r.b = __ldcg(reinterpret_cast<const int4*>(src) + 1);
    const ValVec<G, T> v = __builtin_bit_cast(ValVec<G, T>, r);
#pragma unroll
    for (int e = 0; e < G; ++e) dst[e] = v.v[e];
  } else if constexpr (G == 4) {
    int4 v = __ldcg(reinterpret_cast<const int4*>(src));
    dst[0] = __builtin_bit_cast(T, v.x); dst[1] = __builtin_bit_cast(T, v.y);
    dst[2] = __builtin_bit_cast(T, v.z); dst[3] = __builtin_bit_cast(T, v.w);
  } else {
    int2 v = __ldcg(reinterpret_cast<const int2*>(src));
    dst[0] = __builtin_bit_cast(T, v.x); dst[1] = __builtin_bit_cast(T, v.y);
  }
}
template <int G, typename T>
__device__ __forceinline__ void vstore(T* dst, const T (&src)[G]) {
  if constexpr (sizeof(T) == 8) {
    ValVec<G, T> v;
#pragma unroll
    for (int e = 0; e < G; ++e) v.v[e] = src[e];
    const RawVec<G * 8> r = __builtin_bit_cast(RawVec<G * 8>, v);
    reinterpret_cast<int4*>(dst)[0] = r.a;
    if constexpr (G == 4) reinterpret_cast<int4*>(dst)[1] = r.b;
  } else if constexpr (G == 4) {
    int4 v;
    v.x = __builtin_bit_cast(int, src[0]); v.y = __builtin_bit_cast(int, src[1]);
    v.z = __builtin_bit_cast(int, src[2]); v.w = __builtin_bit_cast(int, src[3]);
    *reinterpret_cast<int4*>(dst) = v;
  } else {
    int2 v;
    v.x = __builtin_bit_cast(int, src[0]); v.y = __builtin_bit_cast(int, src[1]);
    *reinterpret_cast<int2*>(dst) = v;
  }
}
template <int G, typename T>
__device__ __forceinline__ void vload_s(T (&dst)[G], const T* src) {
  if constexpr (sizeof(T) == 8) {
    RawVec<G * 8> r;
    r.a = reinterpret_cast<const int4*>(src)[0];
    if constexpr (G == 4) r.b = reinterpret_cast<const int4*>(src)[1];
    const ValVec<G, T> v = __builtin_bit_cast(ValVec<G, T>, r);
#pragma unroll
    for (int e = 0; e < G; ++e) dst[e] = v.v[e];
  } else if constexpr (G == 4) {
    int4 v = *reinterpret_cast<const int4*>(src);
    dst[0] = __builtin_bit_cast(T, v.x); dst[1] = __builtin_bit_cast(T, v.y);
    dst[2] = __builtin_bit_cast(T, v.z); dst[3] = __builtin_bit_cast(T, v.w);
  } else {
    int2 v = *reinterpret_cast<const int2*>(src);
    dst[0] = __builtin_bit_cast(T, v.x); dst[1] = __builtin_bit_cast(T, v.y);
  }
}

// ------------------------------------------------------------ arguments ----

// Everything one solve needs on the device.  Snapshot arrays have two slots
// (round parity); a slot holds R tiles of BS*BS elements.
template <typename T>
struct Args {
  T* D;                 // n x ld, in place
  int32_t* P;           // n x ld, predecessors
  int64_t n, ld;
  int R;                // tiles per side
  int slot_tiles;       // tiles per snapshot slot (>= R)
  // scheduling state (persistent driver)
  int* ver;             // R*R tile versions: rounds completed on the tile
  int* done;            // [2R]: panel tasks done in round r (done[r]), remaining tiles
                        // done in round r (done[R + r]); they guard snapshot slot reuse
  unsigned* ctr;        // [0] next task
  int* abort_flag;
  int* status;
  const unsigned* stage_off;  // R+2 queue offsets of the stages
  int lookahead;
  int skip_task;
  int64_t timeout_ns;
  int packed;           // int32 only: packed keys allowed
  // snapshots
  T* piv;               // [2][BS*BS] closed pivot tile, row-major
  int32_t* pivP;        // [2][BS*BS]
  uint32_t* colK;       // [2][tiles][BS*BS] column panel tiles, A-form, packed keys
  T* colR;              // [2][tiles][BS*BS] same, raw values
  int32_t* colB;        // [2][tiles] bound of the tile's finite entries
  uint32_t* rowK;       // [2][tiles][BS*BS] row panel tiles, B-form, packed keys
  T* rowR;              // raw
  int32_t* rowP;        // [2][tiles][BS*BS] predecessors of the row panel tiles
  int32_t* rowB;
  // 2-D tensor map of D (CUtensorMap, BS x BS boxes) for the persistent
  // driver's tile loads; null: the tile is copied row by row
  const void* tmapD;
  const void* tmapP;
  // optional per-task trace (persistent driver)
  uint64_t* trace;
  int trace_cap;
  int trace_stride;
};

// -------------------------------------------------------- shared memory ----

template <int BS, typename T>
struct Smem {
  static constexpr int kTile = BS * BS;
  // As and Bs (BS*BS elements each) and Ps (the panel tasks' predecessor
  // source, BS*BS int32); the pivot task reuses As for its row / column
  // broadcast buffers.
  static constexpr size_t bytes() { return (size_t)kTile * (2 * sizeof(T) + 4) + 256; }
};

struct CtaScratch {
  uint64_t bar;        // mbarrier of the operand bulk copies
  int task;            // claimed task index
  int flag;            // broadcast of a thread-0 decision
  int red[2][8];       // per-warp partial maxima
};

// -------------------------------------------------------- tile helpers ----

// Load the thread's micro-tile of tile (ti, tj) of a row-major n x ld matrix
// (L2 only: the tile may have been written by another CTA of this launch).
// Out-of-range entries read as `fill`.
template <int BS, typename T>
__device__ __forceinline__ void load_tile(T (&v)[Geo<BS>::TM][Geo<BS>::TM], const T* M, int64_t n,
                                          int64_t ld, int ti, int tj, int tx, int ty, T fill) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G;
#pragma unroll
  for (int m = 0; m < Gm::TM; ++m) {
    const int64_t gi = (int64_t)ti * BS + Gm::idx(ty, m);
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      const int64_t gj0 = (int64_t)tj * BS + g * Gm::SPAN + tx * G;
      T tmp[G];
      if (gi < n && gj0 < n) {
        vload_cg<G>(tmp, M + gi * ld + gj0);
#pragma unroll
        for (int e = 0; e < G; ++e)
          if (gj0 + e >= n) tmp[e] = fill;
      } else {
#pragma unroll
        for (int e = 0; e < G; ++e) tmp[e] = fill;
      }
#pragma unroll
      for (int e = 0; e < G; ++e) v[m][g * G + e] = tmp[e];
    }
  }
}

// Store the in-range part of a micro-tile.
template <int BS, typename T>
__device__ __forceinline__ void store_tile(T* M, const T (&v)[Geo<BS>::TM][Geo<BS>::TM], int64_t n,
                                           int64_t ld, int ti, int tj, int tx, int ty) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G;
#pragma unroll
  for (int m = 0; m < Gm::TM; ++m) {
    const int64_t gi = (int64_t)ti * BS + Gm::idx(ty, m);
    if (gi >= n) continue;
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      const int64_t gj0 = (int64_t)tj * BS + g * Gm::SPAN + tx * G;
      if (gj0 + G <= n) {
        T tmp[G];
#pragma unroll
        for (int e = 0; e < G; ++e) tmp[e] = v[m][g * G + e];
        vstore<G>(M + gi * ld + gj0, tmp);
      } else {
#pragma unroll
        for (int e = 0; e < G; ++e)
          if (gj0 + e < n) M[gi * ld + gj0 + e] = v[m][g * G + e];
      }
    }
  }
}

// Write a micro-tile into a BS x BS buffer (shared or global), natural layout
// buf[row][col] ("B-form"), or transposed buf[col][row] ("A-form").
template <int BS, bool kTransposed, typename U>
__device__ __forceinline__ void put_tile(U* buf, const U (&v)[Geo<BS>::TM][Geo<BS>::TM], int tx,
                                         int ty) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G;
  if constexpr (!kTransposed) {
#pragma unroll
    for (int m = 0; m < Gm::TM; ++m)
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        U tmp[G];
#pragma unroll
        for (int e = 0; e < G; ++e) tmp[e] = v[m][g * G + e];
        vstore<G>(buf + Gm::idx(ty, m) * BS + g * Gm::SPAN + tx * G, tmp);
      }
  } else {
#pragma unroll
    for (int nn = 0; nn < Gm::TM; ++nn)
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        U tmp[G];
#pragma unroll
        for (int e = 0; e < G; ++e) tmp[e] = v[g * G + e][nn];
        vstore<G>(buf + Gm::idx(tx, nn) * BS + g * Gm::SPAN + ty * G, tmp);
      }
  }
}

// Packed key of a distance: min(d, CAP) << KB (code bits zero).  d >= 0.
template <int BS>
__device__ __forceinline__ uint32_t key_of(int32_t d) {
  return (uint32_t)min(d, Keys<BS>::CAP) << Keys<BS>::KB;
}

// Bound of a value for the packed-key test: finite entries count as
// themselves, INF as 0, negative entries as CAP (they disable the fast path).
template <int BS, typename T>
__device__ __forceinline__ int bound_of(T v) {
  if constexpr (Num<T>::kPacked) {
    if (!Num<T>::finite(v)) return 0;
    return v < 0 ? Keys<BS>::CAP : min((int)v, Keys<BS>::CAP);
  } else {
    return Keys<BS>::CAP;
  }
}

// Predecessors of the int32 solver ("via" encoding).  A remaining-tile task
// that improves (i, j) through vertex k = r*BS + kk records -(k + 2) instead of
// gathering the last hop of (k, j).  (k, j) cannot improve again while (i, j)
// still records k: a later strict improvement of (k, j) through block r'
// improves (i, j) through block r' as well (integer sums are exact).  So the
// last hop of (i, j) is that of (k, j), which may itself be a via code of an
// earlier round; pivot tasks copy such entries as they are, and
// k_resolve_pred follows each chain once the solve is done.  The persistent
// driver's panel tasks record via codes too: a row-panel entry (i, j) improved
// through k of block r names (k, j) of the same tile, which that panel left
// unchanged (had (k, j) improved through k', (i, j) would do better through
// k', the pivot being closed); a column-panel entry names (k, j) of the
// closed pivot.  fp32 keeps gathering real last hops: float
// sums are not associative, and the argument needs them to be.
template <typename T>
struct ViaPred {
  static constexpr bool kOn = Num<T>::kInt;
};
__device__ __forceinline__ int32_t via_code(int64_t k) { return (int32_t)(-(k + 2)); }
// The last hop that entry p of column j stands for (p itself unless a via code).
// A chain takes at most two links per round (a remaining tile's code names an
// entry of its row-panel tile, whose own code, if it has one from the same
// round, names an entry that round left unchanged), so 2 * 1024 + 2 links
// cover every solve; the cap only bounds the walk on a corrupted matrix.
__device__ __forceinline__ int32_t resolve_pred(int32_t p, const int32_t* P, int64_t ld,
                                                int64_t j) {
  for (int hop = 0; p <= -2 && hop <= 2 * 1024 + 2; ++hop)
    p = P[(int64_t)(-(int64_t)p - 2) * ld + j];
  return p;
}

// CTA-wide maximum of two ints (every thread gets the result).
__device__ __forceinline__ void block_max2(int& a, int& b, CtaScratch* cs) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5;
  bar_compute();
  if ((threadIdx.x & 31) == 0) { cs->red[0][w] = a; cs->red[1][w] = b; }
  bar_compute();
  a = cs->red[0][0];
  b = cs->red[1][0];
#pragma unroll
  for (int k = 1; k < kThreads / 32; ++k) { a = max(a, cs->red[0][k]); b = max(b, cs->red[1][k]); }
}

// ---------------------------------------------------------- min-plus cores ----

// acc[m][n] = min(acc[m][n], min_kk key(A[kk][row m]) + key(B[kk][col n]))
// over packed keys: one __viaddmin_u32 (DPX) per relaxation.
template <int BS, int K = BS>
__device__ __forceinline__ void core_packed(const uint32_t* __restrict__ As,
                                            const uint32_t* __restrict__ Bs,
                                            uint32_t (&acc)[Geo<BS>::TM][Geo<BS>::TM], int tx,
                                            int ty) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G, TM = Gm::TM;
  // Unrolled 8 steps: measured at n = 32768 (2.18 / 2.12 / 2.08 / 2.09 / 2.22 / 2.23 s
  // per solve for 2 / 4 / 8 / 16 / 32 / 64): the loop's address and branch
  // instructions share the ALU pipe with the DPX relaxations; beyond 8 the
  // loop body outgrows the instruction cache.
#pragma unroll 8
  for (int kk = 0; kk < K; ++kk) {
    uint32_t a[TM], b[TM];
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      uint32_t ta[G], tb[G];
      vload_s<G>(ta, As + kk * BS + g * Gm::SPAN + ty * G);
      vload_s<G>(tb, Bs + kk * BS + g * Gm::SPAN + tx * G);
#pragma unroll
      for (int e = 0; e < G; ++e) { a[g * G + e] = ta[e]; b[g * G + e] = tb[e]; }
    }
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) acc[m][nn] = __viaddmin_u32(a[m], b[nn], acc[m][nn]);
  }
}

// 1.0f when a < b, else 0.0f, in one instruction (PTX set with a float
// destination).
__device__ __forceinline__ float lt_one(float a, float b) {
  float r;
  asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// fp32 argmin accumulator -> step + 1 (0: no improvement).  The accumulator
// (arg's bits, see core_generic) is 0 or lies in [2^k, 2^(k+1)) for the last
// improving step k, so its exponent field is k + 127.
template <typename T, int TM>
__device__ __forceinline__ void argmin_finish(int (&arg)[TM][TM]) {
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) arg[m][nn] = arg[m][nn] ? (arg[m][nn] >> 23) - 126 : 0;
  }
}

// Generic relaxation with an explicit first-argmin: s = A + B; if (s < acc)
// { acc = s; arg = kk + 1 }.  Used for fp32, the 64-bit types and int32
// tiles whose values exceed the packed-key bound.
//
// fp32 keeps the argmin on the FMA pipe: while the steps run, arg holds the
// bits of a float accumulator to which every improving step k = kk0 + kk adds
// 2^k, rounded toward zero.  Toward zero, a sum of distinct powers of two
// never reaches the power of two above its largest term, so the
// accumulator's exponent is the last improving step -- the first step that
// reached the final minimum, as with the strict compare.  Per relaxation:
// add, set (1.0 / 0.0), min and fma.rz, two ALU-pipe instructions where the
// compare and two selects take three.  k < 128 keeps 2^k finite.  The
// accumulator becomes step + 1 in argmin_finish, at the end of the call
// (kFinish) or after a caller's last chunk.
template <int BS, typename T, int K = BS, bool kFinish = true>
__device__ __forceinline__ void core_generic(const T* __restrict__ As, const T* __restrict__ Bs,
                                             T (&acc)[Geo<BS>::TM][Geo<BS>::TM],
                                             int (&arg)[Geo<BS>::TM][Geo<BS>::TM], int tx, int ty,
                                             int kk0 = 0) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G, TM = Gm::TM;
  static_assert(BS <= 128, "the fp32 argmin accumulator holds steps below 128");
  if constexpr (std::is_same<T, float>::value) {
    // 2 steps (n = 8192 with predecessors: 98.4 ms, 99.8 with 1)
#pragma unroll 2
    for (int kk = 0; kk < K; ++kk) {
      float a[TM], b[TM];
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        float ta[G], tb[G];
        vload_s<G>(ta, As + kk * BS + g * Gm::SPAN + ty * G);
        vload_s<G>(tb, Bs + kk * BS + g * Gm::SPAN + tx * G);
#pragma unroll
        for (int e = 0; e < G; ++e) { a[g * G + e] = ta[e]; b[g * G + e] = tb[e]; }
      }
      const float w = __int_as_float((127 + kk0 + kk) << 23);   // 2^(kk0 + kk)
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) {
          const float s = a[m] + b[nn];
          const float p = lt_one(s, acc[m][nn]);
          acc[m][nn] = fminf(acc[m][nn], s);
          arg[m][nn] = __float_as_int(__fmaf_rz(p, w, __int_as_float(arg[m][nn])));
        }
    }
    if constexpr (kFinish) argmin_finish<T>(arg);
    return;
  }
  // 2 steps (n = 8192 int64 252 -> 246 ms, and fp32 105.6 -> 102.8 ms when it
  // took this loop; 4 and 8 spill at the 168-register cap of the persistent kernel)
#pragma unroll 2
  for (int kk = 0; kk < K; ++kk) {
    T a[TM], b[TM];
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      T ta[G], tb[G];
      vload_s<G>(ta, As + kk * BS + g * Gm::SPAN + ty * G);
      vload_s<G>(tb, Bs + kk * BS + g * Gm::SPAN + tx * G);
#pragma unroll
      for (int e = 0; e < G; ++e) { a[g * G + e] = ta[e]; b[g * G + e] = tb[e]; }
    }
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        T s = a[m] + b[nn];
        bool lt = relax_lt<T>(s, acc[m][nn]);
        acc[m][nn] = lt ? s : acc[m][nn];
        arg[m][nn] = lt ? kk0 + kk + 1 : arg[m][nn];
      }
  }
}

// Distance-only relaxation: acc[m][n] = min(acc[m][n], min_kk A + B), two
// instructions per relaxation (add, min), no argmin.
template <int BS, typename T, int K>
__device__ __forceinline__ void core_min(const T* __restrict__ As, const T* __restrict__ Bs,
                                         T (&acc)[Geo<BS>::TM][Geo<BS>::TM], int tx, int ty) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G, TM = Gm::TM;
  // 8 steps (n = 8192 fp32 distance-only 43.8 -> 42.4 ms)
#pragma unroll 8
  for (int kk = 0; kk < K; ++kk) {
    T a[TM], b[TM];
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      T ta[G], tb[G];
      vload_s<G>(ta, As + kk * BS + g * Gm::SPAN + ty * G);
      vload_s<G>(tb, Bs + kk * BS + g * Gm::SPAN + tx * G);
#pragma unroll
      for (int e = 0; e < G; ++e) { a[g * G + e] = ta[e]; b[g * G + e] = tb[e]; }
    }
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) acc[m][nn] = vmin<T>(a[m] + b[nn], acc[m][nn]);
  }
}

// ------------------------------------------------------------- phase 1 ----

// OR of a predicate over the 256 compute threads (one named barrier).
__device__ __forceinline__ bool bar_compute_or(bool v) {
  unsigned out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"(v ? 1u : 0u)
      : "memory");
  return out != 0;
}

// Negative-cycle check of a closed pivot tile, its stores to the live matrix
// and to the pivot snapshot of slot r&1 (distances and predecessors apart, so
// that the distances leave registers before predecessors are resolved).
template <typename T, int BS>
__device__ __forceinline__ void pivot_store_dist(const Args<T>& a, int r,
                                                 const T (&d)[Geo<BS>::TM][Geo<BS>::TM], int tx,
                                                 int ty) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM;
  bool neg = false;
#pragma unroll
  for (int mm = 0; mm < TM; ++mm)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn)
      if (Gm::idx(ty, mm) == Gm::idx(tx, nn) && d[mm][nn] < T(0)) neg = true;
  if (neg) atomicOr(a.status, kStNegCycle);
  store_tile<BS>(a.D, d, a.n, a.ld, r, r, tx, ty);
  put_tile<BS, false>(a.piv + (size_t)(r & 1) * BS * BS, d, tx, ty);
}
template <typename T, int BS>
__device__ __forceinline__ void pivot_store_pred(const Args<T>& a, int r,
                                                 const int32_t (&p)[Geo<BS>::TM][Geo<BS>::TM],
                                                 int tx, int ty) {
  if (!a.P) return;  // distance-only
  store_tile<BS>(a.P, p, a.n, a.ld, r, r, tx, ty);
  put_tile<BS, false>(a.pivP + (size_t)(r & 1) * BS * BS, p, tx, ty);
}

// Step kk of the packed pivot for the owners of row / column kk+1 (register
// index MP in their micro-tiles, owner thread row / column `own`): relax those
// elements through kk first and publish them as the broadcast of step kk+1,
// so that the next barrier does not wait for a whole step's relaxations.
// Re-relaxing them in the full step afterwards is a no-op (min is idempotent).
template <int BS, int MP>
__device__ __forceinline__ void pivot_publish_next(uint32_t (&acc)[Geo<BS>::TM][Geo<BS>::TM],
                                                   const uint32_t (&cv)[Geo<BS>::TM],
                                                   const uint32_t (&rv)[Geo<BS>::TM], int own,
                                                   int kk1, uint32_t* rowK, uint32_t* colK,
                                                   int tx, int ty) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int buf = kk1 & 1;
  if (ty == own) {
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) acc[MP][nn] = __viaddmin_u32(cv[MP], rv[nn], acc[MP][nn]);
#pragma unroll
    for (int gg = 0; gg < Gm::NG; ++gg) {
      uint32_t v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) v[q] = acc[MP][gg * G + q] & ~K::MASK;
      vstore<G>(rowK + buf * BS + gg * Gm::SPAN + tx * G, v);
    }
  }
  if (tx == own) {
#pragma unroll
    for (int mm = 0; mm < TM; ++mm) acc[mm][MP] = __viaddmin_u32(cv[mm], rv[MP], acc[mm][MP]);
#pragma unroll
    for (int gg = 0; gg < Gm::NG; ++gg) {
      uint32_t v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) v[q] = (acc[gg * G + q][MP] & ~K::MASK) + (uint32_t)(kk1 + 1);
      vstore<G>(colK + buf * BS + gg * Gm::SPAN + ty * G, v);
    }
  }
}

// Packed-key pivot (int32, bounded entries).
template <typename T, int BS>
__device__ __forceinline__ void pivot_packed(const Args<T>& a, int r, void* smem_raw,
                                             const T (&d)[Geo<BS>::TM][Geo<BS>::TM],
                                             const int32_t (&p)[Geo<BS>::TM][Geo<BS>::TM]) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM, G = Gm::G, NG = Gm::NG;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // shared memory: [0, BS^2) the step broadcasts, then (after the steps) nxt;
  // [BS^2, 2 BS^2) val; [2 BS^2, 3 BS^2) the closed distances until stored
  uint32_t* rowK = reinterpret_cast<uint32_t*>(smem_raw);  // [2][BS]
  uint32_t* colK = rowK + 2 * BS;                          // [2][BS]
  int32_t* nxt = reinterpret_cast<int32_t*>(smem_raw);     // [BS][BS], after the steps
  int32_t* val = nxt + BS * BS;                            // [BS][BS]
  T* dst = reinterpret_cast<T*>(val + BS * BS);            // [BS][BS]
  uint32_t acc[TM][TM];
  {
    // the old predecessors wait in shared memory (not in registers) during the steps
#pragma unroll
    for (int mm = 0; mm < TM; ++mm)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        val[Gm::idx(ty, mm) * BS + Gm::idx(tx, nn)] = p[mm][nn];
        acc[mm][nn] = key_of<BS>((int32_t)d[mm][nn]);
      }
  }
  stamp(1);
  // broadcast of step 0: row 0 and column 0 (owner thread row / column 0, register 0)
  if (ty == 0) {
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) {
      uint32_t v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) v[q] = acc[0][gg * G + q];
      vstore<G>(rowK + gg * Gm::SPAN + tx * G, v);
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) {
      uint32_t v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) v[q] = acc[gg * G + q][0] + 1u;
      vstore<G>(colK + gg * Gm::SPAN + ty * G, v);
    }
  }
  static_for<NG>([&](auto gc) {
    constexpr int g = decltype(gc)::value;
#pragma unroll 1
    for (int to = 0; to < 16; ++to) {
      static_for<G>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const int kk = g * Gm::SPAN + to * G + e;  // row kk = register g*G+e of thread row to
        const int buf = kk & 1;
        bar_compute();
        uint32_t cv[TM], rv[TM];
#pragma unroll
        for (int gg = 0; gg < NG; ++gg) {
          uint32_t tc[G], tr[G];
          vload_s<G>(tc, colK + buf * BS + gg * Gm::SPAN + ty * G);
          vload_s<G>(tr, rowK + buf * BS + gg * Gm::SPAN + tx * G);
#pragma unroll
          for (int q = 0; q < G; ++q) { cv[gg * G + q] = tc[q]; rv[gg * G + q] = tr[q]; }
        }
        // row / column kk+1 first
        if constexpr (e + 1 < G) {
          pivot_publish_next<BS, g * G + e + 1>(acc, cv, rv, to, kk + 1, rowK, colK, tx, ty);
        } else {
          if (to < 15) {
            pivot_publish_next<BS, g * G>(acc, cv, rv, to + 1, kk + 1, rowK, colK, tx, ty);
          } else if constexpr (g + 1 < NG) {
            pivot_publish_next<BS, (g + 1) * G>(acc, cv, rv, 0, kk + 1, rowK, colK, tx, ty);
          }
        }
#pragma unroll
        for (int mm = 0; mm < TM; ++mm)
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) acc[mm][nn] = __viaddmin_u32(cv[mm], rv[nn], acc[mm][nn]);
      });
    }
  });
  stamp(2);
  // Chains of last steps: element (a, b) last improved at step kk takes the
  // final last hop of (kk, b), whose own last improving step is earlier; walk
  // each chain down to an element that never improved and take its old
  // predecessor.  The closed distances wait in shared memory: global stores
  // issued now would hold up the walk's shared loads behind them in the
  // load/store queue when memory is busy.
  bar_compute();  // nxt overwrites the last step's broadcast
#pragma unroll
  for (int mm = 0; mm < TM; ++mm)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) {
      const int e = Gm::idx(ty, mm) * BS + Gm::idx(tx, nn);
      nxt[e] = (int)(acc[mm][nn] & K::MASK) - 1;
      const int32_t v = (int32_t)(acc[mm][nn] >> K::KB);
      dst[e] = v == K::CAP ? Num<T>::inf() : (T)v;
    }
  bar_compute();
  int32_t pr[TM][TM];
  if (!a.P) {  // distance-only: no predecessors to resolve
#pragma unroll
    for (int mm = 0; mm < TM; ++mm)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) pr[mm][nn] = -1;
  } else {
    constexpr int kWalk = 8;  // hops walked directly; longer chains fall back to jumping
    bool unresolved = false;
    {
      // all of a thread's chains advance one hop at a time, so that the
      // dependent shared loads of different chains overlap; c is each chain's
      // current row (ended when its nxt entry is negative)
      int c[TM][TM];
#pragma unroll
      for (int mm = 0; mm < TM; ++mm)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) c[mm][nn] = Gm::idx(ty, mm);
      bool moved = true;
#pragma unroll 1
      for (int hop = 0; hop < kWalk && moved; ++hop) {
        moved = false;
#pragma unroll
        for (int mm = 0; mm < TM; ++mm)
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            const int nx = nxt[c[mm][nn] * BS + Gm::idx(tx, nn)];
            if (nx >= 0) {
              c[mm][nn] = nx;
              moved = true;
            }
          }
        moved = __any_sync(0xffffffffu, moved);
      }
      // a warp that still moved on its last allowed hop may hold longer chains
      unresolved = moved;
#pragma unroll
      for (int mm = 0; mm < TM; ++mm)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) pr[mm][nn] = val[c[mm][nn] * BS + Gm::idx(tx, nn)];
    }
    if (bar_compute_or(unresolved)) {
      // pointer jumping: every round doubles the resolved chain length, and a
      // chain is at most BS long (its steps strictly decrease)
      for (int round = 0; (1 << round) <= 2 * BS; ++round) {
        int nk[TM][TM];
#pragma unroll
        for (int mm = 0; mm < TM; ++mm)
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            const int col = Gm::idx(tx, nn);
            const int k = nxt[Gm::idx(ty, mm) * BS + col];
            nk[mm][nn] = -2;
            if (k >= 0) {
              const int nkk = nxt[k * BS + col];
              nk[mm][nn] = nkk;
              if (nkk < 0) pr[mm][nn] = val[k * BS + col];
            }
          }
        bar_compute();
#pragma unroll
        for (int mm = 0; mm < TM; ++mm)
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            if (nk[mm][nn] == -2) continue;
            const int e = Gm::idx(ty, mm) * BS + Gm::idx(tx, nn);
            if (nk[mm][nn] < 0) {
              val[e] = pr[mm][nn];
              nxt[e] = -1;
            } else {
              nxt[e] = nk[mm][nn];
            }
          }
        bar_compute();
      }
#pragma unroll
      for (int mm = 0; mm < TM; ++mm)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) pr[mm][nn] = val[Gm::idx(ty, mm) * BS + Gm::idx(tx, nn)];
    }
  }
  stamp(3);
  // Results out: distances are staged in dst, predecessors go to the nxt
  // region (free once the walk is done); full tiles and the snapshots leave by
  // TMA bulk stores, which do not queue behind one another in the SM's
  // load/store unit the way 64 vector stores per thread do.
  int32_t* pst = nxt;
  bar_compute();
  bool neg = false;
#pragma unroll
  for (int mm = 0; mm < TM; ++mm)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) {
      const int e = Gm::idx(ty, mm) * BS + Gm::idx(tx, nn);
      if (a.P) pst[e] = pr[mm][nn];
      if (Gm::idx(ty, mm) == Gm::idx(tx, nn) && dst[e] < T(0)) neg = true;
    }
  if (neg) atomicOr(a.status, kStNegCycle);
  bar_compute();
  const int64_t r0 = (int64_t)r * BS;
  // Bulk stores of the live tiles only when the pivot tile lies inside the
  // matrix: a tensor store clips at 16-byte granules of a row, so a ragged
  // edge would overwrite the caller's padding columns.
  const bool whole = r0 + BS <= a.n;
  if (tid < 32) {
    fence_proxy_async_shared();
    const size_t slot = (size_t)(r & 1) * BS * BS;
    if (tid == 0) {
      bulk_s2g(a.piv + slot, dst, (unsigned)(BS * BS * sizeof(T)));
      if (a.P) bulk_s2g(a.pivP + slot, pst, (unsigned)(BS * BS * 4));
      if (whole && a.tmapD) tma_store_2d(a.tmapD, (int)r0, (int)r0, dst);
      if (whole && a.P && a.tmapP) tma_store_2d(a.tmapP, (int)r0, (int)r0, pst);
    }
    if (whole && !a.tmapD)
      for (int rr = tid; rr < BS; rr += 32)
        bulk_s2g(a.D + (r0 + rr) * a.ld + r0, dst + rr * BS, (unsigned)(BS * sizeof(T)));
    if (whole && a.P && !a.tmapP)
      for (int rr = tid; rr < BS; rr += 32)
        bulk_s2g(a.P + (r0 + rr) * a.ld + r0, pst + rr * BS, (unsigned)(BS * 4));
    bulk_commit_wait_all();
  }
  if (!whole) {  // ragged pivot tile: in-range stores
    T dd[TM][TM];
#pragma unroll
    for (int mm = 0; mm < TM; ++mm)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) dd[mm][nn] = dst[Gm::idx(ty, mm) * BS + Gm::idx(tx, nn)];
    store_tile<BS>(a.D, dd, a.n, a.ld, r, r, tx, ty);
    if (a.P) store_tile<BS>(a.P, pr, a.n, a.ld, r, r, tx, ty);
  }
}

// The BS steps of the in-place FW closure of one tile held as micro-tiles
// (d, p) by the 256 compute threads: step kk broadcasts row kk and column kk
// through shared memory (double-buffered, one barrier per step) and relaxes
// every owned element through kk with a strict-< compare, the last hop taken
// from row kk's predecessors.  Shared memory: 2 * BS * (2 * sizeof(T) + 4) bytes.
template <typename T, int BS>
__device__ __forceinline__ void closure_steps(T (&d)[Geo<BS>::TM][Geo<BS>::TM],
                                              int32_t (&p)[Geo<BS>::TM][Geo<BS>::TM],
                                              void* smem_raw) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T* rowD = reinterpret_cast<T*>(smem_raw);  // [2][BS]
  int32_t* rowP = reinterpret_cast<int32_t*>(rowD + 2 * BS);
  T* colD = reinterpret_cast<T*>(rowP + 2 * BS);
#pragma unroll
  for (int g = 0; g < Gm::NG; ++g) {
#pragma unroll 1
    for (int to = 0; to < 16; ++to) {
#pragma unroll
      for (int e = 0; e < G; ++e) {
        const int kk = g * Gm::SPAN + to * G + e;
        const int m = g * G + e;  // register index of row / column kk in its owners
        const int buf = kk & 1;
        if (ty == to) {
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            rowD[buf * BS + Gm::idx(tx, nn)] = d[m][nn];
            rowP[buf * BS + Gm::idx(tx, nn)] = p[m][nn];
          }
        }
        if (tx == to) {
#pragma unroll
          for (int mm = 0; mm < TM; ++mm) colD[buf * BS + Gm::idx(ty, mm)] = d[mm][m];
        }
        bar_compute();
        T cv[TM], rv[TM];
        int32_t rp[TM];
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          cv[q] = colD[buf * BS + Gm::idx(ty, q)];
          rv[q] = rowD[buf * BS + Gm::idx(tx, q)];
          rp[q] = rowP[buf * BS + Gm::idx(tx, q)];
        }
#pragma unroll
        for (int mm = 0; mm < TM; ++mm)
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            T s = cv[mm] + rv[nn];
            bool lt = relax_lt<T>(s, d[mm][nn]);
            d[mm][nn] = lt ? s : d[mm][nn];
            p[mm][nn] = lt ? rp[nn] : p[mm][nn];
          }
      }
    }
  }
}

// Eager pivot: compare and select per relaxation (fp32, 64-bit types, large
// int32 entries).
template <typename T, int BS>
__device__ __noinline__ void pivot_eager(const Args<T>& a, int r, void* smem_raw) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T d[TM][TM];
  int32_t p[TM][TM];
  load_tile<BS>(d, a.D, a.n, a.ld, r, r, tx, ty, Num<T>::inf());
  if (a.P) {
    load_tile<BS>(p, a.P, a.n, a.ld, r, r, tx, ty, (int32_t)-1);
  } else {
#pragma unroll
    for (int mm = 0; mm < TM; ++mm)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) p[mm][nn] = -1;
  }
  stamp(1);
  closure_steps<T, BS>(d, p, smem_raw);
  stamp(2);
  stamp(3);
  pivot_store_dist<T, BS>(a, r, d, tx, ty);
  pivot_store_pred<T, BS>(a, r, p, tx, ty);
}

// Pivot tile (r,r): in-place FW over the vertices of block r (Sec. 2.3,
// blocked FW, phase 1).  Each step kk broadcasts row kk and column kk through
// shared memory (double-buffered, one barrier per step) and relaxes every
// owned element through kk.
//
// int32 with bounded entries: packed keys, one __viaddmin_u32 per relaxation;
// the key's code records the LAST step that strictly improved the element.
// That step's row entry is final from then on (a later improvement of it would
// have improved the element again), so the element's last hop is the final
// last hop of (kk, b): predecessors are resolved afterwards down each column.
// Otherwise (fp32, large entries) an eager strict-< update.  Writes the live
// tile and the pivot snapshot of slot r&1.
template <typename T, int BS>
__device__ __noinline__ void task_pivot(const Args<T>& a, int r, void* smem_raw, CtaScratch* cs) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM;
  stamp(0);
  if constexpr (Num<T>::kPacked) {
    // every value formed in the closure is a path of at most BS segments of
    // current entries; keep twice that below CAP.  The tile is loaded once,
    // distances and predecessors together (one memory round trip).
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T d[TM][TM];
    int32_t p[TM][TM];
    load_tile<BS>(d, a.D, a.n, a.ld, r, r, tx, ty, Num<T>::inf());
    if (a.P) {
      load_tile<BS>(p, a.P, a.n, a.ld, r, r, tx, ty, (int32_t)-1);
    } else {
#pragma unroll
      for (int mm = 0; mm < TM; ++mm)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) p[mm][nn] = -1;
    }
    int bnd = 0, dummy = 0;
#pragma unroll
    for (int mm = 0; mm < TM; ++mm)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) bnd = max(bnd, bound_of<BS>(d[mm][nn]));
    block_max2(bnd, dummy, cs);
    if (a.packed && (int64_t)bnd * 2 * BS < (int64_t)K::CAP) {
      pivot_packed<T, BS>(a, r, smem_raw, d, p);
      return;
    }
  }
  pivot_eager<T, BS>(a, r, smem_raw);
}

// ------------------------------------------------------------- phase 2/3 ----

// Micro-tile of a BS x BS buffer with row stride BS (a snapshot or smem tile).
template <int BS, typename T>
__device__ __forceinline__ void load_buf(T (&v)[Geo<BS>::TM][Geo<BS>::TM], const T* buf, int tx,
                                         int ty) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G;
#pragma unroll
  for (int m = 0; m < Gm::TM; ++m)
#pragma unroll
    for (int g = 0; g < Gm::NG; ++g) {
      T tmp[G];
      vload_cg<G>(tmp, buf + Gm::idx(ty, m) * BS + g * Gm::SPAN + tx * G);
#pragma unroll
      for (int e = 0; e < G; ++e) v[m][g * G + e] = tmp[e];
    }
}

// Copy a BS x BS int32 tile into shared memory (row stride BS), cooperatively
// and coalesced: from a row-major n x ld matrix at tile (ti, tj) (entries
// outside [0, n) read as -1), or from a contiguous BS x BS buffer when M is
// null.
template <int BS>
__device__ __forceinline__ void stage_tile_i32(int32_t* dst, const int32_t* M, int64_t n, int64_t ld,
                                               int ti, int tj, const int32_t* buf) {
  constexpr int V = BS / 4;                 // 16-byte vectors per row
  constexpr int NQ = BS * V / kThreads;     // vectors per thread
  static_assert(NQ * kThreads == BS * V, "tile not divisible among the threads");
  // every load first, then every store: one memory round trip, not NQ
  int4 v[NQ];
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const int q = (int)threadIdx.x + u * kThreads;
    const int row = q / V, c4 = (q % V) * 4;
    if (!M) {
      v[u] = __ldcg(reinterpret_cast<const int4*>(buf + row * BS + c4));
    } else {
      const int64_t gi = (int64_t)ti * BS + row, gj = (int64_t)tj * BS + c4;
      v[u] = make_int4(-1, -1, -1, -1);
      if (gi < n && gj < n) {
        v[u] = __ldcg(reinterpret_cast<const int4*>(M + gi * ld + gj));
        if (gj + 1 >= n) v[u].y = -1;
        if (gj + 2 >= n) v[u].z = -1;
        if (gj + 3 >= n) v[u].w = -1;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const int q = (int)threadIdx.x + u * kThreads;
    *reinterpret_cast<int4*>(dst + (q / V) * BS + (q % V) * 4) = v[u];
  }
}

// Results of one group of G micro-tile rows (m = g*G + e) of a panel tile:
// new values s and new predecessors np, with improved flags.  Stores them
// (live tile, snapshot) and returns their bound.  Working one group at a time
// keeps the epilogue's live registers at a quarter of a full micro-tile.
// kSparseP: a row tile too stores the predecessors of its improved entries
// only (the others keep theirs), as "via" codes do not need the full row.
template <typename T, int BS, bool is_row, bool kSparseP = false>
__device__ __forceinline__ int panel_store_group(const Args<T>& a, int r, int t, int g,
                                                 const T (&sv)[Geo<BS>::G][Geo<BS>::TM],
                                                 const int32_t (&np)[Geo<BS>::G][Geo<BS>::TM],
                                                 const bool (&imp)[Geo<BS>::G][Geo<BS>::TM],
                                                 int tx, int ty) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int ti = is_row ? r : t, tj = is_row ? t : r;
  const int slot = r & 1;
  const size_t tile_off = ((size_t)slot * a.slot_tiles + t) * BS * BS;
  // pointers and sizes in registers: read through the reference they would
  // be reloaded after every store (which might alias them)
  T* const D = a.D;
  int32_t* const P = a.P;
  const int64_t n = a.n, ld = a.ld;
  T* const rowR = a.rowR + tile_off;
  int32_t* const rowP = a.rowP + tile_off;
  uint32_t* const rowK = a.rowK + tile_off;
  T* const colR = a.colR;
  uint32_t* const colK = a.colK;
  int nb = 0;
#pragma unroll
  for (int e = 0; e < G; ++e) {
    const int lr = Gm::idx(ty, g * G + e);
    const int64_t gi = (int64_t)ti * BS + lr;
#pragma unroll
    for (int gg = 0; gg < Gm::NG; ++gg) {
      const int lc0 = gg * Gm::SPAN + tx * G;
      const int64_t gj0 = (int64_t)tj * BS + lc0;
      T vs[G];
      int32_t vp[G];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        vs[q] = sv[e][gg * G + q];
        vp[q] = np[e][gg * G + q];
        if constexpr (Num<T>::kPacked) nb = max(nb, bound_of<BS>(vs[q]));
      }
      if (gi < n) {
        if (gj0 + G <= n) {
          vstore<G>(D + gi * ld + gj0, vs);
          if (!P) {
            // distance-only
          } else if constexpr (is_row && !kSparseP) {
            vstore<G>(P + gi * ld + gj0, vp);
          } else {
            bool all = true;
#pragma unroll
            for (int q = 0; q < G; ++q) all &= imp[e][gg * G + q];
            if (all) {
              vstore<G>(P + gi * ld + gj0, vp);  // (early rounds: most groups)
            } else {
#pragma unroll
              for (int q = 0; q < G; ++q)
                if (imp[e][gg * G + q]) P[gi * ld + gj0 + q] = vp[q];
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < G; ++q)
            if (gj0 + q < n) {
              D[gi * ld + gj0 + q] = vs[q];
              if (P && ((is_row && !kSparseP) || imp[e][gg * G + q]))
                P[gi * ld + gj0 + q] = vp[q];
            }
        }
      }
      if constexpr (is_row) {
        // B-form snapshots: raw, pred and packed key (code bits zero)
        vstore<G>(rowR + lr * BS + lc0, vs);
        if constexpr (!ViaPred<T>::kOn) {
          if (P) vstore<G>(rowP + lr * BS + lc0, vp);
        }
        if constexpr (Num<T>::kPacked) {
          uint32_t kq[G];
#pragma unroll
          for (int q = 0; q < G; ++q) kq[q] = key_of<BS>((int32_t)vs[q]);
          vstore<G>(rowK + lr * BS + lc0, kq);
        }
      }
    }
  }
  if constexpr (!is_row) {
    // A-form (transposed) snapshots: raw and packed key with code = column + 1
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) {
      const int lc = Gm::idx(tx, nn);
      const size_t off = tile_off + (size_t)lc * BS + g * Gm::SPAN + ty * G;
      T vs[G];
#pragma unroll
      for (int e = 0; e < G; ++e) vs[e] = sv[e][nn];
      vstore<G>(colR + off, vs);
      if constexpr (Num<T>::kPacked) {
        uint32_t kq[G];
#pragma unroll
        for (int e = 0; e < G; ++e) kq[e] = key_of<BS>((int32_t)vs[e]) + (uint32_t)lc + 1u;
        vstore<G>(colK + off, kq);
      }
    }
  }
  return nb;
}

// Relaxation and epilogue of a panel tile over packed keys (operands already
// in shared memory as keys).  Returns the bound of the new values.
template <typename T, int BS, bool is_row>
__device__ __noinline__ int panel_packed(const Args<T>& a, int r, int t,
                                         const uint32_t* As, const uint32_t* Bs, const int32_t* Ps) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // the tile's own old keys: B-form in Bs for a row tile, A-form in As (with
  // the code of its column) for a column tile
  uint32_t acc[TM][TM];
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int gg = 0; gg < Gm::NG; ++gg) {
      if constexpr (is_row) {
        uint32_t v[G];
        vload_s<G>(v, Bs + Gm::idx(ty, m) * BS + gg * Gm::SPAN + tx * G);
#pragma unroll
        for (int q = 0; q < G; ++q) acc[m][gg * G + q] = v[q];
      }
    }
  if constexpr (!is_row) {
#pragma unroll
    for (int nn = 0; nn < TM; ++nn)
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        uint32_t v[G];
        vload_s<G>(v, As + Gm::idx(tx, nn) * BS + g * Gm::SPAN + ty * G);
#pragma unroll
        for (int e = 0; e < G; ++e) acc[g * G + e][nn] = v[e] & ~K::MASK;
      }
  }
  core_packed<BS>(As, Bs, acc, tx, ty);
  stamp(2);
  // every finite value is below CAP here, so a key decodes exactly and its
  // clamp value can only mean INF
  int nb = 0;
#pragma unroll
  for (int g = 0; g < Gm::NG; ++g) {
    T sv[G][TM];
    int32_t np[G][TM];
    bool imp[G][TM];
#pragma unroll
    for (int e = 0; e < G; ++e) {
      const int m = g * G + e;
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const int lc = Gm::idx(tx, nn);
        const int c = (int)(acc[m][nn] & K::MASK);
        const int32_t v = (int32_t)(acc[m][nn] >> K::KB);
        sv[e][nn] = v == K::CAP ? Num<T>::inf() : (T)v;
        imp[e][nn] = c != 0;
        np[e][nn] = !a.P ? -1 : c ? Ps[(c - 1) * BS + lc] : (is_row ? Ps[Gm::idx(ty, m) * BS + lc] : -1);
      }
    }
    nb = max(nb, panel_store_group<T, BS, is_row>(a, r, t, g, sv, np, imp, tx, ty));
  }
  return nb;
}

// Relaxation and epilogue of a panel tile with an explicit argmin
// (core_generic: fp32, or int32 entries beyond the packed-key bound);
// operands raw in shared memory.
template <typename T, int BS, bool is_row>
__device__ __noinline__ int panel_eager(const Args<T>& a, int r, int t, const T* As,
                                        const T* Bs, const int32_t* Ps) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T s[TM][TM];
  int code[TM][TM];
  if constexpr (is_row) {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int gg = 0; gg < Gm::NG; ++gg) {
        T v[G];
        vload_s<G>(v, Bs + Gm::idx(ty, m) * BS + gg * Gm::SPAN + tx * G);
#pragma unroll
        for (int q = 0; q < G; ++q) s[m][gg * G + q] = v[q];
      }
  } else {
#pragma unroll
    for (int nn = 0; nn < TM; ++nn)
#pragma unroll
      for (int g = 0; g < Gm::NG; ++g) {
        T v[G];
        vload_s<G>(v, As + Gm::idx(tx, nn) * BS + g * Gm::SPAN + ty * G);
#pragma unroll
        for (int e = 0; e < G; ++e) s[g * G + e][nn] = v[e];
      }
  }
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) code[m][nn] = 0;
  core_generic<BS, T>(As, Bs, s, code, tx, ty);
  stamp(2);
  int nb = 0;
#pragma unroll
  for (int g = 0; g < Gm::NG; ++g) {
    T sv[G][TM];
    int32_t np[G][TM];
    bool imp[G][TM];
#pragma unroll
    for (int e = 0; e < G; ++e) {
      const int m = g * G + e;
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const int lc = Gm::idx(tx, nn);
        const int c = code[m][nn];
        sv[e][nn] = s[m][nn];
        imp[e][nn] = c != 0;
        np[e][nn] = !a.P ? -1 : c ? Ps[(c - 1) * BS + lc] : (is_row ? Ps[Gm::idx(ty, m) * BS + lc] : -1);
      }
    }
    nb = max(nb, panel_store_group<T, BS, is_row>(a, r, t, g, sv, np, imp, tx, ty));
  }
  return nb;
}

// Panel tile of round r: a row tile (r, t) when is_row, else a column tile (t, r).
// Row tile:    new[a][b] = min(old[a][b], min_kk Piv[a][kk] + old[kk][b]),
//              pred from the tile's own old pred row kk.
// Column tile: new[a][b] = min(old[a][b], min_kk old[a][kk] + Piv[kk][b]),
//              pred from the pivot's pred row kk.
// With the pivot already closed (phase 1), this product equals the in-place
// sequential update of the blocked FW phases 2 and 3 (Sec. 2.3).  Also writes
// the tile's snapshot (packed keys, raw, pred for row tiles, and its bound)
// into slot r&1.  Shared memory: As | Bs | Ps, three BS x BS tiles; Ps holds
// the predecessor source (own old pred for row tiles, the pivot's for column
// tiles) so that the epilogue gathers from shared memory.
template <typename T, int BS>
__device__ __noinline__ void task_panel(const Args<T>& a, int r, int t, bool is_row, void* smem_raw,
                                        CtaScratch* cs) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM;
  constexpr bool kPacked = Num<T>::kPacked;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int ti = is_row ? r : t, tj = is_row ? t : r;
  const int slot = r & 1;
  // As | Bs: BS*BS elements each (keys or raw values); Ps: BS*BS int32
  unsigned char* sm = reinterpret_cast<unsigned char*>(smem_raw);
  uint32_t* As = reinterpret_cast<uint32_t*>(sm);
  uint32_t* Bs = reinterpret_cast<uint32_t*>(sm + (size_t)BS * BS * sizeof(T));
  int32_t* Ps = reinterpret_cast<int32_t*>(sm + (size_t)2 * BS * BS * sizeof(T));
  stamp(0);

  // predecessor source, staged (its loads overlap the operand loads below)
  if (!a.P) {
    // distance-only: no predecessor source
  } else if (is_row) {
    stage_tile_i32<BS>(Ps, a.P, a.n, a.ld, ti, tj, nullptr);
  } else {
    stage_tile_i32<BS>(Ps, nullptr, 0, 0, 0, 0, a.pivP + (size_t)slot * BS * BS);
  }

  bool fast = false;
  {
    T s[TM][TM], pv[TM][TM];
    load_tile<BS>(s, a.D, a.n, a.ld, ti, tj, tx, ty, Num<T>::inf());
    load_buf<BS>(pv, a.piv + (size_t)slot * BS * BS, tx, ty);
    if constexpr (kPacked) {
      int bs_ = 0, bp_ = 0;
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) {
          bs_ = max(bs_, bound_of<BS>(s[m][nn]));
          bp_ = max(bp_, bound_of<BS>(pv[m][nn]));
        }
      block_max2(bs_, bp_, cs);
      fast = a.packed && (bs_ + bp_ < K::CAP);
    }
    // operands into shared memory: A-form (k-major) on the left, B-form on the right
    if (fast) {
      if constexpr (kPacked) {
        // keys; the A operand carries the code of its column (= kk)
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
          for (int nn = 0; nn < TM; ++nn) {
            const uint32_t code = (uint32_t)Gm::idx(tx, nn) + 1u;
            reinterpret_cast<uint32_t(&)[TM][TM]>(pv)[m][nn] =
                key_of<BS>((int32_t)pv[m][nn]) + (is_row ? code : 0u);
            reinterpret_cast<uint32_t(&)[TM][TM]>(s)[m][nn] =
                key_of<BS>((int32_t)s[m][nn]) + (is_row ? 0u : code);
          }
        if (is_row) {
          put_tile<BS, true>(As, reinterpret_cast<uint32_t(&)[TM][TM]>(pv), tx, ty);
          put_tile<BS, false>(Bs, reinterpret_cast<uint32_t(&)[TM][TM]>(s), tx, ty);
        } else {
          put_tile<BS, true>(As, reinterpret_cast<uint32_t(&)[TM][TM]>(s), tx, ty);
          put_tile<BS, false>(Bs, reinterpret_cast<uint32_t(&)[TM][TM]>(pv), tx, ty);
        }
      }
    } else {
      T* Ast = reinterpret_cast<T*>(As);
      T* Bst = reinterpret_cast<T*>(Bs);
      if (is_row) {
        put_tile<BS, true>(Ast, pv, tx, ty);
        put_tile<BS, false>(Bst, s, tx, ty);
      } else {
        put_tile<BS, true>(Ast, s, tx, ty);
        put_tile<BS, false>(Bst, pv, tx, ty);
      }
    }
  }
  bar_compute();
  stamp(1);

  const T* Ast = reinterpret_cast<const T*>(As);
  const T* Bst = reinterpret_cast<const T*>(Bs);
  int nb;
  if constexpr (kPacked) {
    nb = is_row ? (fast ? panel_packed<T, BS, true>(a, r, t, As, Bs, Ps)
                        : panel_eager<T, BS, true>(a, r, t, Ast, Bst, Ps))
                : (fast ? panel_packed<T, BS, false>(a, r, t, As, Bs, Ps)
                        : panel_eager<T, BS, false>(a, r, t, Ast, Bst, Ps));
  } else {
    nb = is_row ? panel_eager<T, BS, true>(a, r, t, Ast, Bst, Ps)
                : panel_eager<T, BS, false>(a, r, t, Ast, Bst, Ps);
  }
  stamp(3);
  int dummy = 0;
  if constexpr (kPacked) {
    block_max2(nb, dummy, cs);
  } else {
    nb = Keys<BS>::CAP;
  }
  if (tid == 0) {
    int32_t* bnd = is_row ? a.rowB : a.colB;
    bnd[(size_t)slot * a.slot_tiles + t] = nb;
  }
}

// ------------------------------------------------------------- phase 4 ----

// Remaining tile (ti, tj) of round r: D_ij = min(D_ij, A (x) B) with A the
// column-panel snapshot of tile row ti and B the row-panel snapshot of tile
// column tj (Sec. 2.3, blocked FW, phase 4).  Operands arrive by two bulk copies.
// `phase` is the parity of the CTA's operand mbarrier (flipped here).
template <typename T, int BS>
__device__ void task_minplus(const Args<T>& a, int r, int ti, int tj, void* smem_raw,
                             CtaScratch* cs, unsigned& phase) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM;
  constexpr bool kPacked = Num<T>::kPacked;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int slot = r & 1;
  uint32_t* As = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* Bs = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(smem_raw) +
                                             (size_t)BS * BS * sizeof(T));
  const size_t toffA = ((size_t)slot * a.slot_tiles + ti) * BS * BS;
  const size_t toffB = ((size_t)slot * a.slot_tiles + tj) * BS * BS;

  bool fast = false;
  if constexpr (kPacked) {
    if (a.packed) {
      const int ba = __ldcg(a.colB + (size_t)slot * a.slot_tiles + ti);
      const int bb = __ldcg(a.rowB + (size_t)slot * a.slot_tiles + tj);
      fast = ba + bb < K::CAP;
    }
  }
  if (tid == 0) {
    constexpr unsigned bytes = BS * BS * sizeof(T);
    fence_proxy_async();
    mbar_expect_tx(&cs->bar, 2 * bytes);
    const void* srcA = fast ? (const void*)(a.colK + toffA) : (const void*)(a.colR + toffA);
    const void* srcB = fast ? (const void*)(a.rowK + toffB) : (const void*)(a.rowR + toffB);
    bulk_g2s(As, srcA, bytes, &cs->bar);
    bulk_g2s(Bs, srcB, bytes, &cs->bar);
  }
  T old[TM][TM];
  load_tile<BS>(old, a.D, a.n, a.ld, ti, tj, tx, ty, Num<T>::inf());
  {
    // wait for the operands (bounded: a copy that never lands is reported, not hung on)
    const uint64_t t0 = globaltimer();
    int64_t it = 0;
    while (!mbar_try_wait(&cs->bar, phase)) {
      if (globaltimer() - t0 > (uint64_t)a.timeout_ns || ++it > (int64_t)1 << 26) {
        if (tid == 0) atomicOr(a.status, kStTimeout);
        break;
      }
    }
    phase ^= 1u;
  }

  int32_t* rowP = a.rowP + toffB;
  bool neg = false;
  if (kPacked && fast) {
    uint32_t acc[TM][TM];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) acc[m][nn] = kPacked ? key_of<BS>((int32_t)old[m][nn]) : 0u;
    core_packed<BS>(As, Bs, acc, tx, ty);
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      const int64_t gi = (int64_t)ti * BS + Gm::idx(ty, m);
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const uint32_t c = acc[m][nn] & K::MASK;
        const int64_t gj = (int64_t)tj * BS + Gm::idx(tx, nn);
        if (c && gi < a.n && gj < a.n) {
          const int32_t nv = (int32_t)(acc[m][nn] >> K::KB);
          a.D[gi * a.ld + gj] = (T)nv;
          if (a.P) a.P[gi * a.ld + gj] = ViaPred<T>::kOn
                                    ? via_code((int64_t)r * BS + c - 1)
                                    : __ldcg(rowP + (c - 1) * BS + Gm::idx(tx, nn));
          if (gi == gj && nv < 0) neg = true;
        }
      }
    }
  } else {
    int arg[TM][TM];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) arg[m][nn] = 0;
    core_generic<BS, T>(reinterpret_cast<const T*>(As), reinterpret_cast<const T*>(Bs), old, arg,
                        tx, ty);
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      const int64_t gi = (int64_t)ti * BS + Gm::idx(ty, m);
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const int64_t gj = (int64_t)tj * BS + Gm::idx(tx, nn);
        if (arg[m][nn] && gi < a.n && gj < a.n) {
          a.D[gi * a.ld + gj] = old[m][nn];
          if (a.P) a.P[gi * a.ld + gj] = ViaPred<T>::kOn
                                    ? via_code((int64_t)r * BS + arg[m][nn] - 1)
                                    : __ldcg(rowP + (arg[m][nn] - 1) * BS + Gm::idx(tx, nn));
          if (gi == gj && old[m][nn] < T(0)) neg = true;
        }
      }
    }
  }
  if (neg) atomicOr(a.status, kStNegCycle);
}

// ------------------------------------------------------------------ init ----

// pred[i][j] = i where the edge i -> j exists (i != j), else -1.
template <typename T>
__global__ void __launch_bounds__(256) k_init_pred(const T* __restrict__ D, int32_t* __restrict__ P,
                                                   int64_t n, int64_t ld) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const T w = D[i * ld + j];
    P[i * ld + j] = (i != j && Num<T>::finite(w)) ? (int32_t)i : -1;
  }
}

// Final pass of an int32 solve: every via code becomes the last hop its chain
// ends in (see ViaPred).  A chain stays in its column, so the matrix is swept
// in slabs of kResolveSlab columns, every CTA walking the slabs in the same
// order: the random reads of a chain then hit the L2-resident slab instead of
// DRAM.  Each warp takes one row segment of the slab (a 16-byte vector per
// lane).  In place: a concurrent reader of an entry sees either its via code
// or the last hop that code resolves to, and follows either to the same end.
constexpr int kResolveSlab = 128;
static __global__ void __launch_bounds__(256) k_resolve_pred(int32_t* P, int64_t n, int64_t ld) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = 0; c0 < n; c0 += kResolveSlab) {
    const int64_t j = c0 + lane * 4;
    if (j >= n) continue;
    for (int64_t i = warp; i < n; i += nwarps) {
      int32_t* row = P + i * ld;
      if (j + 4 <= n) {
        int4 v = *reinterpret_cast<int4*>(row + j);
        if (min(min(v.x, v.y), min(v.z, v.w)) >= -1) continue;  // no via code here
        v.x = resolve_pred(v.x, P, ld, j);
        v.y = resolve_pred(v.y, P, ld, j + 1);
        v.z = resolve_pred(v.z, P, ld, j + 2);
        v.w = resolve_pred(v.w, P, ld, j + 3);
        *reinterpret_cast<int4*>(row + j) = v;
      } else {
        for (int64_t jj = j; jj < n; ++jj) {
          const int32_t p = row[jj];
          if (p <= -2) row[jj] = resolve_pred(p, P, ld, jj);
        }
      }
    }
  }
}

}  // namespace fwk
