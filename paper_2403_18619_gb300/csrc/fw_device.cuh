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

// Barrier over the 256 compute threads (warps 0-7).  In kernels that add a
// producer warp, that warp does not take part; in 256-thread kernels this is
// the whole CTA.
__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

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

// Packed-key parameters: KB bits hold the code kk+1 (1..BS), CAP bounds the
// distance part so that key(A) + key(B) never wraps a uint32.
template <int BS>
struct Keys {
  static constexpr int KB = (BS == 128) ? 8 : (BS == 64) ? 7 : 6;
  static constexpr uint32_t MASK = (1u << KB) - 1u;
  static constexpr int CAP = (1 << (31 - KB)) - 1;
  static_assert((1 << (KB - 1)) == BS, "BS must be 32, 64 or 128");
};

template <typename T>
struct Num;
template <>
struct Num<int32_t> {
  static constexpr bool kInt = true;
  __device__ __forceinline__ static int32_t inf() { return 1 << 29; }
  __device__ __forceinline__ static bool finite(int32_t v) { return v < (1 << 29); }
};
template <>
struct Num<float> {
  static constexpr bool kInt = false;
  __device__ __forceinline__ static float inf() { return __int_as_float(0x7f800000); }
  __device__ __forceinline__ static bool finite(float v) { return v < __int_as_float(0x7f800000); }
};

// Vector load / store of G consecutive 32-bit elements.
template <int G, typename T>
__device__ __forceinline__ void vload_cg(T (&dst)[G], const T* src) {
  if constexpr (G == 4) {
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
  if constexpr (G == 4) {
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
  if constexpr (G == 4) {
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
  // optional per-task trace (persistent driver)
  uint64_t* trace;
  int trace_cap;
  int trace_stride;
};

// -------------------------------------------------------- shared memory ----

template <int BS>
struct Smem {
  static constexpr int kTile = BS * BS;
  // As and Bs are BS*BS 32-bit words each; the pivot task reuses As for its
  // row / column broadcast buffers.
  static constexpr size_t bytes() { return (size_t)2 * kTile * 4 + 256; }
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
  if constexpr (Num<T>::kInt) {
    if (!Num<T>::finite(v)) return 0;
    return v < 0 ? Keys<BS>::CAP : min((int)v, Keys<BS>::CAP);
  } else {
    return Keys<BS>::CAP;
  }
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
#pragma unroll 2
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

// Generic relaxation with an explicit first-argmin: s = A + B; if (s < acc)
// { acc = s; arg = kk + 1 }.  Used for fp32 and for int32 tiles whose values
// exceed the packed-key bound.
template <int BS, typename T, int K = BS>
__device__ __forceinline__ void core_generic(const T* __restrict__ As, const T* __restrict__ Bs,
                                             T (&acc)[Geo<BS>::TM][Geo<BS>::TM],
                                             int (&arg)[Geo<BS>::TM][Geo<BS>::TM], int tx, int ty,
                                             int kk0 = 0) {
  using Gm = Geo<BS>;
  constexpr int G = Gm::G, TM = Gm::TM;
#pragma unroll 1
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
        bool lt = s < acc[m][nn];
        acc[m][nn] = lt ? s : acc[m][nn];
        arg[m][nn] = lt ? kk0 + kk + 1 : arg[m][nn];
      }
  }
}

// ------------------------------------------------------------- phase 1 ----

// Pivot tile (r,r): in-place FW over the vertices of block r (Sec. 2.3, blocked FW,
// phase 1).  Each step kk broadcasts row kk and column kk through shared
// memory (double-buffered, one barrier per step) and relaxes every owned
// element through kk with an eager strict-< predecessor update.  Writes the
// live tile and the pivot snapshot of slot r&1.
template <typename T, int BS>
__device__ __noinline__ void task_pivot(const Args<T>& a, int r, void* smem_raw, CtaScratch* cs) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM, G = Gm::G;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T d[TM][TM];
  int32_t p[TM][TM];
  load_tile<BS>(d, a.D, a.n, a.ld, r, r, tx, ty, Num<T>::inf());
  load_tile<BS>(p, a.P, a.n, a.ld, r, r, tx, ty, (int32_t)-1);

  T* rowD = reinterpret_cast<T*>(smem_raw);           // [2][BS]
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
            bool lt = s < d[mm][nn];
            d[mm][nn] = lt ? s : d[mm][nn];
            p[mm][nn] = lt ? rp[nn] : p[mm][nn];
          }
      }
    }
  }
  // negative cycle: a negative diagonal entry
  bool neg = false;
#pragma unroll
  for (int mm = 0; mm < TM; ++mm)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn)
      if (Gm::idx(ty, mm) == Gm::idx(tx, nn) && d[mm][nn] < T(0)) neg = true;
  if (neg) atomicOr(a.status, kStNegCycle);

  store_tile<BS>(a.D, d, a.n, a.ld, r, r, tx, ty);
  store_tile<BS>(a.P, p, a.n, a.ld, r, r, tx, ty);
  const int slot = r & 1;
  put_tile<BS, false>(a.piv + (size_t)slot * BS * BS, d, tx, ty);
  put_tile<BS, false>(a.pivP + (size_t)slot * BS * BS, p, tx, ty);
}

// ------------------------------------------------------------- phase 2/3 ----

// Panel tile of round r: a row tile (r, t) when kRow, else a column tile (t, r).
// Row tile:    new[a][b] = min(old[a][b], min_kk Piv[a][kk] + old[kk][b]),
//              pred from the tile's own old pred row kk.
// Column tile: new[a][b] = min(old[a][b], min_kk old[a][kk] + Piv[kk][b]),
//              pred from the pivot's pred row kk.
// With the pivot already closed (phase 1), this product equals the in-place
// sequential update of the blocked FW phases 2 and 3 (Sec. 2.3).  Also writes the tile's
// snapshot (packed keys, raw, pred for row tiles, and its bound) into slot r&1.
template <typename T, int BS>
__device__ __noinline__ void task_panel(const Args<T>& a, int r, int t, bool is_row, void* smem_raw,
                           CtaScratch* cs) {
  using Gm = Geo<BS>;
  using K = Keys<BS>;
  constexpr int TM = Gm::TM;
  constexpr bool kInt = Num<T>::kInt;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int ti = is_row ? r : t, tj = is_row ? t : r;
  const int slot = r & 1;
  uint32_t* As = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* Bs = As + BS * BS;

  T s[TM][TM], pv[TM][TM];
  load_tile<BS>(s, a.D, a.n, a.ld, ti, tj, tx, ty, Num<T>::inf());
  {
    const T* piv = a.piv + (size_t)slot * BS * BS;
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn)
        pv[m][nn] = __ldcg(piv + Gm::idx(ty, m) * BS + Gm::idx(tx, nn));
  }
  int bs_ = 0, bp_ = 0;
  if constexpr (kInt) {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        bs_ = max(bs_, bound_of<BS>(s[m][nn]));
        bp_ = max(bp_, bound_of<BS>(pv[m][nn]));
      }
    block_max2(bs_, bp_, cs);
  }
  const bool fast = kInt && a.packed && (bs_ + bp_ < K::CAP);

  // operands into shared memory: A-form (k-major) on the left, B-form on the right
  if (fast) {
    uint32_t ks[TM][TM], kp[TM][TM];
    if constexpr (kInt) {
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) {
          const uint32_t code = (uint32_t)Gm::idx(tx, nn) + 1u;  // column index = kk for A-form
          ks[m][nn] = key_of<BS>((int32_t)s[m][nn]) + (is_row ? 0u : code);
          kp[m][nn] = key_of<BS>((int32_t)pv[m][nn]) + (is_row ? code : 0u);
        }
    }
    if (is_row) {
      put_tile<BS, true>(As, kp, tx, ty);
      put_tile<BS, false>(Bs, ks, tx, ty);
    } else {
      put_tile<BS, true>(As, ks, tx, ty);
      put_tile<BS, false>(Bs, kp, tx, ty);
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
  bar_compute();

  // relax; afterwards s[][] holds the new values and code[][] the argmin + 1 (0 = unchanged)
  int code[TM][TM];
  if (fast) {
    uint32_t acc[TM][TM];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) acc[m][nn] = kInt ? key_of<BS>((int32_t)s[m][nn]) : 0u;
    core_packed<BS>(As, Bs, acc, tx, ty);
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        code[m][nn] = (int)(acc[m][nn] & K::MASK);
        if (code[m][nn]) s[m][nn] = (T)(int32_t)(acc[m][nn] >> K::KB);
      }
  } else {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) code[m][nn] = 0;
    core_generic<BS, T>(reinterpret_cast<const T*>(As), reinterpret_cast<const T*>(Bs), s, code,
                        tx, ty);
  }

  // predecessors: gather every value first, then write (a row tile reads its own old pred)
  int32_t np[TM][TM];
  {
    const int32_t* pivP = a.pivP + (size_t)slot * BS * BS;
#pragma unroll
    for (int m = 0; m < TM; ++m) {
      const int64_t gi = (int64_t)ti * BS + Gm::idx(ty, m);
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) {
        const int64_t gj = (int64_t)tj * BS + Gm::idx(tx, nn);
        const bool in = gi < a.n && gj < a.n;
        int32_t old = in ? __ldcg(a.P + gi * a.ld + gj) : -1;
        if (code[m][nn] && in) {
          const int kk = code[m][nn] - 1;
          if (is_row) {
            const int64_t gk = (int64_t)r * BS + kk;   // row kk of this tile
            old = gk < a.n ? __ldcg(a.P + gk * a.ld + gj) : -1;
          } else {
            old = __ldcg(pivP + kk * BS + Gm::idx(tx, nn));
          }
        }
        np[m][nn] = old;
      }
    }
  }
  bar_compute();
  store_tile<BS>(a.D, s, a.n, a.ld, ti, tj, tx, ty);
  store_tile<BS>(a.P, np, a.n, a.ld, ti, tj, tx, ty);

  // snapshot for phase 4 of this round
  int nb = 0, dummy = 0;
  if constexpr (kInt) {
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) nb = max(nb, bound_of<BS>(s[m][nn]));
  }
  const size_t tile_off = ((size_t)slot * a.slot_tiles + t) * BS * BS;
  if (is_row) {
    put_tile<BS, false>(a.rowR + tile_off, s, tx, ty);
    put_tile<BS, false>(a.rowP + tile_off, np, tx, ty);
    if constexpr (kInt) {
      uint32_t k[TM][TM];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn) k[m][nn] = key_of<BS>((int32_t)s[m][nn]);
      put_tile<BS, false>(a.rowK + tile_off, k, tx, ty);
    }
  } else {
    put_tile<BS, true>(a.colR + tile_off, s, tx, ty);
    if constexpr (kInt) {
      uint32_t k[TM][TM];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int nn = 0; nn < TM; ++nn)
          k[m][nn] = key_of<BS>((int32_t)s[m][nn]) + (uint32_t)Gm::idx(tx, nn) + 1u;
      put_tile<BS, true>(a.colK + tile_off, k, tx, ty);
    }
  }
  if constexpr (kInt) {
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
  constexpr bool kInt = Num<T>::kInt;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int slot = r & 1;
  uint32_t* As = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* Bs = As + BS * BS;
  const size_t toffA = ((size_t)slot * a.slot_tiles + ti) * BS * BS;
  const size_t toffB = ((size_t)slot * a.slot_tiles + tj) * BS * BS;

  bool fast = false;
  if constexpr (kInt) {
    if (a.packed) {
      const int ba = __ldcg(a.colB + (size_t)slot * a.slot_tiles + ti);
      const int bb = __ldcg(a.rowB + (size_t)slot * a.slot_tiles + tj);
      fast = ba + bb < K::CAP;
    }
  }
  if (tid == 0) {
    constexpr unsigned bytes = BS * BS * 4;
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
  if (fast) {
    uint32_t acc[TM][TM];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) acc[m][nn] = kInt ? key_of<BS>((int32_t)old[m][nn]) : 0u;
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
          a.P[gi * a.ld + gj] = __ldcg(rowP + (c - 1) * BS + Gm::idx(tx, nn));
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
          a.P[gi * a.ld + gj] = __ldcg(rowP + (arg[m][nn] - 1) * BS + Gm::idx(tx, nn));
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

}  // namespace fwk
