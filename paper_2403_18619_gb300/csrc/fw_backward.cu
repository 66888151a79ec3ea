// Backward pass of the fp32 solve: dL/dW from dL/dD through the predecessor
// trees (not part of the paper; it lets a training graph differentiate
// through all-pairs shortest distances).
//
// For source i the recorded paths form a tree with edges pred[i][v] -> v.
// D[i][j] is the sum of the weights on the tree path i -> j, so
//     E[i][v]      = sum of dL/dD[i][j] over j in the subtree of v
//                  = dL/dD[i][v] + sum over tree children c of E[i][c]
//     dL/dW[u][v]  = sum over sources i with pred[i][v] == u of E[i][v].
//
// Both sums are formed EXACTLY in 64-bit fixed point: a value x becomes the
// integer round(x / 2^e), with 2^e chosen so that the largest possible sum
// (the sum of |dL/dD| over the row, or over the graph) stays below 2^61.
// Integer addition is associative, so the result does not depend on the order
// in which the terms arrive: every run gives bit-identical gradients without
// sorting the terms, and the only rounding is the conversion of each input
// term and of the final sum.
//
// Kernel 1 (one CTA per source row, the row owned by that CTA): hop depth of
// every vertex by pointer jumping on packed (ancestor, hop count) words; then
// the levels from the deepest up, every vertex adding its subtree sum into
// its parent's (shared-memory integer adds).  Writes E[i][.] as fp32 and the
// row's sum of |dL/dD|.
// Kernel 2 (one CTA per block of C consecutive columns of one graph): reads
// pred and E in row segments of C entries (whole 32-byte sectors for C = 8),
// adds each E[i][v] into the fixed-point accumulator of (pred[i][v], v), and
// writes the C columns of dL/dW.  No global atomics anywhere; pred == -1 marks
// the diagonal and unreachable pairs, so dist is not read.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_internal.h"

namespace {

// 128 threads per source row: 16 rows per SM fill its 2048 threads within the
// shared memory (0.79 ms for the 64 x 1024 workload; 256 threads 0.86 ms, 512
// threads 1.10 ms); 256 per column block (512: 0.90 ms)
constexpr int kRowThreads = 128;
constexpr int kColThreads = 256;
// Kernel 1 keeps 14 bytes per vertex in shared memory (the accumulator, a
// packed ancestor / hop-count word and the parent): n <= 11264 keeps it under
// 227 KB with room to spare; the 16-bit fields take n <= 32767.
constexpr int64_t kMaxN = 11264;
constexpr size_t kColSmem = 64 * 1024;  // kernel 2 accumulators (C x n x 8 bytes)

// Sum of one float per thread over the CTA in a fixed order (the same tree
// every run): warp butterflies, then the warp partials in warp order.
template <int kT>
__device__ __forceinline__ float block_sum(float x, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  float s = 0.0f;
#pragma unroll
  for (int w = 0; w < kT / 32; ++w) s += red[w];
  return s;
}

// Fixed point.  Every conversion is integer arithmetic on the fp32 fields:
// GB300's FP64 pipe (about 1.7 operations per SM clock) would otherwise set
// the pace of both kernels.
//
// Quantum exponent e for sums whose magnitude is at most `bound`, where bound
// is an fp32 sum of absolute values (so the exact sum is below 2 * bound):
// with e = floor(log2(bound)) - 59, every partial sum stays below 2^61.
__device__ __forceinline__ int quantum_exp(float bound) {
  const int be = (int)((__float_as_uint(bound) >> 23) & 0xffu);
  return (be ? be - 127 : -127) - 59;
}

// round(x / 2^e) for a finite fp32 x (round half up in magnitude).
__device__ __forceinline__ long long to_fixed(float x, int e) {
  const unsigned u = __float_as_uint(x);
  const int be = (int)((u >> 23) & 0xffu);
  const unsigned m = (u & 0x7fffffu) | (be ? 0x800000u : 0u);  // x = m * 2^(max(be,1) - 150)
  const int sh = (be ? be : 1) - 150 - e;
  long long r = 0;
  if (be != 255 && m != 0) {
    if (sh >= 0) r = (long long)m << (sh > 38 ? 38 : sh);
    else if (sh > -25) r = (long long)((m + (1u << (-sh - 1))) >> (-sh));
  }
  return (u >> 31) ? -r : r;
}

// 2^k as fp32 for k in [-126, 127].
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(k + 127) << 23); }

// a * 2^e as fp32: the integer rounded once to 24 bits (nearest, ties to
// even), then scaled by two exact powers of two (only a result below the
// normal range rounds again).
__device__ __forceinline__ float from_fixed(long long a, int e) {
  if (a == 0) return 0.0f;
  const unsigned long long m = a < 0 ? (unsigned long long)(-a) : (unsigned long long)a;
  int top = 63 - __clzll((long long)m);  // leading bit
  unsigned q;
  if (top <= 23) {
    q = (unsigned)m << (23 - top);
  } else {
    const int sh = top - 23;
    const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    q = (unsigned)(m >> sh);
    if (rem > half || (rem == half && (q & 1u))) ++q;
    if (q == (1u << 24)) { q >>= 1; ++top; }
  }
  float f = __uint_as_float(((unsigned)(top + 127) << 23) | (q & 0x7fffffu));
  const int e1 = e >> 1, e2 = e - e1;  // both within [-126, 127] for fp32 sums
  f = f * pow2f(e1) * pow2f(e2);
  return a < 0 ? -f : f;
}

// acc += x for a 64-bit fixed-point accumulator in shared memory, as two
// native 32-bit atomic adds: the low word's add returns the old value, which
// gives its carry into the high word.  Every carry is counted once, so the
// final 64-bit value is the exact sum in any order.  (A 64-bit add would
// retry a compare-and-swap under contention, and many vertices share a
// parent, many sources a last hop.)
__device__ __forceinline__ void add_fixed(long long* acc, long long x) {
  unsigned* w = reinterpret_cast<unsigned*>(acc);  // little-endian: w[0] low, w[1] high
  const unsigned xl = (unsigned)x, xh = (unsigned)((unsigned long long)x >> 32);
  const unsigned old = atomicAdd(w, xl);
  const unsigned hi = xh + ((unsigned)(old + xl) < old ? 1u : 0u);
  if (hi) atomicAdd(w + 1, hi);
}

// Packed pointer-jumping word: ancestor (16 bits, 0xffff = none) and hop count.
__device__ __forceinline__ unsigned pack(int anc, int dist) {
  return ((unsigned)dist << 16) | ((unsigned)anc & 0xffffu);
}
__device__ __forceinline__ int anc_of(unsigned w) { return (w & 0xffffu) == 0xffffu ? -1 : (int)(w & 0xffffu); }
__device__ __forceinline__ int dist_of(unsigned w) { return (int)(w >> 16); }

// Kernel 1: subtree sums of source row i of graph b (block b * n + i).
__global__ void __launch_bounds__(kRowThreads) k_bwd_rows(const float* __restrict__ G,
                                                          const int32_t* __restrict__ P,
                                                          float* __restrict__ E,
                                                          float* __restrict__ Srow, int64_t n,
                                                          int64_t ld, int64_t stride) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int nn = (int)n;
  long long* acc = reinterpret_cast<long long*>(sm);           // n
  unsigned* jw = reinterpret_cast<unsigned*>(acc + nn);        // n: (ancestor, hops)
  unsigned short* par = reinterpret_cast<unsigned short*>(jw + nn);  // n: parent
  __shared__ float red[kRowThreads / 32];
  __shared__ int wmax[kRowThreads / 32];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x / n, i = blockIdx.x % n;
  const int64_t off = b * stride + i * ld;

  // parents (none: the root, unreachable vertices, invalid entries), the
  // adjoints parked in the accumulators, and the row's sum of |dL/dD|
  float sabs = 0.0f;
  for (int v = tid; v < nn; v += kRowThreads) {
    const int p = __ldcs(P + off + v);
    const float g = __ldcs(G + off + v);
    const bool tree = v != i && p >= 0 && p < nn && p != v;
    jw[v] = pack(tree ? p : -1, tree ? 1 : 0);
    par[v] = (unsigned short)(tree ? p : 0);
    acc[v] = tree ? (long long)__float_as_uint(g) : 0ll;
    if (tree) sabs += fabsf(g);
  }
  sabs = block_sum<kRowThreads>(sabs, red);  // (its barriers also order the stores above)
  const int e = quantum_exp(sabs);
  for (int v = tid; v < nn; v += kRowThreads)
    acc[v] = to_fixed(__uint_as_float((unsigned)acc[v]), e);

  // hop depth by pointer jumping, in place: every word holds an ancestor and
  // the hop count to it, read and written as one 32-bit access, so a thread
  // always combines a consistent pair even while other words advance in the
  // same round.  At most ceil(log2(n)) + 1 rounds (more only for an invalid
  // pred with a cycle, which the round cap stops).
  __syncthreads();
  for (int round = 0; (1 << round) <= 2 * nn; ++round) {
    bool moved = false;
    for (int v = tid; v < nn; v += kRowThreads) {
      const unsigned w = jw[v];
      const int a = anc_of(w);
      if (a >= 0) {
        const unsigned wa = jw[a];
        jw[v] = pack(anc_of(wa), dist_of(w) + dist_of(wa));
        moved = true;
      }
    }
    if (!__syncthreads_or(moved)) break;
  }
  int dmax = 0;
  for (int v = tid; v < nn; v += kRowThreads) dmax = max(dmax, dist_of(jw[v]));
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  if ((tid & 31) == 0) wmax[tid >> 5] = dmax;
  __syncthreads();
  dmax = 0;
#pragma unroll
  for (int w = 0; w < kRowThreads / 32; ++w) dmax = max(dmax, wmax[w]);
  if (dmax > nn) dmax = nn;

  // deepest level first: a vertex at depth L is complete once level L+1 has
  // been added, and adds its sum to its parent (exact integer adds: the order
  // within a level does not matter).  Depth 1 adds nothing: its parent is the
  // source, whose own sum is not used.
  for (int L = dmax; L >= 2; --L) {
    for (int v = tid; v < nn; v += kRowThreads)
      if (dist_of(jw[v]) == L) add_fixed(acc + par[v], acc[v]);
    __syncthreads();
  }
  for (int v = tid; v < nn; v += kRowThreads)
    E[off + v] = dist_of(jw[v]) > 0 ? from_fixed(acc[v], e) : 0.0f;
  if (tid == 0) Srow[blockIdx.x] = sabs;
}

// Kernel 2: columns [v0, v0 + C) of dL/dW of graph b (C = kC).
template <int kC>
__global__ void __launch_bounds__(kColThreads) k_bwd_cols(const float* __restrict__ E,
                                                          const int32_t* __restrict__ P,
                                                          const float* __restrict__ Srow,
                                                          float* __restrict__ GW, int64_t n,
                                                          int64_t ld, int64_t stride,
                                                          int64_t blocks_per_graph) {
  extern __shared__ __align__(16) unsigned char sm[];
  long long* acc = reinterpret_cast<long long*>(sm);  // [u][c], c fastest
  __shared__ float red[kColThreads / 32];
  const int tid = threadIdx.x;
  const int nn = (int)n;
  const int64_t b = blockIdx.x / blocks_per_graph;
  const int v0 = (int)(blockIdx.x % blocks_per_graph) * kC;
  const int64_t base = b * stride;
  // the graph's bound: the sum of every row's sum of |dL/dD| (fixed order)
  float s = 0.0f;
  for (int r = tid; r < nn; r += kColThreads) s += Srow[b * n + r];
  s = block_sum<kColThreads>(s, red);
  const int e = quantum_exp(s);
  const int total = nn * kC;
  for (int q = tid; q < total; q += kColThreads) acc[q] = 0;
  __syncthreads();
  // row segments of kC columns: consecutive threads read consecutive columns;
  // four entries per thread are loaded before any of them is added
  constexpr int kU = 4;
  for (int q0 = tid; q0 < total; q0 += kU * kColThreads) {
    int u[kU];
    float x[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int q = q0 + k * kColThreads;
      const int r = q / kC, c = q - r * kC, v = v0 + c;
      u[k] = -1;
      x[k] = 0.0f;
      if (q < total && v < nn && r != v) {
        u[k] = __ldcs(P + base + (int64_t)r * ld + v);
        x[k] = __ldcs(E + base + (int64_t)r * ld + v);
      }
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int q = q0 + k * kColThreads;
      const int c = q % kC, v = v0 + c;
      if (u[k] < 0 || u[k] >= nn || u[k] == v) continue;
      add_fixed(acc + (size_t)u[k] * kC + c, to_fixed(x[k], e));
    }
  }
  __syncthreads();
  for (int q = tid; q < total; q += kColThreads) {
    const int u = q / kC, c = q - u * kC;
    const int v = v0 + c;
    if (v >= nn) continue;
    GW[base + (int64_t)u * ld + v] = u == v ? 0.0f : from_fixed(acc[q], e);
  }
}

size_t rows_smem(int64_t n) { return (size_t)n * 14; }

template <int kC>
fw_status launch_cols(const float* E, const int32_t* P, const float* S, float* GW, int64_t n,
                      int64_t ld, int64_t st, int64_t batch, cudaStream_t s) {
  auto kern = k_bwd_cols<kC>;
  const size_t smem = (size_t)n * kC * 8;
  if (fwh::kernel_setup(reinterpret_cast<const void*>(kern), kColSmem, kColThreads) < 1)
    return FW_ERR_CUDA;
  const int64_t per = (n + kC - 1) / kC;
  kern<<<(unsigned)(per * batch), kColThreads, smem, s>>>(E, P, S, GW, n, ld, st, per);
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

}  // namespace

namespace fwh {
void* backward_scratch(cudaStream_t s, size_t bytes);  // fw_api.cu
}

extern "C" {

fw_status fw_backward_strided(const float* grad_dist, const float* dist, const int32_t* pred,
                              float* grad_w, int64_t n, int64_t ld, int64_t batch, int64_t stride,
                              void* stream) {
  if (!grad_dist || !dist || !pred || !grad_w) return FW_ERR_ARG;
  if (n <= 0 || ld < n || batch < 1 || (batch > 1 && stride < n * ld)) return FW_ERR_ARG;
  if (n > kMaxN) return FW_ERR_UNSUPPORTED;
  if (n * batch > ((int64_t)1 << 31) - 1) return FW_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t st = batch > 1 ? stride : n * ld;
  // scratch: E (batch x st fp32), then the per-row sums of |dL/dD|
  const size_t e_bytes = ((size_t)(batch * st) * 4 + 255) / 256 * 256;
  unsigned char* scratch = reinterpret_cast<unsigned char*>(
      fwh::backward_scratch(s, e_bytes + (size_t)(batch * n) * 4));
  if (!scratch) return FW_ERR_NOMEM;
  float* E = reinterpret_cast<float*>(scratch);
  float* S = reinterpret_cast<float*>(scratch + e_bytes);
  if (fwh::kernel_setup(reinterpret_cast<const void*>(k_bwd_rows), rows_smem(kMaxN), kRowThreads) < 1)
    return FW_ERR_CUDA;
  k_bwd_rows<<<(unsigned)(n * batch), kRowThreads, rows_smem(n), s>>>(grad_dist, pred, E, S, n,
                                                                       ld, st);
  if (cudaGetLastError() != cudaSuccess) return FW_ERR_CUDA;
  // as many columns per CTA as 64 KB of accumulators allow (8 = one 32-byte
  // sector per row segment; 64 KB keeps three CTAs on an SM)
  if (n * 8 * 8 <= (int64_t)kColSmem) return launch_cols<8>(E, pred, S, grad_w, n, ld, st, batch, s);
  if (n * 4 * 8 <= (int64_t)kColSmem) return launch_cols<4>(E, pred, S, grad_w, n, ld, st, batch, s);
  if (n * 2 * 8 <= (int64_t)kColSmem) return launch_cols<2>(E, pred, S, grad_w, n, ld, st, batch, s);
  return launch_cols<1>(E, pred, S, grad_w, n, ld, st, batch, s);
}

fw_status fw_backward(const float* grad_dist, const float* dist, const int32_t* pred,
                      float* grad_w, int64_t n, int64_t ld, void* stream) {
  return fw_backward_strided(grad_dist, dist, pred, grad_w, n, ld, 1, n * ld, stream);
}

}  // extern "C"
