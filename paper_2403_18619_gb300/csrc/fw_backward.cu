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
// every vertex by pointer jumping on packed (ancestor, distance) words; then
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

constexpr int kRowThreads = 256;
constexpr int kColThreads = 256;
// Kernel 1 keeps 20 bytes per vertex in shared memory (accumulator, parent,
// packed ancestor / distance): n <= 11264 fits the 227 KB of one CTA.
constexpr int64_t kMaxN = 11264;
constexpr size_t kColSmem = 128 * 1024;  // kernel 2 accumulators (C x n x 8 bytes)

// Sum of one double per thread over the CTA in a fixed order (the same tree
// every run): warp butterflies, then the warp partials in warp order.
template <int kT>
__device__ __forceinline__ double block_sum(double x, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kT / 32; ++w) s += red[w];
  return s;
}

// Exponent e of the fixed-point quantum 2^e for sums bounded by `bound`:
// bound / 2^e < 2^61.  (bound is a sum of |fp32| values: e stays far inside
// the double range.)
__device__ __forceinline__ int quantum_exp(double bound) {
  int ex = 0;
  frexp(bound, &ex);  // bound = f * 2^ex, f in [0.5, 1); 0 for bound = 0
  return ex - 61;
}

__device__ __forceinline__ unsigned long long pack(int anc, int dist) {
  return ((unsigned long long)(unsigned)dist << 32) | (unsigned)anc;
}
__device__ __forceinline__ int anc_of(unsigned long long w) { return (int)(unsigned)w; }
__device__ __forceinline__ int dist_of(unsigned long long w) { return (int)(w >> 32); }

// Kernel 1: subtree sums of source row i of graph b (block b * n + i).
__global__ void __launch_bounds__(kRowThreads) k_bwd_rows(const float* __restrict__ G,
                                                          const int32_t* __restrict__ P,
                                                          float* __restrict__ E,
                                                          double* __restrict__ Srow, int64_t n,
                                                          int64_t ld, int64_t stride) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int nn = (int)n;
  long long* acc = reinterpret_cast<long long*>(sm);                  // n
  unsigned long long* jw = reinterpret_cast<unsigned long long*>(acc + nn);  // n: (anc, dist)
  int* par = reinterpret_cast<int*>(jw + nn);                         // n
  __shared__ double red[kRowThreads / 32];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x / n, i = blockIdx.x % n;
  const int64_t off = b * stride + i * ld;

  // parents (-1: the root, unreachable vertices, invalid entries) and sum |G|
  double sabs = 0.0;
  for (int v = tid; v < nn; v += kRowThreads) {
    const int p = P[off + v];
    const bool tree = v != i && p >= 0 && p < nn && p != v;
    par[v] = tree ? p : -1;
    jw[v] = pack(tree ? p : -1, tree ? 1 : 0);
    if (tree) sabs += fabs((double)G[off + v]);
  }
  sabs = block_sum<kRowThreads>(sabs, red);
  const int e = quantum_exp(sabs);
  const double to_fix = ldexp(1.0, -e);
  for (int v = tid; v < nn; v += kRowThreads)
    acc[v] = par[v] >= 0 ? __double2ll_rn((double)G[off + v] * to_fix) : 0ll;

  // hop depth by pointer jumping, in place: every word holds an ancestor and
  // the hop count to it, read and written as one 64-bit access, so a thread
  // always combines a consistent pair even while other words advance in the
  // same round.  At most ceil(log2(n)) + 1 rounds (more only for an invalid
  // pred with a cycle, which the round cap stops).
  __syncthreads();
  for (int round = 0; (1 << round) <= 2 * nn; ++round) {
    bool moved = false;
    for (int v = tid; v < nn; v += kRowThreads) {
      const unsigned long long w = jw[v];
      const int a = anc_of(w);
      if (a >= 0) {
        const unsigned long long wa = jw[a];
        jw[v] = pack(anc_of(wa), dist_of(w) + dist_of(wa));
        moved = true;
      }
    }
    if (!__syncthreads_or(moved)) break;
  }
  int dmax = 0;
  for (int v = tid; v < nn; v += kRowThreads) dmax = max(dmax, dist_of(jw[v]));
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  __shared__ int wmax[kRowThreads / 32];
  if ((tid & 31) == 0) wmax[tid >> 5] = dmax;
  __syncthreads();
  dmax = 0;
#pragma unroll
  for (int w = 0; w < kRowThreads / 32; ++w) dmax = max(dmax, wmax[w]);
  if (dmax > nn) dmax = nn;

  // deepest level first: a vertex at depth L is complete once level L+1 has
  // been added, and adds its sum to its parent (exact integer adds: the order
  // within a level does not matter)
  for (int L = dmax; L >= 1; --L) {
    for (int v = tid; v < nn; v += kRowThreads)
      if (par[v] >= 0 && dist_of(jw[v]) == L)
        atomicAdd(reinterpret_cast<unsigned long long*>(acc + par[v]),
                  (unsigned long long)acc[v]);
    __syncthreads();
  }
  const double from_fix = ldexp(1.0, e);
  for (int v = tid; v < nn; v += kRowThreads)
    E[off + v] = par[v] >= 0 ? (float)((double)acc[v] * from_fix) : 0.0f;
  if (tid == 0) Srow[blockIdx.x] = sabs;
}

// Kernel 2: columns [v0, v0 + C) of dL/dW of graph b (C = kC).
template <int kC>
__global__ void __launch_bounds__(kColThreads) k_bwd_cols(const float* __restrict__ E,
                                                          const int32_t* __restrict__ P,
                                                          const double* __restrict__ Srow,
                                                          float* __restrict__ GW, int64_t n,
                                                          int64_t ld, int64_t stride,
                                                          int64_t blocks_per_graph) {
  extern __shared__ __align__(16) unsigned char sm[];
  long long* acc = reinterpret_cast<long long*>(sm);  // [u][c], c fastest
  __shared__ double red[kColThreads / 32];
  const int tid = threadIdx.x;
  const int nn = (int)n;
  const int64_t b = blockIdx.x / blocks_per_graph;
  const int v0 = (int)(blockIdx.x % blocks_per_graph) * kC;
  const int64_t base = b * stride;
  // the graph's bound: the sum of every row's sum of |dL/dD| (fixed order)
  double s = 0.0;
  for (int r = tid; r < nn; r += kColThreads) s += Srow[b * n + r];
  s = block_sum<kColThreads>(s, red);
  const int e = quantum_exp(s);
  const double to_fix = ldexp(1.0, -e), from_fix = ldexp(1.0, e);
  const int total = nn * kC;
  for (int q = tid; q < total; q += kColThreads) acc[q] = 0;
  __syncthreads();
  // row segments of kC columns: consecutive threads read consecutive columns
  for (int q = tid; q < total; q += kColThreads) {
    const int r = q / kC, c = q - r * kC;
    const int v = v0 + c;
    if (v >= nn || r == v) continue;
    const int u = P[base + (int64_t)r * ld + v];
    if (u < 0 || u >= nn || u == v) continue;
    const long long x = __double2ll_rn((double)E[base + (int64_t)r * ld + v] * to_fix);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + (size_t)u * kC + c),
              (unsigned long long)x);
  }
  __syncthreads();
  for (int q = tid; q < total; q += kColThreads) {
    const int u = q / kC, c = q - u * kC;
    const int v = v0 + c;
    if (v >= nn) continue;
    GW[base + (int64_t)u * ld + v] = u == v ? 0.0f : (float)((double)acc[q] * from_fix);
  }
}

size_t rows_smem(int64_t n) { return (size_t)n * 20; }

template <int kC>
fw_status launch_cols(const float* E, const int32_t* P, const double* S, float* GW, int64_t n,
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
  // scratch: E (batch x st fp32), then the per-row sums of |dL/dD| (doubles)
  const size_t e_bytes = ((size_t)(batch * st) * 4 + 255) / 256 * 256;
  unsigned char* scratch = reinterpret_cast<unsigned char*>(
      fwh::backward_scratch(s, e_bytes + (size_t)(batch * n) * 8));
  if (!scratch) return FW_ERR_NOMEM;
  float* E = reinterpret_cast<float*>(scratch);
  double* S = reinterpret_cast<double*>(scratch + e_bytes);
  if (fwh::kernel_setup(reinterpret_cast<const void*>(k_bwd_rows), rows_smem(kMaxN), kRowThreads) < 1)
    return FW_ERR_CUDA;
  k_bwd_rows<<<(unsigned)(n * batch), kRowThreads, rows_smem(n), s>>>(grad_dist, pred, E, S, n,
                                                                       ld, st);
  if (cudaGetLastError() != cudaSuccess) return FW_ERR_CUDA;
  // as many columns per CTA as 128 KB of accumulators allow (8 = one 32-byte
  // sector per row segment)
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
