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
// Kernel 1 (one CTA per source row, the row is owned by that CTA): hop depth by
// pointer jumping, vertices sorted by (parent, id) with a CTA bitonic sort so
// that siblings are contiguous, then subtree sums level by level from the
// deepest level up, each parent adding its children in id order.  No atomics:
// the result is deterministic.
// Kernel 2 (one CTA per column v): the pairs (pred[i][v], i) are sorted and
// every u receives the sum of its E[i][v] in increasing i, again without
// atomics.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_internal.h"

namespace {

constexpr int kBT = 1024;        // threads per CTA
constexpr int64_t kMaxN = 8192;  // rows held in shared memory

__device__ __forceinline__ int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Ascending bitonic sort of N2 (power of two) 64-bit keys in shared memory.
__device__ void cta_bitonic(unsigned long long* key, int N2) {
  for (int size = 2; size <= N2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < N2 / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = key[lo], b = key[hi];
        if ((a > b) == up) {
          key[lo] = b;
          key[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int block_max(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = max(r, red[w]);
  return r;
}

// Subtree sums of every source row of `batch` graphs (row b*n + i).
__global__ void __launch_bounds__(kBT) k_bwd_tree(const float* __restrict__ G,
                                                  const float* __restrict__ D,
                                                  const int32_t* __restrict__ P,
                                                  float* __restrict__ E, int64_t n, int64_t ld,
                                                  int64_t stride) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int nn = (int)n;
  const int N2 = pow2_at_least(nn);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(sm);  // N2
  int* par = reinterpret_cast<int*>(key + N2);                          // n
  int* anc = par + nn;                                                  // n
  int* dep = anc + nn;                                                  // n
  int* seg = dep + nn;                                                  // n: first child position
  float* acc = reinterpret_cast<float*>(seg + nn);                      // n
  __shared__ int red[32];
  const int64_t b = blockIdx.x / n, i = blockIdx.x % n;
  const int64_t rowoff = b * stride + i * ld;
  for (int v = threadIdx.x; v < nn; v += blockDim.x) {
    const int p = P[rowoff + v];
    const float d = D[rowoff + v];
    const bool reach = v != i && p >= 0 && p < nn && d < __int_as_float(0x7f800000);
    par[v] = reach ? p : -1;
    anc[v] = par[v];
    dep[v] = reach ? 1 : 0;
    acc[v] = reach ? G[rowoff + v] : 0.0f;
    seg[v] = -1;
  }
  for (int v = nn + threadIdx.x; v < N2; v += blockDim.x) key[v] = ~0ull;
  __syncthreads();
  // hop depth by pointer jumping (log2 n rounds; a cycle in pred cannot hang it)
  for (int round = 0; (1 << round) < 2 * nn; ++round) {
    int lv[kMaxN / kBT], la[kMaxN / kBT];
    int q = 0;
    for (int v = threadIdx.x; v < nn; v += blockDim.x, ++q) {
      const int a = anc[v];
      lv[q] = a >= 0 ? dep[a] : 0;
      la[q] = a >= 0 ? anc[a] : -1;
    }
    __syncthreads();
    q = 0;
    for (int v = threadIdx.x; v < nn; v += blockDim.x, ++q) {
      if (anc[v] >= 0) {
        dep[v] += lv[q];
        anc[v] = la[q];
      }
    }
    __syncthreads();
  }
  for (int v = threadIdx.x; v < nn; v += blockDim.x)
    key[v] = ((unsigned long long)(unsigned)(par[v] + 1) << 32) | (unsigned)v;
  __syncthreads();
  cta_bitonic(key, N2);
  // first position of every parent's children
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const int pu = (int)(key[q] >> 32) - 1;
    const int prev = q > 0 ? (int)(key[q - 1] >> 32) - 1 : -2;
    if (pu >= 0 && pu != prev) seg[pu] = q;
  }
  int my_max = 0;
  for (int v = threadIdx.x; v < nn; v += blockDim.x) my_max = max(my_max, dep[v]);
  const int M = block_max(my_max, red);
  __syncthreads();
  // deepest level first: every parent at depth L-1 adds its children (depth L)
  for (int L = M; L >= 1; --L) {
    for (int u = threadIdx.x; u < nn; u += blockDim.x) {
      if (seg[u] < 0 || dep[u] != L - 1 || (par[u] < 0 && u != i)) continue;
      float s = acc[u];
      for (int q = seg[u]; q < nn; ++q) {
        const unsigned long long k = key[q];
        if ((int)(k >> 32) - 1 != u) break;
        s += acc[(int)(k & 0xffffffffu)];
      }
      acc[u] = s;
    }
    __syncthreads();
  }
  for (int v = threadIdx.x; v < nn; v += blockDim.x) E[rowoff + v] = v == i ? 0.0f : acc[v];
}

// dL/dW column v of every graph: sum of E[i][v] over sources whose last hop to v is u.
__global__ void __launch_bounds__(kBT) k_bwd_scatter(const float* __restrict__ E,
                                                     const int32_t* __restrict__ P,
                                                     float* __restrict__ GW, int64_t n, int64_t ld,
                                                     int64_t stride) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int nn = (int)n;
  const int N2 = pow2_at_least(nn);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(sm);  // N2
  float* val = reinterpret_cast<float*>(key + N2);                      // n (indexed by i)
  int* seg = reinterpret_cast<int*>(val + nn);                          // n
  const int64_t b = blockIdx.x / n, v = blockIdx.x % n;
  const int64_t base = b * stride;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int p = P[base + (int64_t)i * ld + v];
    const bool edge = p >= 0 && p < nn && p != v && i != v;
    key[i] = edge ? (((unsigned long long)(unsigned)p << 32) | (unsigned)i) : ~0ull;
    val[i] = edge ? E[base + (int64_t)i * ld + v] : 0.0f;
    seg[i] = -1;
  }
  for (int q = nn + threadIdx.x; q < N2; q += blockDim.x) key[q] = ~0ull;
  __syncthreads();
  cta_bitonic(key, N2);
  for (int q = threadIdx.x; q < nn; q += blockDim.x) {
    const unsigned long long k = key[q];
    if (k == ~0ull) continue;
    const int u = (int)(k >> 32);
    if (q == 0 || (int)(key[q - 1] >> 32) != u || key[q - 1] == ~0ull) seg[u] = q;
  }
  __syncthreads();
  for (int u = threadIdx.x; u < nn; u += blockDim.x) {
    float s = 0.0f;
    if (seg[u] >= 0) {
      for (int q = seg[u]; q < nn; ++q) {
        const unsigned long long k = key[q];
        if (k == ~0ull || (int)(k >> 32) != u) break;
        s += val[(int)(k & 0xffffffffu)];
      }
    }
    GW[base + (int64_t)u * ld + v] = s;
  }
}

size_t tree_smem(int64_t n) {
  int64_t N2 = 1;
  while (N2 < n) N2 <<= 1;
  return (size_t)N2 * 8 + (size_t)n * 4 * 5;
}
size_t scatter_smem(int64_t n) {
  int64_t N2 = 1;
  while (N2 < n) N2 <<= 1;
  return (size_t)N2 * 8 + (size_t)n * 4 * 2;
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
  float* E = reinterpret_cast<float*>(fwh::backward_scratch(s, (size_t)(batch * st) * 4));
  if (!E) return FW_ERR_NOMEM;
  const size_t s1 = tree_smem(n), s2 = scatter_smem(n);
  if (fwh::kernel_setup(reinterpret_cast<const void*>(k_bwd_tree), tree_smem(kMaxN), kBT) < 1 ||
      fwh::kernel_setup(reinterpret_cast<const void*>(k_bwd_scatter), scatter_smem(kMaxN), kBT) < 1)
    return FW_ERR_CUDA;
  k_bwd_tree<<<(unsigned)(n * batch), kBT, s1, s>>>(grad_dist, dist, pred, E, n, ld, st);
  if (cudaGetLastError() != cudaSuccess) return FW_ERR_CUDA;
  k_bwd_scatter<<<(unsigned)(n * batch), kBT, s2, s>>>(E, pred, grad_w, n, ld, st);
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

fw_status fw_backward(const float* grad_dist, const float* dist, const int32_t* pred,
                      float* grad_w, int64_t n, int64_t ld, void* stream) {
  return fw_backward_strided(grad_dist, dist, pred, grad_w, n, ld, 1, n * ld, stream);
}

}  // extern "C"
