// Shortest paths read back from a solved predecessor matrix (the paper's P
// "records the paths", Sec. 2.3): for each requested (source, target) pair,
// the vertices from the source to the target, following last hops backwards
// from the target.  One thread per pair; every walk is bounded by n hops, so
// a predecessor matrix that is not a tree (or garbage) ends in an error code,
// never in an endless loop or an out-of-range read.
//
// fw_intermediate turns the last-hop matrix into the bookkeeping of the
// paper's Fig. 1, where P_ij holds the intermediate vertex k through which
// (i, j) last improved.  On a pair with a unique shortest path that vertex is
// the largest intermediate vertex of the path (the path becomes available at
// k = its largest intermediate, and nothing improves it afterwards); the
// kernel computes the largest intermediate vertex of the path the last hops
// record, for every pair.  One CTA per source row (the row owned by that
// CTA): pointer jumping in shared memory on packed (ancestor, largest vertex
// strictly between) words, log2(depth) + 1 rounds.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_internal.h"

namespace {

__global__ void k_paths(const int32_t* __restrict__ P, int64_t n, int64_t ld,
                        const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                        int64_t npairs, int32_t* __restrict__ out, int64_t max_len,
                        int32_t* __restrict__ len) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npairs;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = src[q], t = dst[q];
    if (s < 0 || s >= n || t < 0 || t >= n) {
      len[q] = -1;
      continue;
    }
    const int32_t* row = P + (int64_t)s * ld;
    // 1. count the vertices (bounded walk)
    int64_t cnt = 1;
    int32_t v = t;
    bool ok = true;
    while (v != s) {
      const int32_t u = row[v];
      if (u < 0 || u >= n || cnt >= n) {
        ok = false;
        break;
      }
      v = u;
      ++cnt;
    }
    if (!ok) {
      // no last hop at the target itself: unreachable; anywhere else: not a tree
      len[q] = (v == t && row[t] == -1) ? 0 : -1;
      continue;
    }
    if (cnt > max_len) {
      len[q] = -1;
      continue;
    }
    // 2. the same walk again, writing the vertices from the back
    int32_t* o = out + q * max_len;
    int64_t pos = cnt - 1;
    v = t;
    o[pos] = t;
    while (pos > 0) {
      v = row[v];
      o[--pos] = v;
    }
    len[q] = (int32_t)cnt;
  }
}

// Kernel of fw_intermediate: 4 bytes of shared memory per vertex of the row.
constexpr int kMidThreads = 256;
constexpr int64_t kMidMaxN = 57344;  // 224 KB; the 16-bit fields allow 65535

constexpr unsigned kNone = 0xffffu;
__device__ __forceinline__ unsigned mid_word(unsigned anc, unsigned top1) { return (top1 << 16) | anc; }
__device__ __forceinline__ unsigned mid_anc(unsigned w) { return w & 0xffffu; }
__device__ __forceinline__ unsigned mid_top1(unsigned w) { return w >> 16; }  // largest + 1, 0: none

__global__ void __launch_bounds__(kMidThreads) k_intermediate(const int32_t* P, int32_t* out,
                                                              int64_t n, int64_t ld,
                                                              int64_t stride) {
  extern __shared__ unsigned jw[];
  const int nn = (int)n, tid = threadIdx.x;
  const int64_t b = blockIdx.x / n;
  const int i = (int)(blockIdx.x % n);
  const int64_t off = b * stride + (int64_t)i * ld;
  // ancestor = the last hop (none: the source, unreachable vertices, entries
  // outside [0, n)); nothing strictly between a vertex and its last hop
  for (int v = tid; v < nn; v += kMidThreads) {
    const int p = P[off + v];
    const bool tree = v != i && p >= 0 && p < nn && p != v;
    jw[v] = mid_word(tree ? (unsigned)p : kNone, 0u);
  }
  __syncthreads();
  // jump until every ancestor is the source (whose word has no ancestor):
  // word v = (a, t) becomes (ancestor of a, max(t, a + 1, t of a)).  Every
  // word is one 32-bit access, so a thread combines a consistent pair even
  // while others advance within the same round; the round cap stops a pred
  // with a cycle (its vertices never reach the source and are written -1).
  for (int round = 0; (1 << round) <= 2 * nn; ++round) {
    bool moved = false;
    for (int v = tid; v < nn; v += kMidThreads) {
      const unsigned w = jw[v], a = mid_anc(w);
      if (a == kNone) continue;
      const unsigned wa = jw[a], aa = mid_anc(wa);
      if (aa == kNone) continue;
      jw[v] = mid_word(aa, max(max(mid_top1(w), a + 1u), mid_top1(wa)));
      moved = true;
    }
    if (!__syncthreads_or(moved)) break;
  }
  // the row's reads all precede these writes (the barrier above), so out may
  // be pred itself
  for (int v = tid; v < nn; v += kMidThreads) {
    const unsigned w = jw[v];
    out[off + v] = mid_anc(w) == (unsigned)i ? (int32_t)mid_top1(w) - 1 : -1;
  }
}

}  // namespace

using namespace fwh;

extern "C" fw_status fw_intermediate(const int32_t* pred, int32_t* out, int64_t n, int64_t ld,
                                     int64_t batch, int64_t stride, void* stream) {
  if (!pred || !out) return FW_ERR_ARG;
  if (n < 1 || ld < n || batch < 0) return FW_ERR_ARG;
  if (batch > 1 && stride < n * ld) return FW_ERR_ARG;
  if (n > kMidMaxN) return FW_ERR_UNSUPPORTED;
  if (batch == 0) return FW_OK;
  if (batch * n > 0x7fffffffLL) return FW_ERR_ARG;
  const size_t smem = (size_t)n * sizeof(unsigned);
  if (kernel_setup(reinterpret_cast<const void*>(k_intermediate), (size_t)kMidMaxN * 4,
                   kMidThreads) < 1)
    return FW_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_intermediate<<<(unsigned)(batch * n), kMidThreads, smem, s>>>(pred, out, n, ld,
                                                                   batch > 1 ? stride : 0);
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

extern "C" fw_status fw_paths(const int32_t* pred, int64_t n, int64_t ld, const int32_t* src,
                              const int32_t* dst, int64_t npairs, int32_t* out, int64_t max_len,
                              int32_t* len, void* stream) {
  if (!pred || !src || !dst || !out || !len) return FW_ERR_ARG;
  if (n <= 0 || n > 131072 || ld < n || npairs < 0 || max_len < 1) return FW_ERR_ARG;
  if (npairs == 0) return FW_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t blocks = (npairs + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_paths<<<(unsigned)blocks, 256, 0, s>>>(pred, n, ld, src, dst, npairs, out, max_len, len);
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}
