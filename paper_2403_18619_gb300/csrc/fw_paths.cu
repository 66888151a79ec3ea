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

// Word of vertex v from its last hop p (row i): ancestor p, nothing strictly
// between them yet; no ancestor for the source, unreachable vertices and
// entries outside [0, n).
__device__ __forceinline__ unsigned mid_init(int v, int p, int i, int nn) {
  const bool tree = v != i && p >= 0 && p < nn && p != v;
  return mid_word(tree ? (unsigned)p : kNone, 0u);
}
// Result of a converged word: the largest intermediate vertex, -1 for none
// (the edge itself) and for vertices whose walk never reached the source.
__device__ __forceinline__ int32_t mid_out(unsigned w, int i) {
  return mid_anc(w) == (unsigned)i ? (int32_t)mid_top1(w) - 1 : -1;
}

// One CTA per row.  vec: the row starts on a 16-byte boundary in both
// matrices, so the row moves in 16-byte accesses (the n % 4 tail one by one),
// several in flight per thread.
__global__ void __launch_bounds__(kMidThreads) k_intermediate(const int32_t* P, int32_t* out,
                                                              int64_t n, int64_t ld,
                                                              int64_t stride, int vec) {
  extern __shared__ __align__(16) unsigned jw[];
  const int nn = (int)n, tid = threadIdx.x;
  const int64_t b = blockIdx.x / n;
  const int i = (int)(blockIdx.x % n);
  const int64_t off = b * stride + (int64_t)i * ld;
  const int nv = vec ? nn & ~3 : 0;
#pragma unroll 4
  for (int q = 4 * tid; q < nv; q += 4 * kMidThreads) {
    const int4 p4 = *reinterpret_cast<const int4*>(P + off + q);
    uint4 w4;
    w4.x = mid_init(q, p4.x, i, nn);
    w4.y = mid_init(q + 1, p4.y, i, nn);
    w4.z = mid_init(q + 2, p4.z, i, nn);
    w4.w = mid_init(q + 3, p4.w, i, nn);
    *reinterpret_cast<uint4*>(jw + q) = w4;
  }
  for (int v = nv + tid; v < nn; v += kMidThreads) jw[v] = mid_init(v, P[off + v], i, nn);
  __syncthreads();
  // jump until every ancestor is the source (whose word has no ancestor):
  // word v = (a, t) becomes (ancestor of a, max(t, a + 1, t of a)).  Every
  // word is one 32-bit access, so a thread combines a consistent pair even
  // while others (or its own earlier stores) advance within the same round;
  // each thread reads four words and their ancestors' words before it writes
  // any, so the shared-memory round trips overlap.  The round cap stops a
  // pred with a cycle (its vertices never reach the source and are written
  // -1).
  for (int round = 0; (1 << round) <= 2 * nn; ++round) {
    bool moved = false;
    for (int v0 = tid; v0 < nn; v0 += 4 * kMidThreads) {
      unsigned w[4], wa[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int v = v0 + u * kMidThreads;
        w[u] = v < nn ? jw[v] : mid_word(kNone, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned a = mid_anc(w[u]);
        wa[u] = a != kNone ? jw[a] : mid_word(kNone, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned a = mid_anc(w[u]), aa = mid_anc(wa[u]);
        if (a != kNone && aa != kNone) {
          jw[v0 + u * kMidThreads] =
              mid_word(aa, max(max(mid_top1(w[u]), a + 1u), mid_top1(wa[u])));
          moved = true;
        }
      }
    }
    if (!__syncthreads_or(moved)) break;
  }
  // the row's reads all precede these writes (the barrier above), so out may
  // be pred itself
#pragma unroll 4
  for (int q = 4 * tid; q < nv; q += 4 * kMidThreads) {
    const uint4 w4 = *reinterpret_cast<const uint4*>(jw + q);
    const int4 o = make_int4(mid_out(w4.x, i), mid_out(w4.y, i), mid_out(w4.z, i),
                             mid_out(w4.w, i));
    *reinterpret_cast<int4*>(out + off + q) = o;
  }
  for (int v = nv + tid; v < nn; v += kMidThreads) out[off + v] = mid_out(jw[v], i);
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
  const bool vec = ((uintptr_t)pred % 16) == 0 && ((uintptr_t)out % 16) == 0 && ld % 4 == 0 &&
                   (batch <= 1 || stride % 4 == 0);
  k_intermediate<<<(unsigned)(batch * n), kMidThreads, smem, s>>>(
      pred, out, n, ld, batch > 1 ? stride : 0, vec ? 1 : 0);
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
