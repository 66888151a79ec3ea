// Shortest paths read back from a solved predecessor matrix (the paper's P
// "records the paths", Sec. 2.3): for each requested (source, target) pair,
// the vertices from the source to the target, following last hops backwards
// from the target.  One thread per pair; every walk is bounded by n hops, so
// a predecessor matrix that is not a tree (or garbage) ends in an error code,
// never in an endless loop or an out-of-range read.
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

}  // namespace

using namespace fwh;

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
