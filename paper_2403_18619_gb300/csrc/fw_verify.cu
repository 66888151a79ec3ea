// GPU check of the shortest-path certificate of an int32 solve.
//
// For exact distances D and last hops P of a graph W (nonnegative weights):
//   (a) D[i][i] = 0,
//   (b) every reachable pair is realised by its last hop: D[i][p] + W[p][j] = D[i][j],
//   (c) no edge can shorten any distance: D[i][v] <= D[i][u] + W[u][v] for all i, u, v,
//   (d) pred is -1 exactly on the diagonal and the unreachable pairs.
// (b) says every D[i][j] is the length of a real path, (c) that no path is
// shorter (LP duality), so together they certify D exactly, and (b) makes P a
// valid last hop.  (c) is a full min-plus product D (x) W, checked exhaustively.
// This file is deliberately independent of the solver's kernels.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_internal.h"

namespace {

constexpr int32_t kInf = 1 << 29;

__global__ void k_pointwise(const int32_t* __restrict__ W, const int32_t* __restrict__ D,
                            const int32_t* __restrict__ P, int64_t n, int64_t ld,
                            unsigned long long* bad) {
  unsigned long long b0 = 0, b1 = 0, b3 = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    const int32_t d = D[i * ld + j];
    const int32_t p = P[i * ld + j];
    if (i == j) {
      b0 += d != 0;
      b3 += p != -1;
      continue;
    }
    if (d >= kInf) {
      b3 += p != -1;
      continue;
    }
    if (p < 0 || p >= n || p == j) {
      b1 += 1;
      continue;
    }
    const int32_t w = W[(int64_t)p * ld + j];
    const int32_t dp = D[i * ld + p];
    b1 += (w >= kInf || dp >= kInf || (int64_t)dp + w != (int64_t)d);
  }
  if (b0) atomicAdd(bad + 0, b0);
  if (b1) atomicAdd(bad + 1, b1);
  if (b3) atomicAdd(bad + 3, b3);
}

// 64 x 64 output tile per CTA, 4 x 4 per thread, u streamed in chunks of 16.
__global__ void __launch_bounds__(256) k_feasible(const int32_t* __restrict__ W,
                                                  const int32_t* __restrict__ D, int64_t n,
                                                  int64_t ld, unsigned long long* bad) {
  __shared__ int32_t Ds[16][64 + 1];
  __shared__ int32_t Ws[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * 64, v0 = (int64_t)blockIdx.x * 64;
  int32_t best[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) best[a][b] = 2 * kInf;
  for (int64_t u0 = 0; u0 < n; u0 += 16) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int uu = q / 64, c = q % 64;
      const int64_t gi = i0 + c, gu = u0 + uu, gv = v0 + c;
      Ds[uu][c] = (gi < n && gu < n) ? min(D[gi * ld + gu], kInf) : kInf;
      Ws[uu][c] = (gu < n && gv < n) ? min(W[gu * ld + gv], kInf) : kInf;
    }
    __syncthreads();
    for (int uu = 0; uu < 16; ++uu)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
          best[a][b] = min(best[a][b], Ds[uu][ty * 4 + a] + Ws[uu][tx * 4 + b]);
    __syncthreads();
  }
  unsigned long long cnt = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int64_t gi = i0 + ty * 4 + a, gv = v0 + tx * 4 + b;
      if (gi < n && gv < n && D[gi * ld + gv] > best[a][b]) cnt++;
    }
  if (cnt) atomicAdd(bad + 2, cnt);
}

}  // namespace

extern "C" fw_status fw_verify_certificate(const int32_t* W, const int32_t* dist,
                                           const int32_t* pred, int64_t n, int64_t ld,
                                           int64_t* bad, void* stream) {
  if (!W || !dist || !pred || !bad || n <= 0 || ld < n) return FW_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) return FW_ERR_NOMEM;
  fw_status st = FW_OK;
  cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), s);
  int64_t blocks = (n * n + 255) / 256;
  if (blocks > fwh::num_sms() * 16) blocks = fwh::num_sms() * 16;
  k_pointwise<<<(int)blocks, 256, 0, s>>>(W, dist, pred, n, ld, d);
  const int64_t tiles = (n + 63) / 64;
  k_feasible<<<dim3((unsigned)tiles, (unsigned)tiles), 256, 0, s>>>(W, dist, n, ld, d);
  unsigned long long h[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    st = FW_ERR_CUDA;
  for (int k = 0; k < 4; ++k) bad[k] = (int64_t)h[k];
  cudaFree(d);
  return st;
}
