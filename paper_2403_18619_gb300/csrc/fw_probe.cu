// Min-plus relaxation peak of the GPU (the roofline of the solver's inner loop).
//
// Each thread keeps an 8 x 8 block of relaxation chains in registers and
// relaxes it with the same instruction the solver issues per relaxation:
//   int32: acc = __viaddmin_u32(a, b, acc)     (one DPX instruction)
//   fp32 : acc = fminf(a + b, acc)             (add + min)
// The row operands a[m] are refreshed every 4 steps from the chains themselves,
// so the loop carries a real dependence and nothing can be hoisted out of it.
// One CTA of 512 threads per SM; %clock64 around the loop gives the SM-clock
// rate, CUDA events the wall-clock rate.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_internal.h"

namespace {

constexpr int kProbeThreads = 512;

template <bool kInt>
__global__ void __launch_bounds__(kProbeThreads, 1)
    k_probe(const uint32_t* __restrict__ seed, uint32_t* __restrict__ sink, int iters,
            long long* __restrict__ cycles) {
  uint32_t a[8], b[8], acc[8][8];
  const uint32_t s0 = seed[threadIdx.x & 63];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    a[m] = s0 + m;
    b[m] = (s0 >> 3) + 3 * m;
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[m][n] = s0 + 7 * m + n;
  }
  __syncthreads();
  const long long c0 = clock64();
#pragma unroll 1
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int n = 0; n < 8; ++n) {
          // a different column operand in each of the 4 unrolled steps: with
          // the same one, min(x, min(x, acc)) would fold to a single min
          if constexpr (kInt) {
            acc[m][n] = __viaddmin_u32(a[m], b[(n + u) & 7], acc[m][n]);
          } else {
            float x = __uint_as_float(a[m]) + __uint_as_float(b[(n + u) & 7]);
            acc[m][n] = __float_as_uint(fminf(x, __uint_as_float(acc[m][n])));
          }
        }
#pragma unroll
    for (int m = 0; m < 8; ++m) a[m] = acc[m][m];
  }
  __syncthreads();
  const long long c1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n) x ^= acc[m][n];
  sink[blockIdx.x * kProbeThreads + threadIdx.x] = x;
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

}  // namespace

extern "C" fw_status fw_peak_probe(fw_dtype dtype, double* relax_per_s, double* relax_per_sm_clk,
                                   double* sm_mhz, void* stream) {
  if (dtype != FW_I32 && dtype != FW_F32) return FW_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int sms = fwh::num_sms();
  uint32_t *seed = nullptr, *sink = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fw_status st = FW_OK;
  if (cudaMalloc(&seed, 64 * 4) != cudaSuccess ||
      cudaMalloc(&sink, (size_t)sms * kProbeThreads * 4) != cudaSuccess ||
      cudaMalloc(&cyc, (size_t)sms * 8) != cudaSuccess) {
    st = FW_ERR_NOMEM;
  }
  if (st == FW_OK) {
    uint32_t h[64];
    for (int i = 0; i < 64; ++i)
      h[i] = dtype == FW_I32 ? 1000u + 17u * i : 0x3f800000u + 4096u * i;  // fp32: 1.0f + small
    cudaMemcpy(seed, h, sizeof(h), cudaMemcpyHostToDevice);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 1 << 15;
    auto kern = dtype == FW_I32 ? k_probe<true> : k_probe<false>;
    kern<<<sms, kProbeThreads, 0, s>>>(seed, sink, 1024, cyc);  // warm-up
    cudaEventRecord(e0, s);
    kern<<<sms, kProbeThreads, 0, s>>>(seed, sink, iters, cyc);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = FW_ERR_CUDA;
    } else {
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      long long* hc = new long long[sms];
      cudaMemcpy(hc, cyc, (size_t)sms * 8, cudaMemcpyDeviceToHost);
      double cmax = 0, csum = 0;
      for (int i = 0; i < sms; ++i) { csum += (double)hc[i]; if (hc[i] > cmax) cmax = (double)hc[i]; }
      delete[] hc;
      const double per_sm = (double)kProbeThreads * iters * 64.0;
      const double total = per_sm * sms;
      if (relax_per_s) *relax_per_s = total / (ms * 1e-3);
      if (relax_per_sm_clk) *relax_per_sm_clk = per_sm / (csum / sms);
      if (sm_mhz) *sm_mhz = (csum / sms) / (ms * 1e-3) / 1e6;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (seed) cudaFree(seed);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  return st;
}
