// Min-plus relaxation peak of the GPU (the roofline of the solver's inner loop).
//
// Each thread keeps a block of relaxation chains in registers (8 x 8 for the
// 32-bit types, 1 x 8 for the 64-bit ones, so that 512 threads fit the
// register file) and relaxes it with the instructions the solver issues per
// relaxation:
//   int32 : acc = __viaddmin_u32(a, b, acc)     (one DPX instruction)
//   fp32  : acc = fminf(a + b, acc)             (add + min)
//   fp64  : acc = a + b < acc ? a + b : acc     (DADD, then an integer min of
//                                                the bit patterns, as the solver)
//   int64 : acc = min(a + b, acc)               (64-bit add + compare-select)
// Every unrolled step takes its own column operands b[u][.], so every
// relaxation forms a distinct sum (none can be computed once and reused) and
// min(x, min(x, acc)) cannot fold.  The row operands a[m] are refreshed every 4
// steps from the chains themselves, so the loop carries a real dependence and
// nothing can be hoisted out of it.  One CTA of 512 threads per SM; %clock64
// around the loop gives the SM-clock rate, CUDA events the wall-clock rate.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_internal.h"

namespace {

constexpr int kProbeThreads = 512;

template <typename T> struct ProbeMode;
template <> struct ProbeMode<uint32_t> { static constexpr int M = 8; };
template <> struct ProbeMode<float> { static constexpr int M = 8; };
template <> struct ProbeMode<double> { static constexpr int M = 1; };
template <> struct ProbeMode<int64_t> { static constexpr int M = 1; };

template <typename T>
__device__ __forceinline__ T relax(T a, T b, T acc) {
  if constexpr (std::is_same<T, uint32_t>::value) {
    return __viaddmin_u32(a, b, acc);
  } else if constexpr (std::is_same<T, float>::value) {
    return fminf(a + b, acc);
  } else if constexpr (std::is_same<T, double>::value) {
    const double x = a + b;
    return __double_as_longlong(x) < __double_as_longlong(acc) ? x : acc;
  } else {
    const T x = a + b;
    return x < acc ? x : acc;
  }
}

template <typename T>
__device__ __forceinline__ T seed_value(uint32_t s, int k) {
  if constexpr (std::is_same<T, uint32_t>::value) return s + (uint32_t)k;
  else if constexpr (std::is_same<T, float>::value) return __uint_as_float(s) + (float)k;
  else if constexpr (std::is_same<T, double>::value) return (double)__uint_as_float(s) + (double)k;
  else return (int64_t)s * 1000003ll + k;
}

template <typename T>
__global__ void __launch_bounds__(kProbeThreads, 1)
    k_probe(const uint32_t* __restrict__ seed, uint32_t* __restrict__ sink, int iters,
            long long* __restrict__ cycles) {
  constexpr int M = ProbeMode<T>::M;
  T a[M], b[4][8], acc[M][8];
  const uint32_t s0 = seed[threadIdx.x & 63];
#pragma unroll
  for (int m = 0; m < M; ++m) a[m] = seed_value<T>(s0, m);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int n = 0; n < 8; ++n) b[u][n] = seed_value<T>(s0 >> 3, 3 * n + 29 * u);
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n) acc[m][n] = seed_value<T>(s0, 7 * m + n);
  __syncthreads();
  const long long c0 = clock64();
#pragma unroll 1
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int m = 0; m < M; ++m)
#pragma unroll
        for (int n = 0; n < 8; ++n) acc[m][n] = relax<T>(a[m], b[u][n], acc[m][n]);
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = acc[m][m];
  }
  __syncthreads();
  const long long c1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int m = 0; m < M; ++m)
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      unsigned long long bits;
      if constexpr (std::is_same<T, double>::value) bits = (unsigned long long)__double_as_longlong(acc[m][n]);
      else if constexpr (std::is_same<T, float>::value) bits = __float_as_uint(acc[m][n]);
      else bits = (unsigned long long)acc[m][n];
      x ^= (uint32_t)bits ^ (uint32_t)(bits >> 32);
    }
  sink[blockIdx.x * kProbeThreads + threadIdx.x] = x;
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

}  // namespace

extern "C" fw_status fw_peak_probe(fw_dtype dtype, double* relax_per_s, double* relax_per_sm_clk,
                                   double* sm_mhz, void* stream) {
  if (dtype != FW_I32 && dtype != FW_F32 && dtype != FW_I64 && dtype != FW_F64) return FW_ERR_ARG;
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
    for (int i = 0; i < 64; ++i)  // ints: small values; floats: 1.0f + small
      h[i] = (dtype == FW_I32 || dtype == FW_I64) ? 1000u + 17u * i : 0x3f800000u + 4096u * i;
    cudaMemcpy(seed, h, sizeof(h), cudaMemcpyHostToDevice);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the 64-bit pipes are far slower: fewer iterations for a similar duration
    const bool wide = dtype == FW_I64 || dtype == FW_F64;
    const int iters = wide ? 1 << 13 : 1 << 15;
    const int chains = wide ? 8 : 64;
    auto kern = dtype == FW_I32   ? k_probe<uint32_t>
                : dtype == FW_F32 ? k_probe<float>
                : dtype == FW_F64 ? k_probe<double>
                                  : k_probe<int64_t>;
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
      const double per_sm = (double)kProbeThreads * iters * chains;
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
