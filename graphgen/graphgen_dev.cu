// Device copy of the seeded graph generator in graphgen/__init__.py.
//
// It exists so that large benchmark inputs (n = 32768 is 4 GiB of int32) can be
// drawn in HBM without a host round trip.  It computes exactly the same counter
// hash as the numpy version (SplitMix64, Steele/Lea/Flood 2014) and holds none
// of the shortest-path arithmetic.  Tests check the two for bit equality.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t counter(uint64_t seed, uint64_t n, uint64_t i,
                                           uint64_t j, uint64_t s) {
  return seed * 0x9E3779B97F4A7C15ull + (((i * n + j) << 1) | s);
}

__device__ __forceinline__ bool edge_present(uint64_t seed, uint64_t n, uint64_t i,
                                             uint64_t j, double p) {
  uint64_t h1 = splitmix64(counter(seed, n, i, j, 1));
  return (double)(h1 >> 11) * 0x1p-53 < p;
}

__global__ void fill_i32(int32_t* out, int64_t n, int64_t ld, uint64_t seed, double p,
                         int32_t lo, int32_t hi, int32_t inf) {
  const uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    int32_t v;
    if (i == j) {
      v = 0;
    } else if (edge_present(seed, n, i, j, p)) {
      uint64_t h0 = splitmix64(counter(seed, n, i, j, 0));
      v = (int32_t)((int64_t)lo + (int64_t)(h0 % span));
    } else {
      v = inf;
    }
    out[i * ld + j] = v;
  }
}

__global__ void fill_f32(float* out, int64_t n, int64_t ld, uint64_t seed, double p,
                         int kind) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    float v;
    if (i == j) {
      v = 0.0f;
    } else if (edge_present(seed, n, i, j, p)) {
      uint64_t h0 = splitmix64(counter(seed, n, i, j, 0));
      double top = (double)(h0 >> 40);
      v = kind == 0 ? (float)((top + 1.0) * 0x1p-24) : (float)(1.0 + top * 0x1p-24);
    } else {
      v = __int_as_float(0x7f800000);
    }
    out[i * ld + j] = v;
  }
}

__global__ void fill_i64(int64_t* out, int64_t n, int64_t ld, uint64_t seed, double p,
                         int64_t lo, int64_t hi, int64_t inf) {
  const uint64_t span = (uint64_t)(hi - lo) + 1;
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    int64_t v;
    if (i == j) {
      v = 0;
    } else if (edge_present(seed, n, i, j, p)) {
      uint64_t h0 = splitmix64(counter(seed, n, i, j, 0));
      v = lo + (int64_t)(h0 % span);
    } else {
      v = inf;
    }
    out[i * ld + j] = v;
  }
}

__global__ void fill_f64(double* out, int64_t n, int64_t ld, uint64_t seed, double p,
                         int kind) {
  const int64_t total = n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    double v;
    if (i == j) {
      v = 0.0;
    } else if (edge_present(seed, n, i, j, p)) {
      uint64_t h0 = splitmix64(counter(seed, n, i, j, 0));
      v = kind == 0 ? ((double)(h0 >> 11) + 1.0) * 0x1p-53 : 1.0 + (double)(h0 >> 12) * 0x1p-52;
    } else {
      v = __longlong_as_double(0x7ff0000000000000ll);
    }
    out[i * ld + j] = v;
  }
}

int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

extern "C" {

// Fills the n x n row-major block of `out` (device memory, leading dimension
// ld >= n) with the seeded int32 graph.  Returns 0 on success, 1 on bad
// arguments, 2 on a CUDA launch error.
int graphgen_fill_i32(int32_t* out, int64_t n, int64_t ld, uint64_t seed, double p,
                      int32_t lo, int32_t hi, int32_t inf, void* stream) {
  if (!out || n <= 0 || ld < n || hi < lo) return 1;
  fill_i32<<<grid_for(n * n), 256, 0, (cudaStream_t)stream>>>(out, n, ld, seed, p, lo, hi, inf);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// Same for fp32 weights; kind 0 draws (0,1], kind 1 draws [1,2).
int graphgen_fill_f32(float* out, int64_t n, int64_t ld, uint64_t seed, double p, int kind,
                      void* stream) {
  if (!out || n <= 0 || ld < n || (kind != 0 && kind != 1)) return 1;
  fill_f32<<<grid_for(n * n), 256, 0, (cudaStream_t)stream>>>(out, n, ld, seed, p, kind);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// int64 weights in [lo, hi] (missing edges inf).
int graphgen_fill_i64(int64_t* out, int64_t n, int64_t ld, uint64_t seed, double p, int64_t lo,
                      int64_t hi, int64_t inf, void* stream) {
  if (!out || n <= 0 || ld < n || hi < lo) return 1;
  fill_i64<<<grid_for(n * n), 256, 0, (cudaStream_t)stream>>>(out, n, ld, seed, p, lo, hi, inf);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// fp64 weights; kind 0 draws (0,1], kind 1 draws [1,2).
int graphgen_fill_f64(double* out, int64_t n, int64_t ld, uint64_t seed, double p, int kind,
                      void* stream) {
  if (!out || n <= 0 || ld < n || (kind != 0 && kind != 1)) return 1;
  fill_f64<<<grid_for(n * n), 256, 0, (cudaStream_t)stream>>>(out, n, ld, seed, p, kind);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
