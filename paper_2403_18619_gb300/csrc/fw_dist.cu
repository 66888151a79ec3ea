// Tile-level kernels of the blocked algorithm (Sec. 2.3, Fig. 2) for callers
// that keep the matrix in pieces: a single-graph solve spread over several
// GPUs keeps on each GPU the tiles a 2-D block-cyclic map gives it and runs,
// per round, the pivot closure, the panel updates and the update of its
// remaining tiles with these calls (the exchange of pivot and panels between
// the GPUs is the caller's, by collectives).
//
//   k_tile_closure   phase 1: in-place FW over the BS vertices of one tile
//   k_tile_minplus   phases 2-4: C = min(C, A (x) B) over a grid of BS x BS
//                    output tiles, last hops from the predecessors of B's rows
//   k_block_init     predecessor initialisation of block-cyclic local blocks
//
// All matrices are tile-padded (whole BS x BS tiles; padding vertices are
// isolated: INF off the diagonal), so no kernel here masks ragged edges.
#include <cstdint>
#include <cuda_runtime.h>

#include "fw_device.cuh"
#include "fw_internal.h"

namespace fwk {

// Phase 1 on one BS x BS tile (row-major, leading dimension ld): the strict-<
// closure with last hops.  A negative diagonal entry sets the status bit.
template <typename T, int BS>
__global__ void __launch_bounds__(kThreads, 1)
    k_tile_closure(T* D, int32_t* P, int64_t ld, int* status) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM;
  __shared__ __align__(16) unsigned char sm[2 * BS * (2 * sizeof(T) + 4)];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t big = (int64_t)1 << 40;  // tile-padded: nothing to mask
  T d[TM][TM];
  int32_t p[TM][TM];
  load_tile<BS>(d, D, big, ld, 0, 0, tx, ty, Num<T>::inf());
  if (P) {
    load_tile<BS>(p, P, big, ld, 0, 0, tx, ty, (int32_t)-1);
  } else {
#pragma unroll
    for (int mm = 0; mm < TM; ++mm)
#pragma unroll
      for (int nn = 0; nn < TM; ++nn) p[mm][nn] = -1;
  }
  closure_steps<T, BS>(d, p, sm);
  bool neg = false;
#pragma unroll
  for (int mm = 0; mm < TM; ++mm)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn)
      if (Gm::idx(ty, mm) == Gm::idx(tx, nn) && d[mm][nn] < T(0)) neg = true;
  if (neg) atomicOr(status, kStNegCycle);
  store_tile<BS>(D, d, big, ld, 0, 0, tx, ty);
  if (P) store_tile<BS>(P, p, big, ld, 0, 0, tx, ty);
}

// Output tile (blockIdx.y, blockIdx.x) of C: C = min(C, A_i (x) B_j) with A_i
// the BS x BS block (i, 0) of A and B_j the block (0, j) of B; on a strict
// improvement through step kk, Pc = Pb[kk][column] (the last hop of B's row
// kk).  The CTA stages A_i, B_j and Pb_j in shared memory and C's tile in
// registers before it stores anything, so C may be A when there is one tile
// column, or B (and Pc may be Pb) when there is one tile row.  Tiles in tile
// row skip_i or tile column skip_j are left alone.
template <typename T, int BS>
__global__ void __launch_bounds__(kThreads, 1)
    k_tile_minplus(T* C, int32_t* Pc, int64_t ldc, const T* A, int64_t lda, const T* B,
                   int64_t ldb, const int32_t* Pb, int64_t ldpb, int64_t skip_i,
                   int64_t skip_j) {
  using Gm = Geo<BS>;
  constexpr int TM = Gm::TM;
  extern __shared__ __align__(128) unsigned char smem[];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti == skip_i || tj == skip_j) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t big = (int64_t)1 << 40;
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + BS * BS;
  int32_t* Ps = reinterpret_cast<int32_t*>(Bs + BS * BS);
  {
    T v[TM][TM];
    load_tile<BS>(v, A, big, lda, ti, 0, tx, ty, Num<T>::inf());
    put_tile<BS, true>(As, v, tx, ty);
    load_tile<BS>(v, B, big, ldb, 0, tj, tx, ty, Num<T>::inf());
    put_tile<BS, false>(Bs, v, tx, ty);
  }
  if (Pc) {
    int32_t v[TM][TM];
    load_tile<BS>(v, Pb, big, ldpb, 0, tj, tx, ty, (int32_t)-1);
    put_tile<BS, false>(Ps, v, tx, ty);
  }
  T acc[TM][TM];
  int arg[TM][TM];
  load_tile<BS>(acc, C, big, ldc, ti, tj, tx, ty, Num<T>::inf());
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) arg[m][nn] = 0;
  __syncthreads();
  core_generic<BS, T>(As, Bs, acc, arg, tx, ty);
  // only improved entries change; a group of G with no improvement is left as is
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int64_t gi = (int64_t)ti * BS + Gm::idx(ty, m);
#pragma unroll
    for (int nn = 0; nn < TM; ++nn) {
      if (!arg[m][nn]) continue;
      const int lc = Gm::idx(tx, nn);
      const int64_t gj = (int64_t)tj * BS + lc;
      C[gi * ldc + gj] = acc[m][nn];
      if (Pc) Pc[gi * ldc + gj] = Ps[(arg[m][nn] - 1) * BS + lc];
    }
  }
}

// pred of a rows x cols block-cyclic local block: local row a belongs to the
// global vertex (row_tile0 + (a / bs) * row_tile_step) * bs + a % bs (columns
// likewise); pred = that row's global id where the edge exists (i != j, both
// below n, dist finite), else -1.
template <typename T>
__global__ void __launch_bounds__(256)
    k_block_init(const T* D, int32_t* P, int64_t ld, int64_t rows, int64_t cols, int bs,
                 int64_t n, int64_t rt0, int64_t rts, int64_t ct0, int64_t cts) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / cols, c = e - a * cols;
    const int64_t gi = (rt0 + (a / bs) * rts) * bs + a % bs;
    const int64_t gj = (ct0 + (c / bs) * cts) * bs + c % bs;
    const T w = D[a * ld + c];
    P[a * ld + c] = (gi != gj && gi < n && gj < n && Num<T>::finite(w)) ? (int32_t)gi : -1;
  }
}

}  // namespace fwk

namespace fwh {
int* status_word_for(cudaStream_t s);  // fw_api.cu
int dtype_size(fw_dtype dtype);
bool dtype_valid(fw_dtype dtype);
}  // namespace fwh

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename T>
fw_status closure_bs(T* D, int32_t* P, int64_t ld, int bs, int* st, cudaStream_t s) {
  switch (bs) {
    case 32: fwk::k_tile_closure<T, 32><<<1, fwk::kThreads, 0, s>>>(D, P, ld, st); break;
    case 64: fwk::k_tile_closure<T, 64><<<1, fwk::kThreads, 0, s>>>(D, P, ld, st); break;
    case 128:
      if constexpr (sizeof(T) == 4) {
        fwk::k_tile_closure<T, 128><<<1, fwk::kThreads, 0, s>>>(D, P, ld, st);
        break;
      }
      return FW_ERR_UNSUPPORTED;
    default: return FW_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

template <typename T, int BS>
fw_status minplus_bs(T* C, int32_t* Pc, int64_t ldc, const T* A, int64_t lda, const T* B,
                     int64_t ldb, const int32_t* Pb, int64_t ldpb, int64_t tm, int64_t tn,
                     int64_t si, int64_t sj, cudaStream_t s) {
  auto kern = fwk::k_tile_minplus<T, BS>;
  const size_t smem = (size_t)BS * BS * (2 * sizeof(T) + 4);
  if (fwh::kernel_setup(reinterpret_cast<const void*>(kern), smem, fwk::kThreads) < 1)
    return FW_ERR_CUDA;
  kern<<<dim3((unsigned)tn, (unsigned)tm), fwk::kThreads, smem, s>>>(C, Pc, ldc, A, lda, B, ldb,
                                                                     Pb, ldpb, si, sj);
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

template <typename T>
fw_status minplus_t(void* C, int32_t* Pc, int64_t ldc, const void* A, int64_t lda,
                    const void* B, int64_t ldb, const int32_t* Pb, int64_t ldpb, int64_t tm,
                    int64_t tn, int bs, int64_t si, int64_t sj, cudaStream_t s) {
  T* c = reinterpret_cast<T*>(C);
  const T* a = reinterpret_cast<const T*>(A);
  const T* b = reinterpret_cast<const T*>(B);
  switch (bs) {
    case 32: return minplus_bs<T, 32>(c, Pc, ldc, a, lda, b, ldb, Pb, ldpb, tm, tn, si, sj, s);
    case 64: return minplus_bs<T, 64>(c, Pc, ldc, a, lda, b, ldb, Pb, ldpb, tm, tn, si, sj, s);
    case 128:
      if constexpr (sizeof(T) == 4)
        return minplus_bs<T, 128>(c, Pc, ldc, a, lda, b, ldb, Pb, ldpb, tm, tn, si, sj, s);
      return FW_ERR_UNSUPPORTED;
    default: return FW_ERR_ARG;
  }
}

fw_status check_bs(int bs, fw_dtype dtype) {
  if (!fwh::dtype_valid(dtype)) return FW_ERR_ARG;
  if (bs != 32 && bs != 64 && bs != 128) return FW_ERR_ARG;
  if (bs == 128 && fwh::dtype_size(dtype) == 8) return FW_ERR_UNSUPPORTED;
  return FW_OK;
}

}  // namespace

extern "C" {

fw_status fw_tile_closure(void* tile, int32_t* pred, int64_t ld, int32_t bs, fw_dtype dtype,
                          void* stream) {
  fw_status st = check_bs(bs, dtype);
  if (st != FW_OK) return st;
  if (!tile || ld < bs || (ld % 4) != 0 || !aligned16(tile) || !aligned16(pred))
    return FW_ERR_ARG;
  if ((void*)pred == tile) return FW_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* status = fwh::status_word_for(s);
  if (!status) return FW_ERR_NOMEM;
  switch (dtype) {
    case FW_I32: return closure_bs(reinterpret_cast<int32_t*>(tile), pred, ld, bs, status, s);
    case FW_F32: return closure_bs(reinterpret_cast<float*>(tile), pred, ld, bs, status, s);
    case FW_I64: return closure_bs(reinterpret_cast<int64_t*>(tile), pred, ld, bs, status, s);
    default: return closure_bs(reinterpret_cast<double*>(tile), pred, ld, bs, status, s);
  }
}

fw_status fw_tile_minplus(void* C, int32_t* Pc, int64_t ldc, const void* A, int64_t lda,
                          const void* B, int64_t ldb, const int32_t* Pb, int64_t ldpb,
                          int64_t tiles_m, int64_t tiles_n, int32_t bs, int64_t skip_tile_row,
                          int64_t skip_tile_col, fw_dtype dtype, void* stream) {
  fw_status st = check_bs(bs, dtype);
  if (st != FW_OK) return st;
  if (!C || !A || !B || (!Pc) != (!Pb)) return FW_ERR_ARG;
  if (tiles_m < 0 || tiles_n < 0 || tiles_m > 65535 || tiles_n > ((int64_t)1 << 31) - 1)
    return FW_ERR_ARG;
  if (ldc < tiles_n * bs || lda < bs || ldb < tiles_n * bs || (Pc && ldpb < tiles_n * bs))
    return FW_ERR_ARG;
  if ((ldc % 4) || (lda % 4) || (ldb % 4) || (Pc && (ldpb % 4))) return FW_ERR_ARG;
  if (!aligned16(C) || !aligned16(A) || !aligned16(B) || !aligned16(Pc) || !aligned16(Pb))
    return FW_ERR_ARG;
  // C may share storage with A only for one tile column, with B only for one
  // tile row (each CTA then reads exactly the tile it writes)
  if (C == A && !(tiles_n == 1 && lda == ldc)) return FW_ERR_ARG;
  if (C == B && !(tiles_m == 1 && ldb == ldc)) return FW_ERR_ARG;
  if (Pc && Pc == Pb && !(tiles_m == 1 && ldpb == ldc)) return FW_ERR_ARG;
  if (tiles_m == 0 || tiles_n == 0) return FW_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  switch (dtype) {
    case FW_I32:
      return minplus_t<int32_t>(C, Pc, ldc, A, lda, B, ldb, Pb, ldpb, tiles_m, tiles_n, bs,
                                skip_tile_row, skip_tile_col, s);
    case FW_F32:
      return minplus_t<float>(C, Pc, ldc, A, lda, B, ldb, Pb, ldpb, tiles_m, tiles_n, bs,
                              skip_tile_row, skip_tile_col, s);
    case FW_I64:
      return minplus_t<int64_t>(C, Pc, ldc, A, lda, B, ldb, Pb, ldpb, tiles_m, tiles_n, bs,
                                skip_tile_row, skip_tile_col, s);
    default:
      return minplus_t<double>(C, Pc, ldc, A, lda, B, ldb, Pb, ldpb, tiles_m, tiles_n, bs,
                               skip_tile_row, skip_tile_col, s);
  }
}

fw_status fw_block_init_pred(const void* dist, int32_t* pred, int64_t ld, int64_t rows,
                             int64_t cols, int32_t bs, int64_t n, int64_t row_tile0,
                             int64_t row_tile_step, int64_t col_tile0, int64_t col_tile_step,
                             fw_dtype dtype, void* stream) {
  if (!fwh::dtype_valid(dtype) || !dist || !pred || bs < 1 || rows < 0 || cols < 0 ||
      ld < cols || n < 0 || row_tile0 < 0 || col_tile0 < 0 || row_tile_step < 1 ||
      col_tile_step < 1)
    return FW_ERR_ARG;
  if (rows == 0 || cols == 0) return FW_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t blocks = (rows * cols + 255) / 256;
  if (blocks > (int64_t)fwh::num_sms() * 8) blocks = (int64_t)fwh::num_sms() * 8;
  switch (dtype) {
    case FW_I32:
      fwk::k_block_init<int32_t><<<(int)blocks, 256, 0, s>>>(
          reinterpret_cast<const int32_t*>(dist), pred, ld, rows, cols, bs, n, row_tile0,
          row_tile_step, col_tile0, col_tile_step);
      break;
    case FW_F32:
      fwk::k_block_init<float><<<(int)blocks, 256, 0, s>>>(
          reinterpret_cast<const float*>(dist), pred, ld, rows, cols, bs, n, row_tile0,
          row_tile_step, col_tile0, col_tile_step);
      break;
    case FW_I64:
      fwk::k_block_init<int64_t><<<(int)blocks, 256, 0, s>>>(
          reinterpret_cast<const int64_t*>(dist), pred, ld, rows, cols, bs, n, row_tile0,
          row_tile_step, col_tile0, col_tile_step);
      break;
    default:
      fwk::k_block_init<double><<<(int)blocks, 256, 0, s>>>(
          reinterpret_cast<const double*>(dist), pred, ld, rows, cols, bs, n, row_tile0,
          row_tile_step, col_tile0, col_tile_step);
      break;
  }
  return cudaGetLastError() == cudaSuccess ? FW_OK : FW_ERR_CUDA;
}

}  // extern "C"
