// Split-precision (TF32x3) contraction on tcgen05 tensor cores: interface.
#pragma once

#include <cuda.h>

#include "qrctm_internal.cuh"

namespace qrctm {

// A K-contiguous FP32 operand: element (b, r, k) at ptr[b*batch_stride + r*row_stride + k].
// row_stride and batch_stride (elements) must be multiples of 4 (16 bytes)
// and ptr 16-byte aligned (TMA rules).
// lo != nullptr marks a pre-split operand: ptr holds the TF32 heads and lo
// the TF32 tails (tf32_split, same layout), so the kernel splits nothing; an
// operand reused by many output tiles is split once instead of per tile.
// A may come pre-split only together with B.
struct TcOperand {
  const float* ptr;
  long long rows;
  long long K;
  long long row_stride;
  int batch;               // 1 = shared by every batch entry
  long long batch_stride;
  const float* lo;
};

// D[b](m,n) = alpha * sum_k A[b](m,k) B[b](n,k) + beta * D[b](m,n), D stored
// through index maps, FP32 or FP64.
struct TcGemm {
  TcOperand A, B;
  long long M, N, K;
  int batch;
  void* C;
  bool c_fp64;
  IdxMap c_m, c_n, c_b;
  double alpha, beta;
  int* err;
  // optional split-K scratch (FP32 partial sums, part_elems floats); long K
  // ranges are cut into chunks of at most 512 that are summed in FP64
  float* part;
  long long part_elems;
  // partials_only: write the raw K-chunk partials part[b][z][m][n] (always,
  // even for one chunk) and skip the reduction; *ksplit_out gets the number
  // of chunks.  The consumer sums them.  C, alpha, beta are ignored.
  bool partials_only;
  int* ksplit_out;
  int max_ksplit;      // cap on the number of K chunks (0 = no cap)
  // optional FP32 copy of the final FP64 result (c_fp64 only, no batch):
  // C32[c32_m(m) + c32_n(n)] = (float) D(m, n)
  float* C32;
  IdxMap c32_m, c32_n;
};

// Kernel arguments (device side).
struct TcArgs {
  long long M, N, K;
  void* C;
  int c_fp64;
  IdxMap c_m, c_n, c_b;
  double alpha, beta;
  int a_batched, b_batched;
  int* err;
  int ksplit;          // K chunks per output tile (1 = no split)
  int kb_per_split;    // 32-wide K blocks per chunk
  float* part;         // ksplit > 1 or partials_only: partials [batch][ksplit][M][N]
  int partials_only;
  int batch;           // batch entries (persistent kernel's tile count)
  float* C32;          // optional FP32 copy of the FP64 result
  IdxMap c32_m, c32_n;
};

cudaError_t gemm_tc(const TcGemm& g, cudaStream_t s);

// 2-D TMA map over an FP32 matrix of rows x cols (row stride in elements,
// a multiple of 4; base 16-byte aligned), box box_cols x box_rows, no
// swizzle.  False when the driver's encoder is unavailable or a rule fails.
bool make_map_2d_f32(CUtensorMap* tm, const float* base, long long cols, long long rows,
                     long long row_stride, int box_cols, int box_rows);

}  // namespace qrctm
