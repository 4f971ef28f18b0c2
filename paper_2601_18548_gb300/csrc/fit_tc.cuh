// BF16 tensor-core GEMM used by the differentiable fit (fit_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gcdf {

// What the GEMM's epilogue does with the FP32 accumulator tile before storing.
enum GemmEpiMode : int {
  kEpiStore = 0,     // C = acc (or C += acc)
  kEpiBiasSilu = 1,  // z = acc + bias[n]: C = s(z), s_out = s'(z), s2_out = s''(z)
  kEpiMul = 2        // C = acc * s_in[m, n] (+ add_in[m, n] when given); acc_out = acc
};

// Outputs besides C (each optional, NULL = not written).  img: BF16 copy of
// the stored result, row-major with row stride ld_img; imgT: BF16 copy
// transposed (imgT[n ld_imgT + m]); colsum: per 32-row block b of C the
// column sums of the result, colsum[b ld_colsum + n].  C itself may be NULL
// when only these are wanted.  Not combined with split-K partials.
struct GemmEpilogue {
  int mode;
  const float* bias;
  const float* s_in;
  const float* add_in;   // kEpiMul: added after the multiply (row stride ld_s), or NULL
  float* acc_out;        // kEpiMul: the accumulator before the multiply (row stride ld_s), or NULL
  float* s_out;
  float* s2_out;
  long long ld_s;
  __nv_bfloat16* img;
  long long ld_img;
  __nv_bfloat16* imgT;
  long long ld_imgT;
  float* colsum;
  long long ld_colsum;
};

// Tile of one CTA pair (rows of C x columns of C) and the K granularity.
int tc_gemm_tile_m();
int tc_gemm_tile_n();
int tc_gemm_kblock();

// C_z = A B^T over the K-blocks [z kb_per_split, (z + 1) kb_per_split) for
// z < splits, written (or added, with accumulate) at C + z zstride with row
// stride ldc.  A: M x K and B: N x K BF16 row-major DEVICE images with row
// strides lda, ldb (multiples of 8 elements; 16-byte aligned bases).
// Every split must hold at least one K-block.  Sets *encode_failed when a
// tensor map cannot be built (nothing launched).
cudaError_t tc_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, int M, int N, int K, float* C,
                         long long ldc, long long zstride, int splits, int kb_per_split, bool accumulate, int* err,
                         cudaStream_t s, bool* encode_failed, const GemmEpilogue* ep = nullptr);

// The device status word of the fit's tensor-core kernels on the current
// device (allocated on first use; NULL if that fails).
int* fit_status_word();

}  // namespace gcdf
