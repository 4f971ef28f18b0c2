// BF16 tensor-core GEMM used by the differentiable fit (fit_tc.cu).
#pragma once

#include <cuda_runtime.h>

namespace gcdf {

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
                         cudaStream_t s, bool* encode_failed);

// The device status word of the fit's tensor-core kernels on the current
// device (allocated on first use; NULL if that fails).
int* fit_status_word();

}  // namespace gcdf
