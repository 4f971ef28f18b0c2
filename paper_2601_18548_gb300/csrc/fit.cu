// Differentiable fit of the field (Sec. III-C, distance loss of Table I):
// per-sample values f(q_b, p_b) of an FP32 net given by its flat weights, and
// the vector-Jacobian products with respect to the weights and q for an
// upstream gradient g_b = dL/df_b.
//
//   forward   v = [p, x, y, sin a, cos a, ...]; z_1 = W_1 v + b_1; h_l = s(z_l);
//             z_{l+1} = W_{l+1} h_l + b_{l+1}; f = w_o . h_L + b_o
//   backward  delta_L = g w_o * s'(z_L); delta_{l-1} = (delta_l W_l) * s'(z_{l-1});
//             dW_l = delta_l^T h_{l-1}; db_l = sum_b delta_l; dw_o = h_L^T g; db_o = sum_b g;
//             dv = delta_1 W_1 -> dq (sin/cos chain rule)
//
// The regularisers of Table I (gradient direction, eikonal, tension) are
// functions of grad_q f, so training on them needs the weight gradient of
// sum_b G_b . grad_q f_b: a second-order product.  With a_l the factor of the
// reverse sweep (a_L = w_o, delta_l = a_l * s'(z_l), a_{l-1} = delta_l W_l),
// u = C^T G (C the sin/cos chain rule dv -> dq) and r_1 = u W_1^T,
// r_{l+1} = (r_l * s'(z_l)) W_{l+1}^T:
//   dW_1 += delta_1^T u;  dW_{l+1} += delta_{l+1}^T (r_l * s'(z_l));  dw_o += sum_b r_L * s'(z_L)
// and the second-derivative terms e_l = r_l * a_l * s''(z_l) run back through
// the network with the value term g:
//   eps_L = e_L + g w_o * s'(z_L);  eps_{l-1} = e_{l-1} + (eps_l W_l) * s'(z_{l-1})
//   dW_l += eps_l^T h_{l-1};  db_l = sum_b eps_l;  dw_o += h_L^T g;  db_o = sum_b g
//
// Every matrix product is one strided FP32 GEMM kernel (128 x 128 tiles, 8 x 8
// outputs per thread) or, with BF16 precision, the tcgen05 GEMM of fit_tc.cu on
// BF16 images of its operands (FP32 accumulation; the activations, s'(z) and
// every element-wise step stay FP32); the vector products (the output f, the bias and
// output-weight gradients) are a warp-per-row dot and a column reduction.
// Whatever reduces over the batch (weight and bias gradients) splits it into
// chunks whose partials are summed in a fixed order: deterministic gradients.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fit_tc.cuh"
#include "gcdf_internal.cuh"

namespace gcdf {

int set_error(int code, const char* fmt, ...);
void clear_error();

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 8, kGemmThreads = 256;

// C[m, n] (row-major, ldc) = sum_k A(m, k) B(k, n) over k in this block's
// chunk [z kc, min(K, (z + 1) kc)); with z > 0 chunks the block writes its
// partial tile to C + z M ldc.
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_kernel(const float* __restrict__ A, long long sam, long long sak,
                                                            const float* __restrict__ B, long long sbk,
                                                            long long sbn, float* __restrict__ C, int ldc, int M,
                                                            int N, int K, int kc, int accumulate) {
  // two shared buffers: the next K block's elements are fetched into registers
  // before this block's products and stored to the other buffer after them,
  // so one barrier per K block separates the two (same summation order as a
  // single buffer)
  __shared__ __align__(16) float As[2][kBK][kBM];
  __shared__ __align__(16) float Bs[2][kBK][kBN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  const int k_lo = blockIdx.z * kc, k_hi = min(K, k_lo + kc);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const bool a_kfast = (sak == 1), b_nfast = (sbn == 1);
  constexpr int kRA = (kBK * kBM) / kGemmThreads, kRB = (kBK * kBN) / kGemmThreads;
  float ra[kRA], rb[kRB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < kRA; ++r) {
      const int e = threadIdx.x + r * kGemmThreads;
      const int mm = a_kfast ? e / kBK : e % kBM;
      const int kk = a_kfast ? e % kBK : e / kBM;
      const int m = m0 + mm, k = k0 + kk;
      ra[r] = (m < M && k < k_hi) ? A[(long long)m * sam + (long long)k * sak] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < kRB; ++r) {
      const int e = threadIdx.x + r * kGemmThreads;
      const int nn = b_nfast ? e % kBN : e / kBK;
      const int kk = b_nfast ? e / kBN : e % kBK;
      const int n = n0 + nn, k = k0 + kk;
      rb[r] = (n < N && k < k_hi) ? B[(long long)k * sbk + (long long)n * sbn] : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int r = 0; r < kRA; ++r) {
      const int e = threadIdx.x + r * kGemmThreads;
      As[buf][a_kfast ? e % kBK : e / kBM][a_kfast ? e / kBK : e % kBM] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < kRB; ++r) {
      const int e = threadIdx.x + r * kGemmThreads;
      Bs[buf][b_nfast ? e / kBN : e % kBK][b_nfast ? e % kBN : e / kBK] = rb[r];
    }
  };
  if (k_lo < k_hi) {
    fetch(k_lo);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = k_lo; k0 < k_hi; k0 += kBK) {
    const bool more = k0 + kBK < k_hi;
    if (more) fetch(k0 + kBK);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* Cz = C + (long long)blockIdx.z * M * ldc;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (n < N) {
        float* c = Cz + (long long)m * ldc + n;
        *c = accumulate ? *c + acc[i][j] : acc[i][j];
      }
    }
  }
}

// C = sum over z of the partial tiles, in increasing z.
__global__ void sum_partials_kernel(const float* __restrict__ P, int splits, int M, int N, int ldp,
                                    float* __restrict__ C, int ldc, int accumulate) {
  // grid: x over columns, y over rows (grid-strided), so no index division
  for (int m = blockIdx.y; m < M; m += gridDim.y)
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
      float s = 0.f;
#pragma unroll 8
      for (int z = 0; z < splits; ++z) s += P[((long long)z * M + m) * ldp + n];
      C[(long long)m * ldc + n] = accumulate ? C[(long long)m * ldc + n] + s : s;
    }
}

// launch shape of sum_partials_kernel for an M x N result
dim3 partials_grid(int M, int N) {
  const int gx = (N + 255) / 256, gy = M;
  return dim3((unsigned)(gx < 1 ? 1 : (gx < 64 ? gx : 64)), (unsigned)(gy < 1 ? 1 : (gy < 65535 ? gy : 65535)));
}

// out[c] = sum_b X[b, c] w_b (w NULL: 1) over the rows of one of `chunks`
// consecutive row chunks: partial[chunk, c] (thread = column, coalesced rows).
__global__ void colsum_kernel(const float* __restrict__ X, int rows, int C, const float* __restrict__ w, int chunks,
                              float* __restrict__ partial) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int per = (rows + chunks - 1) / chunks;
  const int r0 = blockIdx.y * per, r1 = min(rows, r0 + per);
  float s = 0.f;
#pragma unroll 8
  for (int b = r0; b < r1; ++b) s = fmaf(X[(long long)b * C + c], w ? w[b] : 1.f, s);
  partial[(long long)blockIdx.y * C + c] = s;
}

// out[c] (= or +=) the sum of partial[k, c] over the chunks k, one warp per
// column: lane-strided sums, then a fixed butterfly (deterministic).
__global__ void colsum_finish_kernel(const float* __restrict__ partial, int chunks, int C, float* __restrict__ out,
                                     int accumulate) {
  const int c = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  float s = 0.f;
  for (int k = lane; k < chunks; k += 32) s += partial[(long long)k * C + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = accumulate ? out[c] + s : s;
}

// f_b = X[b, :] . v + *c0, one warp per row (lane-strided sums, fixed butterfly).
__global__ void rowdot_kernel(const float* __restrict__ X, int rows, int C, const float* __restrict__ v,
                              const float* __restrict__ c0, float* __restrict__ f) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const float* x = X + warp * C;
  float s = 0.f;
  for (int c = lane; c < C; c += 32) s = fmaf(x[c], v[c], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) f[warp] = s + *c0;
}

// v = [p, x, y, sin a_1, cos a_1, ...] per sample.
__global__ void encode_kernel(const float* __restrict__ q, const float* __restrict__ p, int B, int n, int d_in,
                              float* __restrict__ X) {
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
    float* x = X + b * d_in;
    const float* qb = q + b * n;
    x[0] = p[3 * b];
    x[1] = p[3 * b + 1];
    x[2] = p[3 * b + 2];
    x[3] = qb[0];
    x[4] = qb[1];
    for (int a = 0; a < n - 2; ++a) {
      float s, c;
      sincosf(qb[2 + a], &s, &c);
      x[5 + 2 * a] = s;
      x[6 + 2 * a] = c;
    }
  }
}

// z += b (per column); h = s(z) in place; s'(z) -> S; s''(z) -> S2 unless NULL.
// With sg = 1 / (1 + e^-z): s = z sg, s' = sg (1 + z (1 - sg)),
// s'' = sg (1 - sg) (2 + z (1 - 2 sg)).
__global__ void bias_silu_kernel(float* __restrict__ Z, const float* __restrict__ bias, long long rows, int H,
                                 float* __restrict__ S, float* __restrict__ S2) {
  const long long total = rows * H;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float z = Z[e] + bias[e % H];
    const float sg = 1.f / (1.f + expf(-z));
    Z[e] = z * sg;
    S[e] = sg * (1.f + z * (1.f - sg));
    if (S2) S2[e] = sg * (1.f - sg) * (2.f + z * (1.f - 2.f * sg));
  }
}

// delta_L = g w_o * S_L (g NULL: 1)
__global__ void seed_kernel(const float* __restrict__ g, const float* __restrict__ wo, const float* __restrict__ S,
                            long long rows, int H, float* __restrict__ D) {
  const long long total = rows * H;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    D[e] = (g ? g[e / H] : 1.f) * wo[e % H] * S[e];
}

// O = X * Y elementwise (O may alias X or Y)
__global__ void mul2_kernel(float* O, const float* X, const float* Y, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    O[e] = X[e] * Y[e];
}

// E = r * a * S2 with a = A, or the broadcast row wo when A is NULL (E may alias A)
__global__ void second_kernel(const float* __restrict__ R, const float* A, const float* __restrict__ wo,
                              const float* __restrict__ S2, long long rows, int H, float* E) {
  const long long total = rows * H;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    E[e] = R[e] * (A ? A[e] : wo[e % H]) * S2[e];
}

// X = Y + X * S  (eps_{l-1} = e_{l-1} + back * s'(z_{l-1}))
__global__ void addmul_kernel(float* __restrict__ X, const float* __restrict__ S, const float* __restrict__ Y,
                              long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    X[e] = Y[e] + X[e] * S[e];
}

// E += g w_o * S  (the value term of eps_L)
__global__ void seed_add_kernel(const float* __restrict__ g, const float* __restrict__ wo,
                                const float* __restrict__ S, long long rows, int H, float* __restrict__ E) {
  const long long total = rows * H;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    E[e] += g[e / H] * wo[e % H] * S[e];
}

// u = C^T G: the adjoint of the sin/cos chain rule (zeros at the point columns)
__global__ void dq_adjoint_kernel(const float* __restrict__ q, const float* __restrict__ G, int B, int n, int d_in,
                                  float* __restrict__ U) {
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
    const float* gb = G + b * n;
    float* u = U + b * d_in;
    u[0] = u[1] = u[2] = 0.f;
    u[3] = gb[0];
    u[4] = gb[1];
    for (int a = 0; a < n - 2; ++a) {
      float sn, cs;
      sincosf(q[b * n + 2 + a], &sn, &cs);
      u[5 + 2 * a] = cs * gb[2 + a];
      u[6 + 2 * a] = -sn * gb[2 + a];
    }
  }
}

__global__ void mul_kernel(float* __restrict__ D, const float* __restrict__ S, long long total) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    D[e] *= S[e];
}

// dq from dv: x, y direct; angle a: cos a dv[sin a] - sin a dv[cos a]
__global__ void dq_kernel(const float* __restrict__ q, const float* __restrict__ dV, int B, int n, int d_in,
                          float* __restrict__ dq) {
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
    const float* v = dV + b * d_in;
    float* o = dq + b * n;
    o[0] = v[3];
    o[1] = v[4];
    for (int a = 0; a < n - 2; ++a) {
      float s, c;
      sincosf(q[b * n + 2 + a], &s, &c);
      o[2 + a] = c * v[5 + 2 * a] - s * v[6 + 2 * a];
    }
  }
}

int grid1(long long work) {
  const long long b = (work + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

struct Ws {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Ws(cudaStream_t st) : s(st) {}
  template <class T>
  cudaError_t get(T** out, size_t count) {
    size_t bytes = count * sizeof(T);
    cudaError_t e = lib_malloc_async((void**)out, bytes < 16 ? 16 : bytes, s);
    if (e == cudaSuccess) ptrs.push_back(*out);
    return e;
  }
  ~Ws() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// C (M x N, ldc) = (or +=, with accumulate) A(m, k) B(k, n) summed over K; the
// batch-length reductions (large K, few output tiles) go through `splits`
// chunks and the partials array.
cudaError_t gemm(const float* A, long long sam, long long sak, const float* B, long long sbk, long long sbn,
                 float* C, int ldc, int M, int N, int K, float* partials, size_t partial_floats, cudaStream_t s,
                 bool accumulate = false) {
  if (M == 0 || N == 0) return cudaSuccess;
  const int tm = (M + kBM - 1) / kBM, tn = (N + kBN - 1) / kBN;
  int splits = 1;
  if ((long long)tm * tn < 2 * 152 && K > 4096 && partials) {
    splits = (int)std::min<long long>(64, (K + 1023) / 1024);
    while (splits > 1 && (size_t)splits * M * N > partial_floats) --splits;
  }
  const int kc = ((K + splits - 1) / splits + kBK - 1) / kBK * kBK;
  splits = (K + kc - 1) / kc;
  if (splits < 1) splits = 1;
  dim3 grid(tn, tm, splits);
  if (splits == 1) {
    gemm_kernel<<<grid, kGemmThreads, 0, s>>>(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, kc, accumulate ? 1 : 0);
  } else {
    gemm_kernel<<<grid, kGemmThreads, 0, s>>>(A, sam, sak, B, sbk, sbn, partials, N, M, N, K, kc, 0);
    sum_partials_kernel<<<partials_grid(M, N), 256, 0, s>>>(partials, splits, M, N, N, C, ldc, accumulate ? 1 : 0);
  }
  return cudaGetLastError();
}

// out (C) = X^T w over the batch (w NULL: column sums), in a fixed order.
cudaError_t colsum(const float* X, int rows, int C, const float* w, float* out, float* partials, size_t pfl,
                   cudaStream_t s, bool accumulate = false) {
  // enough row chunks that no thread walks more than ~32 rows (up to 1,024
  // chunks and the partials array), then one warp per column over the chunks
  int chunks = (rows + 31) / 32;
  if (chunks > 1024) chunks = 1024;
  if (chunks < 1) chunks = 1;
  while (chunks > 1 && (size_t)chunks * C > pfl) --chunks;
  dim3 grid((C + 255) / 256, chunks);
  colsum_kernel<<<grid, 256, 0, s>>>(X, rows, C, w, chunks, partials);
  colsum_finish_kernel<<<(unsigned)((C + 7) / 8), 256, 0, s>>>(partials, chunks, C, out, accumulate ? 1 : 0);
  return cudaGetLastError();
}

// Y (rows x cols, row stride ldy) = BF16 rounding of X (rows x cols, row stride ldx)
__global__ void cast_bf16_kernel(const float* __restrict__ X, long long rows, int cols, long long ldx,
                                 __nv_bfloat16* __restrict__ Y, long long ldy) {
  for (long long r = blockIdx.x; r < rows; r += gridDim.x)
    for (int c = threadIdx.x; c < cols; c += blockDim.x) Y[r * ldy + c] = __float2bfloat16_rn(X[r * ldx + c]);
}

// Y[c, r] = BF16 rounding of X[r, c] for X rows x cols (row stride ldx), Y cols x
// rows (row stride ldy): 32 x 32 tiles through shared memory, block 32 x 8
// (blockIdx.x: row tile, blockIdx.y: column tile).
__global__ void transpose_bf16_kernel(const float* __restrict__ X, long long rows, int cols, long long ldx,
                                      __nv_bfloat16* __restrict__ Y, long long ldy) {
  __shared__ float t[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const long long r = r0 + i;
    const int c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < rows && c < cols) ? X[r * ldx + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i;
    const long long r = r0 + threadIdx.x;
    if (c < cols && r < rows) Y[(long long)c * ldy + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
  }
}

long long pad8(long long x) { return (x + 7) / 8 * 8; }

// The BF16 weight images of every layer in one launch: W_l (H x K_l, row stride
// K_l) rounded row by row into Wr[l] (row stride pad8(K_l)) and transposed into
// Wt[l] (K_l x H), either absent per layer.  32 x 32 tiles of all layers in one
// grid (tile0: the first tile of each layer), block 32 x 8.
struct WeightImages {
  const float* W[16];
  __nv_bfloat16* Wr[16];
  __nv_bfloat16* Wt[16];
  int K[16];
  int tile0[17];
  int H, L;
};

__global__ void weight_images_kernel(const WeightImages a) {
  __shared__ float t[32][33];
  int l = 0;
  while (l + 1 < a.L && (int)blockIdx.x >= a.tile0[l + 1]) ++l;
  const int K = a.K[l], H = a.H;
  const int tile = (int)blockIdx.x - a.tile0[l];
  const int tcols = (K + 31) / 32;
  const int r0 = (tile / tcols) * 32, c0 = (tile % tcols) * 32;  // rows over H, columns over K
  const float* W = a.W[l];
  __nv_bfloat16* Wr = a.Wr[l];
  const long long ldr = (K + 7) / 8 * 8;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    const bool in = r < H && c < K;
    const float v = in ? W[(long long)r * K + c] : 0.f;
    t[i][threadIdx.x] = v;
    if (in && Wr) Wr[(long long)r * ldr + c] = __float2bfloat16_rn(v);
  }
  __nv_bfloat16* Wt = a.Wt[l];
  if (Wt) {  // the same for the whole block
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int c = c0 + i, r = r0 + threadIdx.x;
      if (c < K && r < H) Wt[(long long)c * H + r] = __float2bfloat16_rn(t[threadIdx.x][i]);
    }
  }
}

// One launch of weight_images_kernel for layers 1..L of the flat weights w
// (layer l at w_off[l], fan-in K[l]); Wr / Wt indexed by layer, entries may be
// NULL (the arrays themselves too).
cudaError_t weight_images(const float* w, const long long* w_off, const int* K, int L, int H,
                          __nv_bfloat16* const* Wr, __nv_bfloat16* const* Wt, cudaStream_t s) {
  if (L < 1 || L > 16) return cudaErrorInvalidValue;
  WeightImages a{};
  a.H = H;
  a.L = L;
  int tiles = 0;
  for (int l = 1; l <= L; ++l) {
    a.W[l - 1] = w + w_off[l];
    a.Wr[l - 1] = Wr ? Wr[l] : nullptr;
    a.Wt[l - 1] = Wt ? Wt[l] : nullptr;
    a.K[l - 1] = K[l];
    a.tile0[l - 1] = tiles;
    tiles += ((H + 31) / 32) * ((K[l] + 31) / 32);
  }
  a.tile0[L] = tiles;
  if (tiles == 0) return cudaSuccess;
  weight_images_kernel<<<tiles, dim3(32, 8), 0, s>>>(a);
  return cudaGetLastError();
}

// The products of one call: FP32 SIMT GEMMs, or the BF16 tensor-core GEMM on
// K-major BF16 images of both operands (an operand whose K index is already the
// contiguous one is rounded row by row, the other one is transposed).
struct Ctx {
  cudaStream_t s;
  float* partials = nullptr;
  size_t pfl = 0;
  bool bf16 = false;
  __nv_bfloat16 *sa = nullptr, *sb = nullptr;
  size_t cap = 0;  // elements of sa and of sb
  int* err = nullptr;

  // the operand images for products among batch B and widths up to maxK
  cudaError_t reserve(Ws& ws, long long B, long long maxK) {
    if (!bf16) return cudaSuccess;
    cap = (size_t)std::max({maxK * pad8(B), B * pad8(maxK), maxK * pad8(maxK)});
    cudaError_t e;
    if ((e = ws.get(&sa, cap)) || (e = ws.get(&sb, cap))) return e;
    err = fit_status_word();
    return err ? cudaSuccess : cudaErrorMemoryAllocation;
  }

  // K-major BF16 image (rows x K, row stride ld) of X(r, k) = X[r srow + k sk]
  cudaError_t image(const float* X, long long srow, long long sk, int rows, int K, __nv_bfloat16* Y, long long ld) {
    if (sk == 1) {
      cast_bf16_kernel<<<(int)std::min<long long>(rows, 152 * 16), 128, 0, s>>>(X, rows, K, srow, Y, ld);
    } else if (srow == 1) {  // X is K x rows with row stride sk
      if ((rows + 31) / 32 > 65535) return cudaErrorInvalidValue;  // grid y limit (rows are feature widths)
      dim3 grid((unsigned)((K + 31) / 32), (unsigned)((rows + 31) / 32));
      transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(X, K, rows, sk, Y, ld);
    } else {
      return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }

  // C (M x N, ldc) = (or +=) A(m, k) B(k, n) summed over K; `split`: the
  // product may split K over the partials array
  cudaError_t mm(const float* A, long long sam, long long sak, const float* B, long long sbk, long long sbn, float* C,
                 int ldc, int M, int N, int K, bool split, bool accumulate = false) {
    if (!bf16) return gemm(A, sam, sak, B, sbk, sbn, C, ldc, M, N, K, split ? partials : nullptr, split ? pfl : 0, s,
                           accumulate);
    if (M == 0 || N == 0) return cudaSuccess;
    const long long ld = pad8(K);
    if ((size_t)M * ld > cap || (size_t)N * ld > cap) return cudaErrorInvalidValue;
    cudaError_t e;
    // A(m, k) = A[m sam + k sak]; B as an N x K operand: B(k, n) = B[n sbn + k sbk]
    if ((e = image(A, sam, sak, M, K, sa, ld)) || (e = image(B, sbn, sbk, N, K, sb, ld))) return e;
    return mm_images(sa, ld, sb, ld, M, N, K, C, ldc, split, accumulate, nullptr);
  }

  // C (M x N, ldc) = (or +=) A B^T on BF16 images A (M x K, row stride lda) and
  // B (N x K, ldb), with an optional fused epilogue (not with `split`)
  cudaError_t mm_images(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B, long long ldb, int M, int N,
                        int K, float* C, long long ldc, bool split, bool accumulate, const GemmEpilogue* ep) {
    if (M == 0 || N == 0) return cudaSuccess;
    cudaError_t e;
    const int kb = tc_gemm_kblock();
    const long long kblocks = (K + kb - 1) / kb;
    const long long tiles = (long long)((M + tc_gemm_tile_m() - 1) / tc_gemm_tile_m()) *
                            ((N + tc_gemm_tile_n() - 1) / tc_gemm_tile_n());
    long long splits = 1;
    if (split && partials && tiles < 152 && kblocks >= 16) {
      splits = std::min<long long>((152 + tiles - 1) / tiles, kblocks / 8);
      while (splits > 1 && (size_t)splits * M * N > pfl) --splits;
    }
    if (ep) splits = 1;
    const long long per = (kblocks + splits - 1) / splits;
    splits = (kblocks + per - 1) / per;
    bool enc_fail = false;
    if (splits == 1) {
      e = tc_gemm_bf16(A, lda, B, ldb, M, N, K, C, ldc, 0, 1, (int)per, accumulate, err, s, &enc_fail, ep);
    } else {
      e = tc_gemm_bf16(A, lda, B, ldb, M, N, K, partials, N, (long long)M * N, (int)splits, (int)per, false, err, s,
                       &enc_fail);
      if (e == cudaSuccess && !enc_fail)
        sum_partials_kernel<<<partials_grid(M, N), 256, 0, s>>>(partials, (int)splits, M, N, N, C, ldc,
                                                                accumulate ? 1 : 0);
    }
    if (enc_fail) return cudaErrorInvalidValue;
    return e != cudaSuccess ? e : cudaGetLastError();
  }
};

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct Shape {
  int n, H, L, d_in;
  size_t off_out;  // offset of w_o in the flat layout
  size_t total;
  size_t off(int l) const {  // offset of W_l (l = 1 .. L)
    if (l == 1) return 0;
    return (size_t)H * d_in + H + (size_t)(l - 2) * ((size_t)H * H + H);
  }
  int fan_in(int l) const { return l == 1 ? d_in : H; }
  bool bf16;
};

int check(const gcdf_fit_desc* d, const float* w, const float* q, const float* p, int B, Shape& sh) {
  if (!d) return set_error(GCDF_EINVAL, "desc is NULL");
  if (d->n_dof < 3 || d->n_dof > kMaxDof || d->hidden < 1 || d->hidden > 4096 || d->n_hidden_layers < 1 ||
      d->n_hidden_layers > 16)
    return set_error(GCDF_EINVAL, "bad shape (n_dof %d, hidden %d, layers %d)", d->n_dof, d->hidden,
                     d->n_hidden_layers);
  if (d->precision != GCDF_FP32 && d->precision != GCDF_BF16)
    return set_error(GCDF_EINVAL, "fit precision %d is neither GCDF_FP32 nor GCDF_BF16", d->precision);
  if (B < 0) return set_error(GCDF_EINVAL, "batch %d < 0", B);
  if (B > 0 && (!w || !q || !p || !al16(w) || !al16(q) || !al16(p)))
    return set_error(GCDF_EINVAL, "weights, q or p NULL or not 16-byte aligned");
  sh.n = d->n_dof;
  sh.H = d->hidden;
  sh.L = d->n_hidden_layers;
  sh.d_in = 3 + 2 + 2 * (sh.n - 2);
  sh.off_out = sh.off(sh.L + 1);
  sh.total = sh.off_out + sh.H + 1;
  sh.bf16 = d->precision == GCDF_BF16;
  return GCDF_OK;
}

// Forward pass storing h_l (Hs[l], l = 0 .. L, Hs[0] = v), s'(z_l) (Ss[l - 1])
// and, when S2s is given, s''(z_l) (S2s[l - 1]).
int forward(const Shape& sh, const float* w, const float* q, const float* p, int B, float** Hs, float** Ss, float* f,
            Ctx& cx, float** S2s = nullptr) {
  const cudaStream_t s = cx.s;
  cudaError_t e;
  encode_kernel<<<grid1(B), 256, 0, s>>>(q, p, B, sh.n, sh.d_in, Hs[0]);
  for (int l = 1; l <= sh.L; ++l) {
    const int K = sh.fan_in(l);
    const float* W = w + sh.off(l);
    // Z (B x H) = H_{l-1} (B x K) W^T
    if ((e = cx.mm(Hs[l - 1], K, 1, W, 1, K, Hs[l], sh.H, B, sh.H, K, false)))
      return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    bias_silu_kernel<<<grid1((long long)B * sh.H), 256, 0, s>>>(Hs[l], W + (size_t)sh.H * K, B, sh.H, Ss[l - 1],
                                                                S2s ? S2s[l - 1] : nullptr);
  }
  if (f) {
    // f (B) = H_L w_o + b_o
    rowdot_kernel<<<(int)(((long long)B * 32 + 255) / 256), 256, 0, s>>>(Hs[sh.L], B, sh.H, w + sh.off_out,
                                                                      w + sh.off_out + sh.H, f);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit forward launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

// Reverse sweep of the field's own gradient: delta_l = a_l * s'(z_l) into
// D[l - 1], a_L = w_o, a_{l-1} = delta_l W_l into A[l - 2] (A[l - 2] may be
// D[l - 2]: then only delta survives), for l = L .. 1.
int reverse_sweep(const Shape& sh, const float* w, int B, float** Ss, float** D, float** A, Ctx& cx) {
  const cudaStream_t s = cx.s;
  const int H = sh.H;
  const long long n = (long long)B * H;
  seed_kernel<<<grid1(n), 256, 0, s>>>(nullptr, w + sh.off_out, Ss[sh.L - 1], B, H, D[sh.L - 1]);
  for (int l = sh.L; l >= 2; --l) {
    cudaError_t e = cx.mm(D[l - 1], H, 1, w + sh.off(l), H, 1, A[l - 2], H, B, H, H, false);
    if (e) return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    mul2_kernel<<<grid1(n), 256, 0, s>>>(D[l - 2], A[l - 2], Ss[l - 2], n);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "reverse sweep launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

// Context of the BF16 image path: no staging images (the producers write them).
int make_ctx_images(Ctx& cx, cudaStream_t s, float* partials, size_t pfl) {
  cx.s = s;
  cx.partials = partials;
  cx.pfl = pfl;
  cx.bf16 = true;
  cx.err = fit_status_word();
  if (!cx.err) return set_error(GCDF_ENOMEM, "fit status word unavailable");
  return GCDF_OK;
}

int make_ctx(Ctx& cx, Ws& ws, const Shape& sh, int B, cudaStream_t s, float* partials, size_t pfl) {
  cx.s = s;
  cx.partials = partials;
  cx.pfl = pfl;
  cx.bf16 = sh.bf16;
  cudaError_t e = cx.reserve(ws, B, std::max(sh.H, sh.d_in));
  if (e != cudaSuccess) return set_error(GCDF_ENOMEM, "fit operand images: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

// ---- BF16 path: operand images written by their producers -----------------------
//
// With BF16 products the operands are needed as BF16 images in two layouts:
// row-major (batch x features: the A operand of the layer and back products,
// whose K index is the feature) and transposed (features x batch: both
// operands of the batch-length weight-gradient products).  Instead of rounding
// FP32 arrays into images before every product, each producer writes them
// directly: the input encoding writes both images of v; a layer product's
// epilogue applies bias + SiLU and writes s'(z), the next layer's row image and
// the transposed image; a back product's epilogue multiplies by s'(z_{l-1})
// and writes both images of delta_{l-1} and its per-32-row column sums (the
// bias gradient, summed over the row blocks in a fixed order).  The rounding
// points are those of the generic path: every product operand is the BF16
// rounding of the FP32 value the generic path would have computed.

// v = [p, x, y, sin a, cos a, ...] as BF16 images Xr (B x ldr) and Xc (d_in x ldc)
__global__ void encode_bf16_kernel(const float* __restrict__ q, const float* __restrict__ p, int B, int n, int d_in,
                                   __nv_bfloat16* __restrict__ Xr, long long ldr, __nv_bfloat16* __restrict__ Xc,
                                   long long ldc) {
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
    float x[3 + 2 + 2 * kMaxAngles];
    const float* qb = q + b * n;
    x[0] = p[3 * b];
    x[1] = p[3 * b + 1];
    x[2] = p[3 * b + 2];
    x[3] = qb[0];
    x[4] = qb[1];
    for (int a = 0; a < n - 2; ++a) sincosf(qb[2 + a], &x[5 + 2 * a], &x[6 + 2 * a]);
    for (int k = 0; k < d_in; ++k) {
      const __nv_bfloat16 v = __float2bfloat16_rn(x[k]);
      Xr[b * ldr + k] = v;
      if (Xc) Xc[(long long)k * ldc + b] = v;
    }
  }
}

// delta_L = g w_o * s'(z_L) (g NULL: 1) straight into its BF16 images: row-major
// Dr (B x H) and transposed Dc (H x ldc, NULL: not written), with the column
// sums of every 32-row block in cs (NULL: none).  Block (32, 8) per 32 x 32 tile.
// seed_images_kernel over 32 x 128 blocks: lane tx handles columns c0 + tx + 32 k
// (k = 0..3) of rows ty, ty + 8, .. (four coalesced loads and stores per row
// and warp instruction), 16 elements per thread; the same arithmetic and the
// same column-sum order as seed_images_kernel.
__global__ void seed_images_wide_kernel(const float* __restrict__ g, const float* __restrict__ wo,
                                        const float* __restrict__ S, int B, int H, __nv_bfloat16* __restrict__ Dr,
                                        __nv_bfloat16* __restrict__ Dc, long long ldc, float* __restrict__ cs) {
  __shared__ float t[32][129];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 128;
  const int tx = threadIdx.x, ty = threadIdx.y;
  float wk[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) wk[k] = c0 + tx + 32 * k < H ? wo[c0 + tx + 32 * k] : 0.f;
  for (int i = ty; i < 32; i += 8) {
    const long long r = r0 + i;
    const float gr = (r < B && g) ? g[r] : 1.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = c0 + tx + 32 * k;
      float d = 0.f;
      if (r < B && c < H) {
        d = gr * wk[k] * S[r * H + c];
        Dr[r * H + c] = __float2bfloat16_rn(d);
      }
      t[i][tx + 32 * k] = d;
    }
  }
  __syncthreads();
  if (cs && ty < 4) {
    const int col = ty * 32 + tx, c = c0 + col;
    if (c < H) {
      float sum = 0.f;
      for (int i = 0; i < 32; ++i)
        if (r0 + i < B) sum += t[i][col];
      cs[(long long)blockIdx.x * H + c] = sum;
    }
  }
  if (Dc) {
    const long long r = r0 + tx;
    for (int cc = ty; cc < 128; cc += 8) {
      const int c = c0 + cc;
      if (c < H && r < B) Dc[(long long)c * ldc + r] = __float2bfloat16_rn(t[tx][cc]);
    }
  }
}

__global__ void seed_images_kernel(const float* __restrict__ g, const float* __restrict__ wo,
                                   const float* __restrict__ S, int B, int H, __nv_bfloat16* __restrict__ Dr,
                                   __nv_bfloat16* __restrict__ Dc, long long ldc, float* __restrict__ cs) {
  __shared__ float t[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = c0 + tx;
  for (int i = ty; i < 32; i += 8) {
    const long long r = r0 + i;
    float d = 0.f;
    if (r < B && c < H) {
      d = (g ? g[r] : 1.f) * wo[c] * S[r * H + c];
      Dr[r * H + c] = __float2bfloat16_rn(d);
    }
    t[i][tx] = d;
  }
  __syncthreads();
  if (cs && ty == 0 && c < H) {
    float sum = 0.f;
    for (int i = 0; i < 32; ++i)
      if (r0 + i < B) sum += t[i][tx];
    cs[(long long)blockIdx.x * H + c] = sum;
  }
  if (Dc) {
    for (int i = ty; i < 32; i += 8) {
      const int cc = c0 + i;
      const long long r = r0 + tx;
      if (cc < H && r < B) Dc[(long long)cc * ldc + r] = __float2bfloat16_rn(t[tx][i]);
    }
  }
}

// u = C^T G (the adjoint of the sin/cos chain rule) as BF16 images Ur (B x ldr)
// and Uc (d_in x ldc), with the arithmetic of dq_adjoint_kernel.
__global__ void adjoint_images_kernel(const float* __restrict__ q, const float* __restrict__ G, int B, int n,
                                      int d_in, __nv_bfloat16* __restrict__ Ur, long long ldr,
                                      __nv_bfloat16* __restrict__ Uc, long long ldc) {
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
    float u[3 + 2 + 2 * kMaxAngles];
    const float* gb = G + b * n;
    u[0] = u[1] = u[2] = 0.f;
    u[3] = gb[0];
    u[4] = gb[1];
    for (int a = 0; a < n - 2; ++a) {
      float sn, cs;
      sincosf(q[b * n + 2 + a], &sn, &cs);
      u[5 + 2 * a] = cs * gb[2 + a];
      u[6 + 2 * a] = -sn * gb[2 + a];
    }
    for (int k = 0; k < d_in; ++k) {
      const __nv_bfloat16 v = __float2bfloat16_rn(u[k]);
      Ur[b * ldr + k] = v;
      Uc[(long long)k * ldc + b] = v;
    }
  }
}

// One layer of the second-order sweep, element-wise on a 32 x 32 tile (block
// (32, 8)): E = r * a * s''(z) (a = A, or the broadcast row wo when A is NULL;
// E may alias A) and rs = r * s'(z) as BF16 images (row-major rsr, transposed
// rsc with row stride ldc; either may be NULL) and per-32-row column sums cs
// (NULL: none); the arithmetic of second_kernel and mul2_kernel.
__global__ void second_images_kernel(const float* __restrict__ R, const float* A, const float* __restrict__ wo,
                                     const float* __restrict__ S1, const float* __restrict__ S2, int B, int H,
                                     float* E, __nv_bfloat16* __restrict__ rsr, __nv_bfloat16* __restrict__ rsc,
                                     long long ldc, float* __restrict__ cs) {
  __shared__ float t[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = c0 + tx;
  for (int i = ty; i < 32; i += 8) {
    const long long r = r0 + i;
    float v = 0.f;
    if (r < B && c < H) {
      const long long e = r * H + c;
      const float rv = R[e];
      E[e] = rv * (A ? A[e] : wo[c]) * S2[e];
      v = rv * S1[e];
      if (rsr) rsr[e] = __float2bfloat16_rn(v);
    }
    t[i][tx] = v;
  }
  __syncthreads();
  if (cs && ty == 0 && c < H) {
    float sum = 0.f;
    for (int i = 0; i < 32; ++i)
      if (r0 + i < B) sum += t[i][tx];
    cs[(long long)blockIdx.x * H + c] = sum;
  }
  if (rsc) {
    for (int i = ty; i < 32; i += 8) {
      const int cc = c0 + i;
      const long long r = r0 + tx;
      if (cc < H && r < B) rsc[(long long)cc * ldc + r] = __float2bfloat16_rn(t[tx][i]);
    }
  }
}

// eps_L = E_L + g w_o * s'(z_L) as BF16 images (row-major Er, transposed Ec)
// and per-32-row column sums cs; the arithmetic of seed_add_kernel.
__global__ void eps_seed_images_kernel(const float* __restrict__ Ein, const float* __restrict__ g,
                                       const float* __restrict__ wo, const float* __restrict__ S, int B, int H,
                                       __nv_bfloat16* __restrict__ Er, __nv_bfloat16* __restrict__ Ec, long long ldc,
                                       float* __restrict__ cs) {
  __shared__ float t[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = c0 + tx;
  for (int i = ty; i < 32; i += 8) {
    const long long r = r0 + i;
    float v = 0.f;
    if (r < B && c < H) {
      const long long e = r * H + c;
      v = Ein[e] + g[r] * wo[c] * S[e];
      Er[e] = __float2bfloat16_rn(v);
    }
    t[i][tx] = v;
  }
  __syncthreads();
  if (ty == 0 && c < H) {
    float sum = 0.f;
    for (int i = 0; i < 32; ++i)
      if (r0 + i < B) sum += t[i][tx];
    cs[(long long)blockIdx.x * H + c] = sum;
  }
  for (int i = ty; i < 32; i += 8) {
    const int cc = c0 + i;
    const long long r = r0 + tx;
    if (cc < H && r < B) Ec[(long long)cc * ldc + r] = __float2bfloat16_rn(t[tx][i]);
  }
}

struct Bf16Fwd {
  __nv_bfloat16* Xr = nullptr;  // v, B x ldx
  __nv_bfloat16* Xc = nullptr;  // v^T, d_in x ldb (kept for dW_1)
  long long ldx = 0, ldb = 0;
  __nv_bfloat16* Hr[17] = {};   // h_l, B x H, l = 1 .. L-1
  __nv_bfloat16* Hc[17] = {};   // h_l^T, H x ldb (kept for dW_{l+1})
  __nv_bfloat16* Wr[17] = {};   // W_l, H x pad8(fan_in)
  __nv_bfloat16* Wt[17] = {};   // W_l^T, fan_in x H
};

// Buffers of the BF16 path.  keep_cols: the transposed images for the weight
// gradients; rev: the transposed weights for the back products.
cudaError_t alloc_bf16(Ws& ws, const Shape& sh, int B, bool keep_cols, bool rev, Bf16Fwd& bf) {
  cudaError_t e;
  bf.ldx = pad8(sh.d_in);
  bf.ldb = pad8(B);
  if ((e = ws.get(&bf.Xr, (size_t)B * bf.ldx))) return e;
  if (keep_cols && (e = ws.get(&bf.Xc, (size_t)sh.d_in * bf.ldb))) return e;
  for (int l = 1; l < sh.L; ++l) {
    if (l <= 2) {  // the row images are read by the next layer only: two alternate
      if ((e = ws.get(&bf.Hr[l], (size_t)B * sh.H))) return e;
    } else {
      bf.Hr[l] = bf.Hr[l - 2];
    }
    if (keep_cols && (e = ws.get(&bf.Hc[l], (size_t)sh.H * bf.ldb))) return e;
  }
  for (int l = 1; l <= sh.L; ++l) {
    if ((e = ws.get(&bf.Wr[l], (size_t)sh.H * pad8(sh.fan_in(l))))) return e;
    if (rev && (e = ws.get(&bf.Wt[l], (size_t)sh.fan_in(l) * sh.H))) return e;
  }
  return cudaSuccess;
}

// Forward pass on images: S_l = s'(z_l) (Ss[l-1], may be NULL), s''(z_l) (S2s,
// may be NULL), h_L in FP32 (HL), f (may be NULL).
int forward_bf16(const Shape& sh, const float* w, const float* q, const float* p, int B, Bf16Fwd& bf, float** Ss,
                 float* HL, float* f, Ctx& cx, float** S2s = nullptr) {
  const cudaStream_t s = cx.s;
  cudaError_t e;
  encode_bf16_kernel<<<grid1(B), 256, 0, s>>>(q, p, B, sh.n, sh.d_in, bf.Xr, bf.ldx, bf.Xc, bf.ldb);
  {
    long long offs[17];
    int fan[17];
    for (int l = 1; l <= sh.L; ++l) {
      offs[l] = (long long)sh.off(l);
      fan[l] = sh.fan_in(l);
    }
    if ((e = weight_images(w, offs, fan, sh.L, sh.H, bf.Wr, bf.Wt, s)))
      return set_error(GCDF_ECUDA, "weight images: %s", cudaGetErrorString(e));
  }
  for (int l = 1; l <= sh.L; ++l) {
    const int K = sh.fan_in(l);
    const float* W = w + sh.off(l);
    GemmEpilogue ep{};
    ep.mode = kEpiBiasSilu;
    ep.bias = W + (size_t)sh.H * K;
    ep.s_out = Ss ? Ss[l - 1] : nullptr;
    ep.s2_out = S2s ? S2s[l - 1] : nullptr;
    ep.ld_s = sh.H;
    if (l < sh.L) {
      ep.img = bf.Hr[l];
      ep.ld_img = sh.H;
      ep.imgT = bf.Hc[l];
      ep.ld_imgT = bf.ldb;
    }
    const __nv_bfloat16* A = l == 1 ? bf.Xr : bf.Hr[l - 1];
    const long long lda = l == 1 ? bf.ldx : sh.H;
    if ((e = cx.mm_images(A, lda, bf.Wr[l], pad8(K), B, sh.H, K, l == sh.L ? HL : nullptr, sh.H, false, false, &ep)))
      return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
  }
  if (f)
    rowdot_kernel<<<(int)(((long long)B * 32 + 255) / 256), 256, 0, s>>>(HL, B, sh.H, w + sh.off_out,
                                                                      w + sh.off_out + sh.H, f);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit forward launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

// Reverse sweep on images from delta_L = g w_o * s'(z_L) (g NULL: 1): for l = L .. 1,
//   with_grads: dW_l = delta_l^T h_{l-1} (transposed images) and db_l (the
//   per-32-row column sums of delta_l, summed over the row blocks in order);
//   delta_{l-1} = (delta_l W_l) * s'(z_{l-1}) through the back product's epilogue;
//   at l = 1 (dv not NULL): dv = delta_1 W_1 (FP32).
int reverse_bf16(const Shape& sh, int B, Bf16Fwd& bf, float** Ss, const float* g, const float* wo, bool with_grads,
                 float* dweights, float* dv, Ws& ws, Ctx& cx) {
  const cudaStream_t s = cx.s;
  const int H = sh.H;
  cudaError_t e;
  __nv_bfloat16 *Dr[2] = {}, *Dc[2] = {};
  float* cs = nullptr;
  const long long nblk = (B + 31) / 32;
  for (int k = 0; k < 2; ++k)
    if ((e = ws.get(&Dr[k], (size_t)B * H)) || (with_grads && (e = ws.get(&Dc[k], (size_t)H * bf.ldb))))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  if (with_grads && (e = ws.get(&cs, (size_t)nblk * H))) return set_error(GCDF_ENOMEM, "cudaMallocAsync");
  // delta_L straight into its images and column sums
  {
    dim3 grid((unsigned)nblk, (unsigned)((H + 127) / 128));
    seed_images_wide_kernel<<<grid, dim3(32, 8), 0, s>>>(g, wo, Ss[sh.L - 1], B, H, Dr[0],
                                                         with_grads ? Dc[0] : nullptr, bf.ldb,
                                                         with_grads ? cs : nullptr);
  }
  int cur = 0;
  for (int l = sh.L; l >= 1; --l) {
    const int K = sh.fan_in(l);
    if (with_grads) {
      // dW_l (H x K) = delta_l^T (H x B) . h_{l-1} (B x K): both transposed images
      const __nv_bfloat16* Bop = l == 1 ? bf.Xc : bf.Hc[l - 1];
      if ((e = cx.mm_images(Dc[cur], bf.ldb, Bop, bf.ldb, H, K, B, dweights + sh.off(l), K, true, false, nullptr)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
      // db_l: the column sums left by the seed (l = L) or by the back product of layer l + 1
      if ((e = colsum(cs, (int)nblk, H, nullptr, dweights + sh.off(l) + (size_t)H * K, cx.partials, cx.pfl, s)))
        return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
    }
    if (l > 1) {
      GemmEpilogue ep{};
      ep.mode = kEpiMul;
      ep.s_in = Ss[l - 2];
      ep.ld_s = H;
      ep.img = Dr[cur ^ 1];
      ep.ld_img = H;
      if (with_grads) {
        ep.imgT = Dc[cur ^ 1];
        ep.ld_imgT = bf.ldb;
        ep.colsum = cs;
        ep.ld_colsum = H;
      }
      // delta_{l-1} (B x K) = (delta_l (B x H) W_l (H x K)) * s'(z_{l-1}); B operand W_l^T (K x H)
      if ((e = cx.mm_images(Dr[cur], H, bf.Wt[l], H, B, K, H, nullptr, K, false, false, &ep)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
      cur ^= 1;
    } else if (dv) {
      if ((e = cx.mm_images(Dr[cur], H, bf.Wt[1], H, B, sh.d_in, H, dv, sh.d_in, false, false, nullptr)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit backward launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

// Second-order weight VJP (gcdf_fit_vjp2) on images: the generic scheme's
// arithmetic and rounding points, with every product operand written as BF16
// images by its producer (forward and back-product epilogues, the element-wise
// kernels above) and the bias gradients summed per 32-row block.
int vjp2_bf16(const Shape& sh, const float* w, const float* q, const float* p, int B, const float* g_f,
              const float* G_q, float* dweights, Ws& ws, cudaStream_t s) {
  const int H = sh.H, L = sh.L;
  const long long n = (long long)B * H;
  const long long nblk = (B + 31) / 32;
  const size_t pfl = (size_t)64 * H * (H > sh.d_in ? H : sh.d_in);
  cudaError_t e;
  int rc;
  Bf16Fwd bf;
  float *S1[17], *S2[17], *AE[17];
  float *HL = nullptr, *R = nullptr, *cs = nullptr, *partials = nullptr;
  __nv_bfloat16 *Dr[2] = {}, *Dc[17] = {}, *Ur = nullptr, *Uc = nullptr, *rsr = nullptr, *rsc = nullptr;
  __nv_bfloat16 *Er[2] = {}, *Ec = nullptr;
  for (int l = 1; l <= L; ++l)
    if ((e = ws.get(&S1[l - 1], (size_t)n)) || (e = ws.get(&S2[l - 1], (size_t)n)) || (e = ws.get(&AE[l - 1], (size_t)n)) ||
        (e = ws.get(&Dc[l - 1], (size_t)H * pad8(B))))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  if ((e = alloc_bf16(ws, sh, B, true, true, bf)) || (e = ws.get(&HL, (size_t)n)) || (e = ws.get(&R, (size_t)n)) ||
      (e = ws.get(&cs, (size_t)nblk * H)) || (e = ws.get(&partials, pfl)) || (e = ws.get(&Dr[0], (size_t)n)) ||
      (e = ws.get(&Dr[1], (size_t)n)) || (e = ws.get(&Ur, (size_t)B * bf.ldx)) ||
      (e = ws.get(&Uc, (size_t)sh.d_in * bf.ldb)) || (e = ws.get(&rsr, (size_t)n)) ||
      (e = ws.get(&rsc, (size_t)H * bf.ldb)) || (e = ws.get(&Er[0], (size_t)n)) || (e = ws.get(&Er[1], (size_t)n)) ||
      (e = ws.get(&Ec, (size_t)H * bf.ldb)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  Ctx cx;
  if ((rc = make_ctx_images(cx, s, partials, pfl))) return rc;
  if ((rc = forward_bf16(sh, w, q, p, B, bf, S1, HL, nullptr, cx, S2))) return rc;
  const float* wo = w + sh.off_out;
  float* dwo = dweights + sh.off_out;
  const dim3 tgrid((unsigned)nblk, (unsigned)((H + 31) / 32)), tblk(32, 8);
  // the field's reverse sweep: delta_L = w_o s'(z_L); a_{l-1} = delta_l W_l (FP32,
  // AE[l-2]), delta_{l-1} = a_{l-1} s'(z_{l-1}); transposed images of every delta
  seed_images_kernel<<<tgrid, tblk, 0, s>>>(nullptr, wo, S1[L - 1], B, H, Dr[0], Dc[L - 1], bf.ldb, nullptr);
  int cur = 0;
  for (int l = L; l >= 2; --l) {
    GemmEpilogue ep{};
    ep.mode = kEpiMul;
    ep.s_in = S1[l - 2];
    ep.acc_out = AE[l - 2];
    ep.ld_s = H;
    ep.img = Dr[cur ^ 1];
    ep.ld_img = H;
    ep.imgT = Dc[l - 2];
    ep.ld_imgT = bf.ldb;
    if ((e = cx.mm_images(Dr[cur], H, bf.Wt[l], H, B, H, H, nullptr, H, false, false, &ep)))
      return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    cur ^= 1;
  }
  // first-derivative terms: u = C^T G; dW_1 = delta_1^T u; r_1 = u W_1^T
  adjoint_images_kernel<<<grid1(B), 256, 0, s>>>(q, G_q, B, sh.n, sh.d_in, Ur, bf.ldx, Uc, bf.ldb);
  if ((e = cx.mm_images(Dc[0], bf.ldb, Uc, bf.ldb, H, sh.d_in, B, dweights, sh.d_in, true, false, nullptr)) ||
      (e = cx.mm_images(Ur, bf.ldx, bf.Wr[1], bf.ldx, B, H, sh.d_in, R, H, false, false, nullptr)))
    return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
  for (int l = 1; l <= L; ++l) {
    // e_l = r a_l s''(z_l) in place of a_l; rs = r s'(z_l)
    second_images_kernel<<<tgrid, tblk, 0, s>>>(R, l < L ? AE[l - 1] : nullptr, wo, S1[l - 1], S2[l - 1], B, H,
                                                AE[l - 1], l < L ? rsr : nullptr, l < L ? rsc : nullptr, bf.ldb,
                                                l < L ? nullptr : cs);
    if (l < L) {
      // dW_{l+1} = delta_{l+1}^T rs;  r_{l+1} = rs W_{l+1}^T
      if ((e = cx.mm_images(Dc[l], bf.ldb, rsc, bf.ldb, H, H, B, dweights + sh.off(l + 1), H, true, false, nullptr)) ||
          (e = cx.mm_images(rsr, H, bf.Wr[l + 1], H, B, H, H, R, H, false, false, nullptr)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    } else if ((e = colsum(cs, (int)nblk, H, nullptr, dwo, partials, pfl, s))) {  // dw_o = sum_b r_L s'(z_L)
      return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
    }
  }
  // value and second-derivative terms (accumulated; biases written)
  if ((e = colsum(HL, B, H, g_f, dwo, partials, pfl, s, true)) || (e = colsum(g_f, B, 1, nullptr, dwo + H, partials, pfl, s)))
    return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
  eps_seed_images_kernel<<<tgrid, tblk, 0, s>>>(AE[L - 1], g_f, wo, S1[L - 1], B, H, Er[0], Ec, bf.ldb, cs);
  cur = 0;
  for (int l = L; l >= 1; --l) {
    const int K = sh.fan_in(l);
    const __nv_bfloat16* Bop = l == 1 ? bf.Xc : bf.Hc[l - 1];
    if ((e = cx.mm_images(Ec, bf.ldb, Bop, bf.ldb, H, K, B, dweights + sh.off(l), K, true, true, nullptr)) ||
        (e = colsum(cs, (int)nblk, H, nullptr, dweights + sh.off(l) + (size_t)H * K, partials, pfl, s)))
      return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    if (l > 1) {
      // eps_{l-1} = e_{l-1} + (eps_l W_l) s'(z_{l-1})
      GemmEpilogue ep{};
      ep.mode = kEpiMul;
      ep.s_in = S1[l - 2];
      ep.add_in = AE[l - 2];
      ep.ld_s = H;
      ep.img = Er[cur ^ 1];
      ep.ld_img = H;
      ep.imgT = Ec;
      ep.ld_imgT = bf.ldb;
      ep.colsum = cs;
      ep.ld_colsum = H;
      if ((e = cx.mm_images(Er[cur], H, bf.Wt[l], H, B, H, H, nullptr, H, false, false, &ep)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
      cur ^= 1;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit vjp2 launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

}  // namespace
}  // namespace gcdf

using namespace gcdf;


// The tape of a BF16 forward pass: what the reverse sweep of gcdf_fit_vjp reads
// (the transposed image of v and of h_1 .. h_{L-1}, s'(z_1) .. s'(z_L) and
// h_L in FP32), each part 256-byte aligned.
struct TapeLayout {
  size_t xc, hc, ss, hl, total;
};
size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }
TapeLayout tape_layout(const Shape& sh, int B) {
  TapeLayout t{};
  const size_t ldb = (size_t)pad8(B);
  t.xc = up256((size_t)sh.d_in * ldb * sizeof(__nv_bfloat16));
  t.hc = up256((size_t)sh.H * ldb * sizeof(__nv_bfloat16));
  t.ss = up256((size_t)B * sh.H * sizeof(float));
  t.hl = t.ss;
  t.total = t.xc + (size_t)(sh.L - 1) * t.hc + (size_t)sh.L * t.ss + t.hl;
  return t;
}
// Point the tape-held buffers of a BF16 pass into `tape`.
void tape_carve(const Shape& sh, int B, void* tape, Bf16Fwd& bf, float** Ss, float** HL) {
  const TapeLayout t = tape_layout(sh, B);
  unsigned char* c = static_cast<unsigned char*>(tape);
  bf.Xc = reinterpret_cast<__nv_bfloat16*>(c);
  c += t.xc;
  for (int l = 1; l < sh.L; ++l) {
    bf.Hc[l] = reinterpret_cast<__nv_bfloat16*>(c);
    c += t.hc;
  }
  for (int l = 1; l <= sh.L; ++l) {
    Ss[l - 1] = reinterpret_cast<float*>(c);
    c += t.ss;
  }
  *HL = reinterpret_cast<float*>(c);
}
// Buffers of a BF16 pass that are not on the tape: the row images (v, h_l)
// and the weight images (fwd: W_l for the layer products; rev: W_l^T for the
// back products).
cudaError_t alloc_bf16_work(Ws& ws, const Shape& sh, int B, bool fwd, bool rev, Bf16Fwd& bf) {
  cudaError_t e;
  bf.ldx = pad8(sh.d_in);
  bf.ldb = pad8(B);
  if (fwd) {
    if ((e = ws.get(&bf.Xr, (size_t)B * bf.ldx))) return e;
    for (int l = 1; l < sh.L; ++l) {
      if (l <= 2) {
        if ((e = ws.get(&bf.Hr[l], (size_t)B * sh.H))) return e;
      } else {
        bf.Hr[l] = bf.Hr[l - 2];
      }
    }
  }
  for (int l = 1; l <= sh.L; ++l) {
    if (fwd && (e = ws.get(&bf.Wr[l], (size_t)sh.H * pad8(sh.fan_in(l))))) return e;
    if (rev && (e = ws.get(&bf.Wt[l], (size_t)sh.fan_in(l) * sh.H))) return e;
  }
  return cudaSuccess;
}

extern "C" {

int gcdf_fit_device_status(int* status) {
  if (!status) return set_error(GCDF_EINVAL, "status is NULL");
  int* w = fit_status_word();
  if (!w) return set_error(GCDF_ECUDA, "fit status word unavailable");
  cudaError_t e;
  int v = 0;
  if ((e = cudaDeviceSynchronize()) || (e = cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost)) ||
      (e = cudaMemset(w, 0, sizeof(int))))
    return set_error(GCDF_ECUDA, "fit status: %s", cudaGetErrorString(e));
  *status = v;
  clear_error();
  return GCDF_OK;
}

int gcdf_fit_forward(const gcdf_fit_desc* desc, const float* weights, const float* q, const float* p, int batch,
                     float* f, gcdf_stream_t stream) {
  Shape sh;
  int rc = check(desc, weights, q, p, batch, sh);
  if (rc) return rc;
  if (batch == 0) { clear_error(); return GCDF_OK; }
  if (!f || !al16(f)) return set_error(GCDF_EINVAL, "f NULL or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Ws ws(s);
  float* Hs[18];
  float* Ss[17];
  cudaError_t e;
  if (sh.bf16) {
    Bf16Fwd bf;
    float* HL = nullptr;
    Ctx cx;
    if ((e = alloc_bf16(ws, sh, batch, false, false, bf)) || (e = ws.get(&HL, (size_t)batch * sh.H)))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
    if ((rc = make_ctx_images(cx, s, nullptr, 0))) return rc;
    if ((rc = forward_bf16(sh, weights, q, p, batch, bf, nullptr, HL, f, cx))) return rc;
    clear_error();
    return GCDF_OK;
  }
  if ((e = ws.get(&Hs[0], (size_t)batch * sh.d_in))) return set_error(GCDF_ENOMEM, "cudaMallocAsync");
  // two alternating activation buffers suffice without a backward pass
  float *h0, *h1, *sc;
  if ((e = ws.get(&h0, (size_t)batch * sh.H)) || (e = ws.get(&h1, (size_t)batch * sh.H)) ||
      (e = ws.get(&sc, (size_t)batch * sh.H)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  for (int l = 1; l <= sh.L; ++l) {
    Hs[l] = (l & 1) ? h0 : h1;
    Ss[l - 1] = sc;
  }
  Ctx cx;
  if ((rc = make_ctx(cx, ws, sh, batch, s, nullptr, 0))) return rc;
  rc = forward(sh, weights, q, p, batch, Hs, Ss, f, cx);
  if (rc) return rc;
  clear_error();
  return GCDF_OK;
}

int gcdf_fit_vjp(const gcdf_fit_desc* desc, const float* weights, const float* q, const float* p, int batch,
                 const float* g_f, float* dweights, float* dq, gcdf_stream_t stream) {
  Shape sh;
  int rc = check(desc, weights, q, p, batch, sh);
  if (rc) return rc;
  if (!dweights || !al16(dweights)) return set_error(GCDF_EINVAL, "dweights NULL or not 16-byte aligned");
  if (dq && !al16(dq)) return set_error(GCDF_EINVAL, "dq not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (batch == 0) {
    if ((e = cudaMemsetAsync(dweights, 0, sh.total * sizeof(float), s)))
      return set_error(GCDF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    clear_error();
    return GCDF_OK;
  }
  if (!g_f || !al16(g_f)) return set_error(GCDF_EINVAL, "g_f NULL or not 16-byte aligned");
  Ws ws(s);
  float* Hs[18];
  float* Ss[17];
  float *D0, *D1, *partials;
  const size_t pfl = (size_t)64 * sh.H * (sh.H > sh.d_in ? sh.H : sh.d_in);
  if (sh.bf16) {
    const int H = sh.H;
    Bf16Fwd bf;
    float *HL = nullptr, *dv = nullptr;
    Ctx cx;
    for (int l = 1; l <= sh.L; ++l)
      if ((e = ws.get(&Ss[l - 1], (size_t)batch * H))) return set_error(GCDF_ENOMEM, "cudaMallocAsync");
    if ((e = alloc_bf16(ws, sh, batch, true, true, bf)) || (e = ws.get(&HL, (size_t)batch * H)) ||
        (e = ws.get(&partials, pfl)) ||
        (dq && (e = ws.get(&dv, (size_t)batch * sh.d_in))))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
    if ((rc = make_ctx_images(cx, s, partials, pfl))) return rc;
    if ((rc = forward_bf16(sh, weights, q, p, batch, bf, Ss, HL, nullptr, cx))) return rc;
    float* dwo = dweights + sh.off_out;
    if ((e = colsum(HL, batch, H, g_f, dwo, partials, pfl, s)) || (e = colsum(g_f, batch, 1, nullptr, dwo + H, partials, pfl, s)))
      return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
    if ((rc = reverse_bf16(sh, batch, bf, Ss, g_f, weights + sh.off_out, true, dweights, dv, ws, cx))) return rc;
    if (dq) dq_kernel<<<grid1(batch), 256, 0, s>>>(q, dv, batch, sh.n, sh.d_in, dq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit backward launch: %s", cudaGetErrorString(e));
    clear_error();
    return GCDF_OK;
  }
  if ((e = ws.get(&Hs[0], (size_t)batch * sh.d_in))) return set_error(GCDF_ENOMEM, "cudaMallocAsync");
  for (int l = 1; l <= sh.L; ++l)
    if ((e = ws.get(&Hs[l], (size_t)batch * sh.H)) || (e = ws.get(&Ss[l - 1], (size_t)batch * sh.H)))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  const size_t dcols = (size_t)(sh.H > sh.d_in ? sh.H : sh.d_in);
  if ((e = ws.get(&D0, (size_t)batch * dcols)) || (e = ws.get(&D1, (size_t)batch * dcols)) ||

      (e = ws.get(&partials, pfl)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  Ctx cx;
  if ((rc = make_ctx(cx, ws, sh, batch, s, partials, pfl))) return rc;
  rc = forward(sh, weights, q, p, batch, Hs, Ss, nullptr, cx);
  if (rc) return rc;

  const int H = sh.H;
  float* dwo = dweights + sh.off_out;
  // dw_o (H) = H_L^T g;  db_o = g^T 1
  if ((e = colsum(Hs[sh.L], batch, H, g_f, dwo, partials, pfl, s)) ||
      (e = colsum(g_f, batch, 1, nullptr, dwo + H, partials, pfl, s)))
    return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
  // delta_L = g w_o * s'(z_L)
  float* D = D1;
  seed_kernel<<<grid1((long long)batch * H), 256, 0, s>>>(g_f, weights + sh.off_out, Ss[sh.L - 1], batch, H, D);
  for (int l = sh.L; l >= 1; --l) {
    const int K = sh.fan_in(l);
    const float* W = weights + sh.off(l);
    float* dW = dweights + sh.off(l);
    // dW_l (H x K) = delta^T (H x B) H_{l-1} (B x K);  db_l = delta^T 1
    if ((e = cx.mm(D, 1, H, Hs[l - 1], K, 1, dW, K, H, K, batch, true)) ||
        (e = colsum(D, batch, H, nullptr, dW + (size_t)H * K, partials, pfl, s)))
      return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    if (l > 1 || dq) {
      // back (B x K) = delta (B x H) W_l (H x K)
      float* back = (D == D1) ? D0 : D1;  // never the buffer it reads
      if ((e = cx.mm(D, H, 1, W, K, 1, back, K, batch, K, H, false)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
      if (l > 1) {
        mul_kernel<<<grid1((long long)batch * K), 256, 0, s>>>(back, Ss[l - 2], (long long)batch * K);
        D = back;
      } else {
        dq_kernel<<<grid1(batch), 256, 0, s>>>(q, back, batch, sh.n, sh.d_in, dq);
      }
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit backward launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}

int gcdf_fit_value_grad(const gcdf_fit_desc* desc, const float* weights, const float* q, const float* p, int batch,
                        float* f, float* dq, gcdf_stream_t stream) {
  Shape sh;
  int rc = check(desc, weights, q, p, batch, sh);
  if (rc) return rc;
  if (batch == 0) { clear_error(); return GCDF_OK; }
  if (!f || !al16(f) || !dq || !al16(dq)) return set_error(GCDF_EINVAL, "f or dq NULL or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Ws ws(s);
  float* Hs[18];
  float* Ss[17];
  float* D[17];
  float *d0, *d1, *dv;
  cudaError_t e;
  if (sh.bf16) {
    Bf16Fwd bf;
    float* HL = nullptr;
    Ctx cx;
    for (int l = 1; l <= sh.L; ++l)
      if ((e = ws.get(&Ss[l - 1], (size_t)batch * sh.H))) return set_error(GCDF_ENOMEM, "cudaMallocAsync");
    if ((e = alloc_bf16(ws, sh, batch, false, true, bf)) || (e = ws.get(&HL, (size_t)batch * sh.H)) ||
        (e = ws.get(&dv, (size_t)batch * sh.d_in)))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
    if ((rc = make_ctx_images(cx, s, nullptr, 0))) return rc;
    if ((rc = forward_bf16(sh, weights, q, p, batch, bf, Ss, HL, f, cx))) return rc;
    if ((rc = reverse_bf16(sh, batch, bf, Ss, nullptr, weights + sh.off_out, false, nullptr, dv, ws, cx))) return rc;
    dq_kernel<<<grid1(batch), 256, 0, s>>>(q, dv, batch, sh.n, sh.d_in, dq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit value/grad launch: %s", cudaGetErrorString(e));
    clear_error();
    return GCDF_OK;
  }
  if ((e = ws.get(&Hs[0], (size_t)batch * sh.d_in)) || (e = ws.get(&dv, (size_t)batch * sh.d_in)) ||
      (e = ws.get(&d0, (size_t)batch * sh.H)) || (e = ws.get(&d1, (size_t)batch * sh.H)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  for (int l = 1; l <= sh.L; ++l)
    if ((e = ws.get(&Hs[l], (size_t)batch * sh.H)) || (e = ws.get(&Ss[l - 1], (size_t)batch * sh.H)))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  Ctx cx;
  if ((rc = make_ctx(cx, ws, sh, batch, s, nullptr, 0))) return rc;
  rc = forward(sh, weights, q, p, batch, Hs, Ss, f, cx);
  if (rc) return rc;
  // delta ping-pongs between two buffers, a_{l-1} computed in place of delta_{l-1}
  for (int l = 1; l <= sh.L; ++l) D[l - 1] = ((sh.L - l) & 1) ? d1 : d0;
  if ((rc = reverse_sweep(sh, weights, batch, Ss, D, D, cx))) return rc;
  // dv (B x d_in) = delta_1 W_1
  if ((e = cx.mm(D[0], sh.H, 1, weights, sh.d_in, 1, dv, sh.d_in, batch, sh.d_in, sh.H, false)))
    return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
  dq_kernel<<<grid1(batch), 256, 0, s>>>(q, dv, batch, sh.n, sh.d_in, dq);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit value/grad launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}

int gcdf_fit_vjp2(const gcdf_fit_desc* desc, const float* weights, const float* q, const float* p, int batch,
                  const float* g_f, const float* G_q, float* dweights, gcdf_stream_t stream) {
  Shape sh;
  int rc = check(desc, weights, q, p, batch, sh);
  if (rc) return rc;
  if (!dweights || !al16(dweights)) return set_error(GCDF_EINVAL, "dweights NULL or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (batch == 0) {
    if ((e = cudaMemsetAsync(dweights, 0, sh.total * sizeof(float), s)))
      return set_error(GCDF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    clear_error();
    return GCDF_OK;
  }
  if (!g_f || !al16(g_f) || !G_q || !al16(G_q))
    return set_error(GCDF_EINVAL, "g_f or G_q NULL or not 16-byte aligned");
  if (sh.bf16) {
    Ws ws(s);
    if ((rc = vjp2_bf16(sh, weights, q, p, batch, g_f, G_q, dweights, ws, s))) return rc;
    clear_error();
    return GCDF_OK;
  }
  const int H = sh.H, L = sh.L;
  const long long n = (long long)batch * H;
  Ws ws(s);
  float *Hs[18], *S1[17], *S2[17], *D[17], *AE[17];
  float *U, *R0, *R1, *partials;
  const size_t pfl = (size_t)64 * H * (H > sh.d_in ? H : sh.d_in);
  if ((e = ws.get(&Hs[0], (size_t)batch * sh.d_in)) || (e = ws.get(&U, (size_t)batch * sh.d_in)) ||
      (e = ws.get(&R0, (size_t)n)) || (e = ws.get(&R1, (size_t)n)) || (e = ws.get(&partials, pfl)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  for (int l = 1; l <= L; ++l)
    if ((e = ws.get(&Hs[l], (size_t)n)) || (e = ws.get(&S1[l - 1], (size_t)n)) || (e = ws.get(&S2[l - 1], (size_t)n)) ||
        (e = ws.get(&D[l - 1], (size_t)n)) || (e = ws.get(&AE[l - 1], (size_t)n)))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  Ctx cx;
  if ((rc = make_ctx(cx, ws, sh, batch, s, partials, pfl))) return rc;
  if ((rc = forward(sh, weights, q, p, batch, Hs, S1, nullptr, cx, S2))) return rc;
  // a_l (l < L) into AE[l - 1]; a_L = w_o is never stored
  if ((rc = reverse_sweep(sh, weights, batch, S1, D, AE, cx))) return rc;
  const float* wo = weights + sh.off_out;
  float* dwo = dweights + sh.off_out;
  // first-derivative terms (written): u = C^T G; dW_1 = delta_1^T u; r_1 = u W_1^T
  dq_adjoint_kernel<<<grid1(batch), 256, 0, s>>>(q, G_q, batch, sh.n, sh.d_in, U);
  if ((e = cx.mm(D[0], 1, H, U, sh.d_in, 1, dweights, sh.d_in, H, sh.d_in, batch, true)) ||
      (e = cx.mm(U, sh.d_in, 1, weights, 1, sh.d_in, R0, H, batch, H, sh.d_in, false)))
    return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
  float *r = R0, *rs = R1;
  for (int l = 1; l <= L; ++l) {
    // e_l = r_l * a_l * s''(z_l), in place of a_l
    second_kernel<<<grid1(n), 256, 0, s>>>(r, l < L ? AE[l - 1] : nullptr, wo, S2[l - 1], batch, H, AE[l - 1]);
    mul2_kernel<<<grid1(n), 256, 0, s>>>(rs, r, S1[l - 1], n);
    if (l < L) {
      // dW_{l+1} = delta_{l+1}^T rs;  r_{l+1} = rs W_{l+1}^T
      const float* W = weights + sh.off(l + 1);
      if ((e = cx.mm(D[l], 1, H, rs, H, 1, dweights + sh.off(l + 1), H, H, H, batch, true)) ||
          (e = cx.mm(rs, H, 1, W, 1, H, r, H, batch, H, H, false)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    } else if ((e = colsum(rs, batch, H, nullptr, dwo, partials, pfl, s))) {  // dw_o = sum_b r_L * s'(z_L)
      return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
    }
  }
  // value and second-derivative terms (accumulated; biases written)
  if ((e = colsum(Hs[L], batch, H, g_f, dwo, partials, pfl, s, true)) ||
      (e = colsum(g_f, batch, 1, nullptr, dwo + H, partials, pfl, s)))
    return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
  float* eps = AE[L - 1];
  seed_add_kernel<<<grid1(n), 256, 0, s>>>(g_f, wo, S1[L - 1], batch, H, eps);
  for (int l = L; l >= 1; --l) {
    const int K = sh.fan_in(l);
    float* dW = dweights + sh.off(l);
    if ((e = cx.mm(eps, 1, H, Hs[l - 1], K, 1, dW, K, H, K, batch, true, true)) ||
        (e = colsum(eps, batch, H, nullptr, dW + (size_t)H * K, partials, pfl, s)))
      return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    if (l > 1) {
      // eps_{l-1} = e_{l-1} + (eps_l W_l) * s'(z_{l-1})
      float* back = (eps == R0) ? R1 : R0;
      if ((e = cx.mm(eps, H, 1, weights + sh.off(l), H, 1, back, H, batch, H, H, false)))
        return set_error(GCDF_ECUDA, "gemm: %s", cudaGetErrorString(e));
      addmul_kernel<<<grid1(n), 256, 0, s>>>(back, S1[l - 2], AE[l - 2], n);
      eps = back;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit vjp2 launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}


int gcdf_fit_tape_bytes(const gcdf_fit_desc* desc, int batch, size_t* bytes) {
  Shape sh;
  if (!bytes) return set_error(GCDF_EINVAL, "bytes is NULL");
  // shape checks only (no data pointer is read)
  alignas(16) static const float none[4] = {0.f, 0.f, 0.f, 0.f};
  int rc = check(desc, none, none, none, batch, sh);
  if (rc) return rc;
  if (!sh.bf16) return set_error(GCDF_EINVAL, "the tape is kept by the BF16 path only");
  *bytes = batch > 0 ? tape_layout(sh, batch).total : 0;
  clear_error();
  return GCDF_OK;
}

int gcdf_fit_forward_tape(const gcdf_fit_desc* desc, const float* weights, const float* q, const float* p, int batch,
                          float* f, void* tape, size_t tape_bytes, gcdf_stream_t stream) {
  Shape sh;
  int rc = check(desc, weights, q, p, batch, sh);
  if (rc) return rc;
  if (!sh.bf16) return set_error(GCDF_EINVAL, "the tape is kept by the BF16 path only");
  if (batch == 0) { clear_error(); return GCDF_OK; }
  if (!f || !al16(f)) return set_error(GCDF_EINVAL, "f NULL or not 16-byte aligned");
  if (!tape || (reinterpret_cast<uintptr_t>(tape) & 255) != 0)
    return set_error(GCDF_EINVAL, "tape NULL or not 256-byte aligned");
  if (tape_bytes < tape_layout(sh, batch).total)
    return set_error(GCDF_EINVAL, "tape of %zu bytes, %zu needed", tape_bytes, tape_layout(sh, batch).total);
  cudaStream_t s = (cudaStream_t)stream;
  Ws ws(s);
  Bf16Fwd bf;
  float* Ss[17];
  float* HL = nullptr;
  Ctx cx;
  cudaError_t e;
  tape_carve(sh, batch, tape, bf, Ss, &HL);
  if ((e = alloc_bf16_work(ws, sh, batch, true, false, bf)))
    return set_error(GCDF_ENOMEM, "temporaries: %s", cudaGetErrorString(e));
  if ((rc = make_ctx_images(cx, s, nullptr, 0))) return rc;
  if ((rc = forward_bf16(sh, weights, q, p, batch, bf, Ss, HL, f, cx))) return rc;
  clear_error();
  return GCDF_OK;
}

int gcdf_fit_vjp_tape(const gcdf_fit_desc* desc, const float* weights, const float* q, const float* p, int batch,
                      const float* g_f, const void* tape, size_t tape_bytes, float* dweights, float* dq,
                      gcdf_stream_t stream) {
  Shape sh;
  int rc = check(desc, weights, q, p, batch, sh);
  if (rc) return rc;
  if (!sh.bf16) return set_error(GCDF_EINVAL, "the tape is kept by the BF16 path only");
  if (!dweights || !al16(dweights)) return set_error(GCDF_EINVAL, "dweights NULL or not 16-byte aligned");
  if (dq && !al16(dq)) return set_error(GCDF_EINVAL, "dq not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (batch == 0) {
    if ((e = cudaMemsetAsync(dweights, 0, sh.total * sizeof(float), s)))
      return set_error(GCDF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    clear_error();
    return GCDF_OK;
  }
  if (!g_f || !al16(g_f)) return set_error(GCDF_EINVAL, "g_f NULL or not 16-byte aligned");
  if (!tape || (reinterpret_cast<uintptr_t>(tape) & 255) != 0)
    return set_error(GCDF_EINVAL, "tape NULL or not 256-byte aligned");
  if (tape_bytes < tape_layout(sh, batch).total)
    return set_error(GCDF_EINVAL, "tape of %zu bytes, %zu needed", tape_bytes, tape_layout(sh, batch).total);
  Ws ws(s);
  Bf16Fwd bf;
  float* Ss[17];
  float *HL = nullptr, *dv = nullptr, *partials = nullptr;
  const size_t pfl = (size_t)64 * sh.H * (sh.H > sh.d_in ? sh.H : sh.d_in);
  Ctx cx;
  tape_carve(sh, batch, const_cast<void*>(tape), bf, Ss, &HL);
  if ((e = alloc_bf16_work(ws, sh, batch, false, true, bf)) || (e = ws.get(&partials, pfl)) ||
      (dq && (e = ws.get(&dv, (size_t)batch * sh.d_in))))
    return set_error(GCDF_ENOMEM, "temporaries: %s", cudaGetErrorString(e));
  if ((rc = make_ctx_images(cx, s, partials, pfl))) return rc;
  // the transposed weight images of the back products (the tape holds the
  // activations, not the weights)
  {
    long long offs[17];
    int fan[17];
    for (int l = 1; l <= sh.L; ++l) {
      offs[l] = (long long)sh.off(l);
      fan[l] = sh.fan_in(l);
    }
    if ((e = weight_images(weights, offs, fan, sh.L, sh.H, nullptr, bf.Wt, s)))
      return set_error(GCDF_ECUDA, "weight images: %s", cudaGetErrorString(e));
  }
  float* dwo = dweights + sh.off_out;
  if ((e = colsum(HL, batch, sh.H, g_f, dwo, partials, pfl, s)) ||
      (e = colsum(g_f, batch, 1, nullptr, dwo + sh.H, partials, pfl, s)))
    return set_error(GCDF_ECUDA, "colsum: %s", cudaGetErrorString(e));
  if ((rc = reverse_bf16(sh, batch, bf, Ss, g_f, weights + sh.off_out, true, dweights, dv, ws, cx))) return rc;
  if (dq) dq_kernel<<<grid1(batch), 256, 0, s>>>(q, dv, batch, sh.n, sh.d_in, dq);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "fit backward launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}

}  // extern "C"
