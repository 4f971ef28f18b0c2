// BF16 tensor-core GEMM of the differentiable fit (Sec. III-C): every matrix
// product of a training step — the layer products, the back-products and the
// batch-length weight-gradient reductions — with BF16 operands and FP32
// accumulation on tcgen05.
//
//   C_z[m, n] = sum over the K-blocks of split z of A[m, k] B[n, k]
//
// A (M x K) and B (N x K) are row-major BF16 images (K contiguous, any row
// stride that is a multiple of 8 elements), loaded by TMA in 128-byte swizzled
// slabs of 64 K values; rows and K positions past the matrix come in as zeros.
// A CTA pair (cluster of 2) computes one 256 x 128 tile of C with
// tcgen05.mma.cta_group::2 (M = 256, N = 128, K = 16 per instruction): each
// CTA holds 128 rows of A and 64 rows of B per stage and its own 128 x 128
// FP32 accumulator in TMEM, which eight epilogue warps read back with
// tcgen05.ld and store (or add) to C.  72 KB of shared memory (a 3-stage
// ring, reused by the epilogue) and 128 TMEM columns per CTA, so three CTAs
// share an SM and their epilogues overlap each other's main loops (measured
// 9 % faster per training step than 4 stages with two CTAs per SM).
//
// Every wait is bounded (about a second); on expiry the kernel sets bit 1 of
// the status word, stops issuing, drains its copies and MMAs and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>
#include <mutex>

#include "fit_tc.cuh"
#include "tc_ptx.cuh"

namespace gcdf {
namespace {

constexpr int kRowsA = 128;                    // A rows per CTA (M = 256 per pair)
constexpr int kTileN = 128;                    // C columns per pair tile
constexpr int kRowsB = kTileN / 2;             // B rows per CTA
constexpr int kKBlock = 64;                    // K per stage: one 128-byte swizzled row
constexpr int kStages = 3;
constexpr int kABytes = kRowsA * 128;          // 16 KB
constexpr int kBBytes = kRowsB * 128;          // 8 KB
constexpr int kStageBytes = kABytes + kBBytes; // 24 KB, a multiple of the 1024-byte swizzle atom
constexpr int kThreads = 320;                  // TMA warp, MMA warp, 8 epilogue warps
constexpr uint32_t kTmemCols = 128;
constexpr int kOffBar = kStages * kStageBytes;
constexpr int B_FULL0 = 0, B_EMPTY0 = kStages, B_ACC = 2 * kStages;
constexpr int kNumBars = 2 * kStages + 1;
constexpr int kOffSlot = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffSlot + 16 + 1024;  // + alignment slack
// the epilogue's two 33 x 32 float tiles per epilogue warp reuse the idle ring
static_assert(8 * 2 * 33 * 32 * 4 <= kStages * kStageBytes, "epilogue tiles fit in the ring");
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s

struct GemmArgs {
  int M, N, kblocks;   // kblocks: K-blocks of the whole product
  int kb_per_split;
  int tiles_n;
  float* C;
  long long ldc;
  long long zstride;   // elements between the outputs of consecutive splits
  int accumulate;
  int* err;
  GemmEpilogue ep;
};

__device__ __forceinline__ uint32_t bar(uint32_t base, int i) { return base + kOffBar + 8 * i; }

// sigma(z) of the BF16 products' epilogues (s(z), s'(z) and s''(z) all use it)
__device__ __forceinline__ float fast_sigmoid(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

__device__ __forceinline__ bool wait_bounded(uint32_t b, uint32_t parity, volatile int* abort_flag, int* err) {
  if (ptx::mbar_try_wait(b, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait(b, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicOr(err, 2);
      return false;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 3)
tc_gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
               const GemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (ptx::smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - ptx::smem_u32(smem_raw));
  __shared__ int abort_flag_s;
  volatile int* abort_flag = &abort_flag_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_ctarank();
  const bool leader = rank == 0;
  const int t = (int)blockIdx.x >> 1;
  const int tm = t / a.tiles_n, tn = t - tm * a.tiles_n;
  const int kb0 = (int)blockIdx.y * a.kb_per_split;
  const int nkb = min(a.kb_per_split, a.kblocks - kb0);  // >= 1 (the host sizes the splits)

  if (threadIdx.x == 0) {
    abort_flag_s = 0;
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(bar(base, B_FULL0 + s), 1);
      ptx::mbar_init(bar(base, B_EMPTY0 + s), 1);
    }
    ptx::mbar_init(bar(base, B_ACC), 1);
    ptx::fence_barrier_init();
    ptx::prefetch_tensormap(&map_a);
    ptx::prefetch_tensormap(&map_b);
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(base + kOffSlot, kTmemCols);
    ptx::tmem_relinquish_pair();
  }
  // both CTAs' barriers are initialised before either signals the other's
  ptx::tc_fence_before();
  ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + kOffSlot);

  if (warp == 0) {
    // ---- TMA producer (both CTAs): this CTA's A rows and B rows of every K-block,
    // completing on the even CTA's FULL barrier
    if (lane == 0) {
      const uint32_t full_lead = ptx::mapa_shared(bar(base, B_FULL0), 0);
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int st = i % kStages;
        if (i >= kStages && !wait_bounded(bar(base, B_EMPTY0 + st), ((uint32_t)(i / kStages) & 1u) ^ 1u,
                                          abort_flag, a.err))
          break;
        if (leader) ptx::mbar_arrive_expect_tx(bar(base, B_FULL0 + st), 2u * kStageBytes);
        const int x = (kb0 + i) * kKBlock;
        const uint32_t fb = full_lead + 8u * (uint32_t)st;
        ptx::tma_load_2d_pair(base + st * kStageBytes, &map_a, x, tm * 2 * kRowsA + (int)rank * kRowsA, fb);
        ptx::tma_load_2d_pair(base + st * kStageBytes + kABytes, &map_b, x, tn * kTileN + (int)rank * kRowsB, fb);
        ++issued;
      }
      // drain (even CTA): only the last kStages stages can still be in flight
      if (leader) {
        for (int k = (issued > kStages ? issued - kStages : 0); k < issued; ++k) {
          const long long t0 = clock64();
          while (!ptx::mbar_try_wait(bar(base, B_FULL0 + k % kStages), (uint32_t)(k / kStages) & 1u))
            if (clock64() - t0 > kWaitCycles) { atomicOr(a.err, 2); break; }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer (even CTA, for both)
    if (lane == 0 && leader) {
      const uint32_t idesc = ptx::idesc_f16kind(2 * kRowsA, kTileN, false);
      const uint64_t d0 = ptx::smem_desc_sw128(base, 1024);
      int issued = 0;
      bool ok = true;
      for (int i = 0; i < nkb; ++i) {
        const int st = i % kStages;
        if (!wait_bounded(bar(base, B_FULL0 + st), (uint32_t)(i / kStages) & 1u, abort_flag, a.err)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint64_t da = d0 + (uint64_t)((st * kStageBytes) >> 4);
        const uint64_t db = d0 + (uint64_t)((st * kStageBytes + kABytes) >> 4);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)  // 32 bytes of K per instruction
          ptx::mma_pair(tmem, da + (uint64_t)(2 * ks), db + (uint64_t)(2 * ks), idesc, (i > 0 || ks > 0) ? 1u : 0u);
        ptx::mma_commit_pair(bar(base, B_EMPTY0 + st));
        ++issued;
      }
      if (ok) ptx::mma_commit_pair(bar(base, B_ACC));
      // every issued MMA completes before TMEM is released
      for (int k = (issued > kStages ? issued - kStages : 0); k < issued; ++k) {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar(base, B_EMPTY0 + k % kStages), (uint32_t)(k / kStages) & 1u))
          if (clock64() - t0 > kWaitCycles) { atomicOr(a.err, 2); break; }
      }
    }
  } else {
    // ---- epilogue: 8 warps; warp w reads TMEM lanes [32 (w mod 4), +32) (its 32
    // rows of the CTA's 128) and columns [64 ch, 64 ch + 64) of the tile, ch = (w - 2) / 4
    const int q = warp & 3;
    const int ch = (warp - 2) >> 2;
    bool ok = true;
    {
      const long long t0 = clock64();
      while (!ptx::mbar_try_wait(bar(base, B_ACC), 0u)) {
        if (*abort_flag || clock64() - t0 > kWaitCycles) {
          atomicOr(a.err, 2);
          ok = false;
          break;
        }
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      ptx::tc_fence_after();
      // Each 32 x 32 block (lane = row after tcgen05.ld) is transposed through
      // shared memory, so that each store instruction writes 32 consecutive
      // values of one row (one 128-byte line of FP32) instead of one value in
      // 32 rows.  The operand ring is idle once the accumulator is complete
      // (every MMA, and so every TMA load, has finished): each warp uses two
      // 33 x 32 float tiles of it (row stride 33: conflict-free both ways), one
      // for the result and one for s'(z) or the incoming factor.
      float* tile = reinterpret_cast<float*>(gbase) + (warp - 2) * (2 * 32 * 33);
      float* tile2 = tile + 32 * 33;
      const int row0 = tm * 2 * kRowsA + (int)rank * kRowsA + q * 32;
      float* cz = a.C ? a.C + (long long)blockIdx.y * a.zstride : nullptr;
      const int n0 = tn * kTileN;
      const GemmEpilogue& ep = a.ep;
      const bool silu = ep.mode == kEpiBiasSilu;
      const bool mul = ep.mode == kEpiMul;
#pragma unroll 1
      for (int c0 = 64 * ch; c0 < 64 * ch + 64; c0 += 32) {
        const int nb = n0 + c0;  // first column of the block
        if (nb >= a.N) break;
        // the block's 32 biases, one per lane, handed to every lane by shuffles
        const float bias_l = silu ? __ldg(ep.bias + min(nb + lane, a.N - 1)) : 0.f;
        if (ep.mode == kEpiMul) {
          // the factor block (and the added block) come in coalesced (lane = column)
#pragma unroll 4
          for (int r = 0; r < 32; ++r) {
            const int rr = row0 + r, n = nb + lane;
            const bool ok_rc = rr < a.M && n < a.N;
            tile2[r * 33 + lane] = ok_rc ? ep.s_in[(long long)rr * ep.ld_s + n] : 0.f;
            if (ep.add_in) tile[r * 33 + lane] = ok_rc ? ep.add_in[(long long)rr * ep.ld_s + n] : 0.f;
          }
          __syncwarp();
        }
        uint32_t u[32];
        ptx::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, u);
        ptx::tmem_wait_ld();
        // this row's 32 results into the tile (s'(z) into the second tile)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float v = __uint_as_float(u[j]);
          if (ep.mode == kEpiMul) {
            const float raw = v;
            v *= tile2[lane * 33 + j];
            if (ep.add_in) v += tile[lane * 33 + j];
            if (ep.acc_out) tile2[lane * 33 + j] = raw;  // (this thread's own element, read above)
          } else if (silu) {
            // h = s(z), z = acc + b; the sigmoid from the fast exponential and
            // division intrinsics (a few ulp in FP32, far below the BF16
            // rounding of every product operand), the same as for s'' below
            const float z = v + __shfl_sync(0xffffffffu, bias_l, j);
            const float sg = fast_sigmoid(z);
            v = z * sg;
            tile2[lane * 33 + j] = sg * (1.f + z * (1.f - sg));
          }
          tile[lane * 33 + j] = v;
        }
        __syncwarp();
        // row-major outputs, lane = column: C (or C += for split partials),
        // s'(z), the BF16 image and the column sums
        const int n = nb + lane;
        if (n < a.N) {
          float cs = 0.f;
#pragma unroll 4
          for (int r = 0; r < 32; ++r) {
            const int rr = row0 + r;
            if (rr < a.M) {
              const float x = tile[r * 33 + lane];
              if (cz) {
                float* c = cz + (long long)rr * a.ldc + n;
                *c = a.accumulate ? *c + x : x;
              }
              if (silu && ep.s_out) ep.s_out[(long long)rr * ep.ld_s + n] = tile2[r * 33 + lane];
              if (mul && ep.acc_out) ep.acc_out[(long long)rr * ep.ld_s + n] = tile2[r * 33 + lane];
              if (ep.img) ep.img[(long long)rr * ep.ld_img + n] = __float2bfloat16_rn(x);
              cs += x;
            }
          }
          // column sums of this block's rows, summed later over the row blocks
          // in a fixed order (blocks past the last row hold no rows)
          if (ep.colsum && row0 < a.M) ep.colsum[(long long)(row0 >> 5) * ep.ld_colsum + n] = cs;
        }
        if (silu && ep.s2_out) {
          // s''(z) for the second-order products: recomputed from the accumulators
          // still in registers, then stored row by row like s'(z)
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float z = __uint_as_float(u[j]) + __shfl_sync(0xffffffffu, bias_l, j);
            const float sg = fast_sigmoid(z);
            tile2[lane * 33 + j] = sg * (1.f - sg) * (2.f + z * (1.f - 2.f * sg));
          }
          __syncwarp();
          if (n < a.N) {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const int rr = row0 + r;
              if (rr < a.M) ep.s2_out[(long long)rr * ep.ld_s + n] = tile2[r * 33 + lane];
            }
          }
        }
        if (ep.imgT && row0 + lane < a.M) {
          // transposed BF16 image: for each column the 32 lanes write 32
          // consecutive rows (64 contiguous bytes)
#pragma unroll 4
          for (int j = 0; j < 32; ++j)
            if (nb + j < a.N)
              ep.imgT[(long long)(nb + j) * ep.ld_imgT + row0 + lane] = __float2bfloat16_rn(tile[lane * 33 + j]);
        }
        __syncwarp();
      }
    }
  }

  // every thread of both CTAs gets here (all waits are bounded)
  __syncwarp();
  ptx::tc_fence_before();
  ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, kTmemCols);
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// rows x cols BF16, row stride ld elements; boxes of 64 K values x box_rows rows;
// positions past rows / cols read as zero
bool encode(CUtensorMap* m, const void* p, long long rows, long long cols, long long ld, int box_rows) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(p), gdim, gstride, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_gemm_tile_m() { return 2 * kRowsA; }
int tc_gemm_tile_n() { return kTileN; }
int tc_gemm_kblock() { return kKBlock; }

namespace {
std::mutex g_fit_mutex;  // guards the per-device status words and attribute flags
}  // namespace

int* fit_status_word() {
  static int* words[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_fit_mutex);
  if (!words[dev]) {
    int* w = nullptr;
    if (cudaMalloc(&w, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(w, 0, sizeof(int)) != cudaSuccess) { cudaFree(w); return nullptr; }
    words[dev] = w;
  }
  return words[dev];
}

cudaError_t tc_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, int M, int N, int K, float* C,
                         long long ldc, long long zstride, int splits, int kb_per_split, bool accumulate, int* err,
                         cudaStream_t s, bool* encode_failed, const GemmEpilogue* ep) {
  *encode_failed = false;
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  {
    // opt in, once per device, to the kernel's dynamic shared memory
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_fit_mutex);
    if (!attr_set[dev]) {
      e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
      if (e != cudaSuccess) return e;
      attr_set[dev] = true;
    }
  }
  CUtensorMap ma, mb;
  if (!encode(&ma, A, M, K, lda, kRowsA) || !encode(&mb, B, N, K, ldb, kRowsB)) {
    *encode_failed = true;
    return cudaSuccess;
  }
  GemmArgs g;
  g.M = M;
  g.N = N;
  g.kblocks = (K + kKBlock - 1) / kKBlock;
  g.kb_per_split = kb_per_split;
  g.tiles_n = (N + kTileN - 1) / kTileN;
  g.C = C;
  g.ldc = ldc;
  g.zstride = zstride;
  g.accumulate = accumulate ? 1 : 0;
  g.err = err;
  if (ep) {
    g.ep = *ep;
  } else {
    memset(&g.ep, 0, sizeof(g.ep));
    g.ep.mode = kEpiStore;
  }
  const int tiles_m = (M + 2 * kRowsA - 1) / (2 * kRowsA);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2u * (unsigned)(tiles_m * g.tiles_n), (unsigned)splits, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tc_gemm_kernel, ma, mb, g);
}

}  // namespace gcdf
