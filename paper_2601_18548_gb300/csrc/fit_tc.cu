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
// the epilogue's two 32 x 36 float tiles per epilogue warp reuse the idle ring
static_assert(8 * 2 * 36 * 32 * 4 <= kStages * kStageBytes, "epilogue tiles fit in the ring");
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

// Rows of p (leading dimension ld elements of eb bytes) all start on an
// `align`-byte boundary (or p is absent).
__device__ __forceinline__ bool rows_aligned(const void* p, long long ld, int eb, int align) {
  return p == nullptr || ((reinterpret_cast<uintptr_t>(p) % align) == 0 && (ld * eb) % align == 0);
}

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
    // the biases of the warp's two 32-column blocks, one per lane, fetched
    // while the main loop runs (handed to every lane by shuffles later)
    float bias_b0 = 0.f, bias_b1 = 0.f;
    if (a.ep.mode == kEpiBiasSilu) {
      const int nb0 = tn * kTileN + 64 * ch;
      if (nb0 < a.N) bias_b0 = __ldg(a.ep.bias + min(nb0 + lane, a.N - 1));
      if (nb0 + 32 < a.N) bias_b1 = __ldg(a.ep.bias + min(nb0 + 32 + lane, a.N - 1));
    }
    // the factor (and added) rows of the warp's 32 rows x 64 columns pulled into
    // L2 while the main loop runs: one 128-byte line per row and block
    if (a.ep.mode == kEpiMul) {
      const int nb0 = tn * kTileN + 64 * ch;
      const int rr = tm * 2 * kRowsA + (int)rank * kRowsA + q * 32 + lane;
      if (rr < a.M) {
#pragma unroll
        for (int bk = 0; bk < 2; ++bk) {
          const int n = nb0 + 32 * bk;
          if (n < a.N) {
            const long long o = (long long)rr * a.ep.ld_s + n;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.ep.s_in + o));
            if (a.ep.add_in) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.ep.add_in + o));
          }
        }
      }
    }
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
      // shared memory, so that global stores run along rows.  The operand ring
      // is idle once the accumulator is complete (every MMA, and so every TMA
      // load, has finished): each warp uses two 32 x 36 float tiles of it (row
      // stride 36 = 144 bytes: 16-byte accesses of a row by the 32 lanes and of
      // 4 rows x 8 column quads by a warp are both conflict-free), one for the
      // result and one for s'(z) or the incoming factor.  Where the block lies
      // inside the matrix and every output row is 16-byte aligned, lane
      // (rg, ck) = (lane / 8, lane mod 8) moves columns 4 ck .. 4 ck + 3 of rows
      // 4 r + rg with 16-byte accesses (a warp covers 4 rows x 128 bytes per
      // instruction); otherwise lane = column, one element per access.
      constexpr int kTs = 36;
      float* tile = reinterpret_cast<float*>(gbase) + (warp - 2) * (2 * 32 * kTs);
      float* tile2 = tile + 32 * kTs;
      const int row0 = tm * 2 * kRowsA + (int)rank * kRowsA + q * 32;
      float* cz = a.C ? a.C + (long long)blockIdx.y * a.zstride : nullptr;
      const int n0 = tn * kTileN;
      const GemmEpilogue& ep = a.ep;
      const bool silu = ep.mode == kEpiBiasSilu;
      const bool mul = ep.mode == kEpiMul;
      const bool vec = rows_aligned(cz, a.ldc, 4, 16) && rows_aligned(ep.s_in, ep.ld_s, 4, 16) &&
                       rows_aligned(ep.add_in, ep.ld_s, 4, 16) && rows_aligned(ep.s_out, ep.ld_s, 4, 16) &&
                       rows_aligned(ep.acc_out, ep.ld_s, 4, 16) && rows_aligned(ep.s2_out, ep.ld_s, 4, 16) &&
                       rows_aligned(ep.img, ep.ld_img, 2, 8) && rows_aligned(ep.colsum, ep.ld_colsum, 4, 16);
      const int rg = lane >> 3, ck = lane & 7;
#pragma unroll 1
      for (int c0 = 64 * ch; c0 < 64 * ch + 64; c0 += 32) {
        const int nb = n0 + c0;  // first column of the block
        if (nb >= a.N) break;
        const bool vb = vec && nb + 32 <= a.N;
        const float bias_l = c0 == 64 * ch ? bias_b0 : bias_b1;
        if (mul) {
          // the factor block (and the added block) come in along rows
          if (vb) {
#pragma unroll 4
            for (int r4 = 0; r4 < 8; ++r4) {
              const int r = 4 * r4 + rg, rr = row0 + r;
              const long long o = (long long)rr * ep.ld_s + nb + 4 * ck;
              const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
              *reinterpret_cast<float4*>(tile2 + r * kTs + 4 * ck) =
                  rr < a.M ? *reinterpret_cast<const float4*>(ep.s_in + o) : z4;
              if (ep.add_in)
                *reinterpret_cast<float4*>(tile + r * kTs + 4 * ck) =
                    rr < a.M ? *reinterpret_cast<const float4*>(ep.add_in + o) : z4;
            }
          } else {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const int rr = row0 + r, n = nb + lane;
              const bool ok_rc = rr < a.M && n < a.N;
              tile2[r * kTs + lane] = ok_rc ? ep.s_in[(long long)rr * ep.ld_s + n] : 0.f;
              if (ep.add_in) tile[r * kTs + lane] = ok_rc ? ep.add_in[(long long)rr * ep.ld_s + n] : 0.f;
            }
          }
          __syncwarp();
        }
        uint32_t u[32];
        ptx::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, u);
        ptx::tmem_wait_ld();
        // this row's 32 results into the tile (s'(z), or the raw accumulator,
        // into the second tile), four columns per 16-byte access; the
        // transposed BF16 image straight from registers: for each column the 32
        // lanes write 32 consecutive rows (64 contiguous bytes)
        const bool row_ok = row0 + lane < a.M;
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f), a4 = f4;
          if (mul) {
            f4 = *reinterpret_cast<const float4*>(tile2 + lane * kTs + 4 * j4);
            if (ep.add_in) a4 = *reinterpret_cast<const float4*>(tile + lane * kTs + 4 * j4);
          }
          const float fj[4] = {f4.x, f4.y, f4.z, f4.w}, aj[4] = {a4.x, a4.y, a4.z, a4.w};
          float vv[4], ww[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int j = 4 * j4 + t;
            float v = __uint_as_float(u[j]);
            float w2 = 0.f;
            if (mul) {
              w2 = v;  // the raw accumulator, for acc_out
              v *= fj[t];
              if (ep.add_in) v += aj[t];
            } else if (silu) {
              // h = s(z), z = acc + b; the sigmoid from the fast exponential and
              // division intrinsics (a few ulp in FP32, far below the BF16
              // rounding of every product operand), the same as for s'' below
              const float z = v + __shfl_sync(0xffffffffu, bias_l, j);
              const float sg = fast_sigmoid(z);
              v = z * sg;
              w2 = sg * (1.f + z * (1.f - sg));
            }
            vv[t] = v;
            ww[t] = w2;
            if (ep.imgT && row_ok && nb + j < a.N)
              ep.imgT[(long long)(nb + j) * ep.ld_imgT + row0 + lane] = __float2bfloat16_rn(v);
          }
          *reinterpret_cast<float4*>(tile + lane * kTs + 4 * j4) = make_float4(vv[0], vv[1], vv[2], vv[3]);
          if (silu || (mul && ep.acc_out))
            *reinterpret_cast<float4*>(tile2 + lane * kTs + 4 * j4) = make_float4(ww[0], ww[1], ww[2], ww[3]);
        }
        __syncwarp();
        // row-major outputs: C (or C += for split partials), s'(z) or the raw
        // accumulator, the BF16 image and the column sums
        if (vb) {
          float4 cs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
          for (int r4 = 0; r4 < 8; ++r4) {
            const int r = 4 * r4 + rg, rr = row0 + r;
            if (rr < a.M) {
              const int n = nb + 4 * ck;
              const float4 x = *reinterpret_cast<const float4*>(tile + r * kTs + 4 * ck);
              if (cz) {
                float4* c = reinterpret_cast<float4*>(cz + (long long)rr * a.ldc + n);
                if (a.accumulate) {
                  const float4 o = *c;
                  *c = make_float4(o.x + x.x, o.y + x.y, o.z + x.z, o.w + x.w);
                } else {
                  *c = x;
                }
              }
              if ((silu && ep.s_out) || (mul && ep.acc_out)) {
                float* dst = silu ? ep.s_out : ep.acc_out;
                *reinterpret_cast<float4*>(dst + (long long)rr * ep.ld_s + n) =
                    *reinterpret_cast<const float4*>(tile2 + r * kTs + 4 * ck);
              }
              if (ep.img) {
                const __nv_bfloat162 lo = __floats2bfloat162_rn(x.x, x.y), hi = __floats2bfloat162_rn(x.z, x.w);
                uint2 pk;
                pk.x = *reinterpret_cast<const uint32_t*>(&lo);
                pk.y = *reinterpret_cast<const uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(ep.img + (long long)rr * ep.ld_img + n) = pk;
              }
              cs.x += x.x;
              cs.y += x.y;
              cs.z += x.z;
              cs.w += x.w;
            }
          }
          // column sums of this block's rows (the four row groups added in a
          // fixed order), summed later over the row blocks in a fixed order
          // (blocks past the last row hold no rows)
#pragma unroll
          for (int o = 8; o <= 16; o <<= 1) {
            cs.x += __shfl_xor_sync(0xffffffffu, cs.x, o);
            cs.y += __shfl_xor_sync(0xffffffffu, cs.y, o);
            cs.z += __shfl_xor_sync(0xffffffffu, cs.z, o);
            cs.w += __shfl_xor_sync(0xffffffffu, cs.w, o);
          }
          if (ep.colsum && row0 < a.M && rg == 0)
            *reinterpret_cast<float4*>(ep.colsum + (long long)(row0 >> 5) * ep.ld_colsum + nb + 4 * ck) = cs;
        } else {
          const int n = nb + lane;
          if (n < a.N) {
            float cs = 0.f;
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const int rr = row0 + r;
              if (rr < a.M) {
                const float x = tile[r * kTs + lane];
                if (cz) {
                  float* c = cz + (long long)rr * a.ldc + n;
                  *c = a.accumulate ? *c + x : x;
                }
                if (silu && ep.s_out) ep.s_out[(long long)rr * ep.ld_s + n] = tile2[r * kTs + lane];
                if (mul && ep.acc_out) ep.acc_out[(long long)rr * ep.ld_s + n] = tile2[r * kTs + lane];
                if (ep.img) ep.img[(long long)rr * ep.ld_img + n] = __float2bfloat16_rn(x);
                cs += x;
              }
            }
            if (ep.colsum && row0 < a.M) ep.colsum[(long long)(row0 >> 5) * ep.ld_colsum + n] = cs;
          }
        }
        if (silu && ep.s2_out) {
          // s''(z) for the second-order products: recomputed from the accumulators
          // still in registers, then stored along rows like s'(z)
          __syncwarp();
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) {
            float ww[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const int j = 4 * j4 + t;
              const float z = __uint_as_float(u[j]) + __shfl_sync(0xffffffffu, bias_l, j);
              const float sg = fast_sigmoid(z);
              ww[t] = sg * (1.f - sg) * (2.f + z * (1.f - 2.f * sg));
            }
            *reinterpret_cast<float4*>(tile2 + lane * kTs + 4 * j4) = make_float4(ww[0], ww[1], ww[2], ww[3]);
          }
          __syncwarp();
          if (vb) {
#pragma unroll 2
            for (int r4 = 0; r4 < 8; ++r4) {
              const int r = 4 * r4 + rg, rr = row0 + r;
              if (rr < a.M)
                *reinterpret_cast<float4*>(ep.s2_out + (long long)rr * ep.ld_s + nb + 4 * ck) =
                    *reinterpret_cast<const float4*>(tile2 + r * kTs + 4 * ck);
            }
          } else if (nb + lane < a.N) {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const int rr = row0 + r;
              if (rr < a.M) ep.s2_out[(long long)rr * ep.ld_s + nb + lane] = tile2[r * kTs + lane];
            }
          }
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
