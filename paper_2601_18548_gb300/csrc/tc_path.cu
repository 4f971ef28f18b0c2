// BF16 / FP16 tensor-core fused GCDF kernel (tcgen05 + TMEM + TMA), sm_103a.
//
// What it computes per (waypoint i, point j) pair — the same network and
// reverse sweep as the FP32 path (Sec. III-C network, Sec. IV-A batched values
// and gradients):
//   z_1 = A_i + W_1p p_j,  h_l = s(z_l),  z_{l+1} = W_{l+1} h_l + b_{l+1},
//   f = w_o . s(z_L) + b_o,
//   g_L = w_o * s'(z_L),  g_{l-1} = (W_l^T g_l) * s'(z_{l-1}),  df/denc = W_1q^T g_1,
// followed by the sin/cos chain rule and either per-pair outputs or a
// per-tile partial of the min / soft-min / hinge reduction.
//
// Mapping onto the SM.  A tile is 128 pairs of one waypoint (the MMA's M).
// Every H x H product — forward and reverse — is one 128 x 256 x 256 MMA
// chain issued by one thread: D (TMEM, FP32) = A (shared, 16-bit, 128 pairs x K)
// x B (shared, 16-bit weight slab); the 16-bit format is BF16 or FP16.  A holds the current activations h_l (or
// reverse gradients g_l) and is rewritten in place by the epilogue warps after
// each MMA chain completes.  Weights stream through a ring of 32 KB slabs
// (256 rows x 64 K, 128-byte swizzle) loaded by TMA; the forward operand of
// layer l is W_l and the reverse operand is a stored copy of W_l^T, so both
// are K-major.  s'(z_l) of layers 2..L-1 is kept in TMEM next to the
// accumulator as packed FP16 pairs (an internal value, so it takes the 16-bit
// format with more mantissa bits whatever the operand format); s'(z_1) is
// recomputed from A_i + W_1p p_j.
//
// TMEM columns (512 allocated): [0, 256) accumulator; [256 + 128 s, 384 + 128 s)
// stash of s'(z_{s+2}), s = 0..L-3.
//
// Warp roles (320 threads): warp 0 issues TMA loads, warp 1 allocates TMEM and
// issues MMAs, warps 2..9 are the epilogue (thread = one pair row; warps
// 2..5 take columns 0..127, warps 6..9 columns 128..255).
//
// Every wait on an mbarrier is bounded (about a second); on expiry the kernel
// records an error in a device status word, stops issuing work, drains its
// outstanding copies and MMAs and frees TMEM before returning.
#include <cstring>
#include <vector>

#include "gcdf_internal.cuh"
#include "tc_ptx.cuh"

namespace gcdf {

namespace {

constexpr int kTile = 128;          // pairs per tile (MMA M)
constexpr int kH = 256;             // hidden width handled by this kernel
constexpr int kStages = 4;          // weight ring depth
constexpr int kSlabBytes = kH * 128;  // 256 rows x 64 bf16
constexpr int kABytes = kTile * kH * 2;
constexpr int kThreads = 320;
constexpr int kEpiThreads = 256;
constexpr uint32_t kTmemCols = 512;

// shared memory map (offsets from the 1024-aligned base)
constexpr int kOffA = 0;
constexpr int kOffRing = kOffA + kABytes;                     // 65536
constexpr int kOffJ = kOffRing + kStages * kSlabBytes;        // 196608
constexpr int kJBytesMax = 4 * 32 * 128;                      // nj <= 32
constexpr int kOffBias = kOffJ + kJBytesMax;                  // (L-1) x 256 floats, L <= 4
constexpr int kOffW1p = kOffBias + 3 * kH * 4;
constexpr int kOffWout = kOffW1p + 3 * kH * 4;
constexpr int kOffAi = kOffWout + kH * 4;
constexpr int kOffPts = kOffAi + kH * 4;                      // 128 x float4
constexpr int kOffF = kOffPts + kTile * 16;                   // 2 x 128 floats
constexpr int kOffPart = kOffF + 2 * kTile * 4;               // 4 partial records
constexpr int kOffBar = kOffPart + 4 * (int)sizeof(Partial);
constexpr int kNumBars = 2 * kStages + 4;
constexpr int kOffSlot = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffSlot + 16 + 1024;              // + alignment slack

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at GB300 clocks

struct Shared {
  uint32_t base;      // shared-window address of the aligned base
  uint8_t* gbase;     // generic pointer to the aligned base
};

__device__ __forceinline__ uint32_t bar_addr(const Shared& sh, int i) { return sh.base + kOffBar + 8 * i; }
// barrier indices
__device__ __forceinline__ int B_FULL(int s) { return s; }
__device__ __forceinline__ int B_EMPTY(int s) { return kStages + s; }
constexpr int B_J = 2 * kStages;
constexpr int B_ACC = 2 * kStages + 1;
constexpr int B_AFULL = 2 * kStages + 2;
constexpr int B_DONE = 2 * kStages + 3;

// Bounded wait; returns false (and raises the abort flag) on expiry or when
// another role has already aborted.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      atomicOr(err, 1);
      return false;
    }
  }
}

__device__ __forceinline__ float silu_sig(float z) { return fmaf(0.5f, ptx::tanh_approx(0.5f * z), 0.5f); }

// Byte offset of element (row, k) of a 128-row, 256-wide K-major BF16 operand
// stored as four 64-wide chunks in the 128-byte swizzle layout; k multiple of 8.
__device__ __forceinline__ uint32_t a_offset(int row, int k) {
  const int chunk = k >> 6;
  const int j = (k & 63) >> 3;
  return chunk * (kTile * 128) + (row >> 3) * 1024 + (row & 7) * 128 + ((j ^ (row & 7)) << 4);
}

__device__ __forceinline__ int total_tiles(const WorkDesc& w) {
  return w.tile_start ? w.tile_start[w.N] : w.n_tiles;
}

template <bool kF16>
__global__ void __launch_bounds__(kThreads, 1)
tc_fused_kernel(const WorkDesc w, const __grid_constant__ CUtensorMap map_w,
                const __grid_constant__ CUtensorMap map_j, const TcWeights tw) {
  extern __shared__ uint8_t smem_raw[];
  Shared sh;
  sh.base = (ptx::smem_u32(smem_raw) + 1023u) & ~1023u;
  sh.gbase = smem_raw + (sh.base - ptx::smem_u32(smem_raw));
  __shared__ int abort_flag_s;
  volatile int* abort_flag = &abort_flag_s;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int L = tw.L;
  const int n_wphases = 2 * (L - 1);       // MMA chains that read weight slabs, per tile
  const int n_phases = n_wphases + 1;      // plus the input-Jacobian chain
  const int nj = tw.nj;
  const int ntiles = total_tiles(w);
  int my_tiles = 0;
  if ((int)blockIdx.x < ntiles) my_tiles = (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;

  float* s_bias = reinterpret_cast<float*>(sh.gbase + kOffBias);
  float* s_w1p = reinterpret_cast<float*>(sh.gbase + kOffW1p);
  float* s_wout = reinterpret_cast<float*>(sh.gbase + kOffWout);
  float* s_ai = reinterpret_cast<float*>(sh.gbase + kOffAi);
  float4* s_pts = reinterpret_cast<float4*>(sh.gbase + kOffPts);
  float* s_f = reinterpret_cast<float*>(sh.gbase + kOffF);
  Partial* s_part = reinterpret_cast<Partial*>(sh.gbase + kOffPart);
  uint32_t* s_slot = reinterpret_cast<uint32_t*>(sh.gbase + kOffSlot);

  // ---- setup -------------------------------------------------------------------
  if (tid == 0) {
    abort_flag_s = 0;
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(bar_addr(sh, B_FULL(s)), 1);
      ptx::mbar_init(bar_addr(sh, B_EMPTY(s)), 1);
    }
    ptx::mbar_init(bar_addr(sh, B_J), 1);
    ptx::mbar_init(bar_addr(sh, B_ACC), 1);
    ptx::mbar_init(bar_addr(sh, B_AFULL), kEpiThreads);
    ptx::mbar_init(bar_addr(sh, B_DONE), 1);
    ptx::fence_barrier_init();
    ptx::prefetch_tensormap(&map_w);
    ptx::prefetch_tensormap(&map_j);
  }
  if (warp == 1) {
    ptx::tmem_alloc(sh.base + kOffSlot, kTmemCols);
    ptx::tmem_relinquish();
  }
  for (int i = tid; i < (L - 1) * kH; i += kThreads) s_bias[i] = tw.bias[i];
  for (int i = tid; i < 3 * kH; i += kThreads) s_w1p[i] = tw.W1p[i];
  for (int i = tid; i < kH; i += kThreads) s_wout[i] = tw.wout[i];
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *s_slot;

  if (warp == 0) {
    // ================= TMA producer =================
    if (lane == 0 && my_tiles > 0) {
      const uint32_t jbytes = 4u * nj * 128u;
      ptx::mbar_arrive_expect_tx(bar_addr(sh, B_J), jbytes);
      for (int kc = 0; kc < 4; ++kc)
        ptx::tma_load_2d(sh.base + kOffJ + kc * nj * 128, &map_j, kc * 64, 0, bar_addr(sh, B_J));
      long long g = 0;
      bool ok = true;
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int ph = 0; ph < n_wphases && ok; ++ph) {
          const int row = (ph < L - 1) ? ph * kH : (L - 1 + (2 * L - 3 - ph)) * kH;
          for (int kc = 0; kc < 4; ++kc, ++g) {
            const int s = (int)(g % kStages);
            const uint32_t u = (uint32_t)(g / kStages);
            if (u > 0 && !wait_bar(bar_addr(sh, B_EMPTY(s)), (u - 1) & 1u, abort_flag, tw.err)) { ok = false; break; }
            ptx::mbar_arrive_expect_tx(bar_addr(sh, B_FULL(s)), kSlabBytes);
            ptx::tma_load_2d(sh.base + kOffRing + s * kSlabBytes, &map_w, kc * 64, row, bar_addr(sh, B_FULL(s)));
          }
        }
      }
      // drain: every issued load must land before the CTA exits
      for (long long k = (g > kStages ? g - kStages : 0); k < g; ++k) {
        const int s = (int)(k % kStages);
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar_addr(sh, B_FULL(s)), (uint32_t)(k / kStages) & 1u))
          if (clock64() - t0 > kWaitCycles) { atomicOr(tw.err, 2); break; }
      }
      {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar_addr(sh, B_J), 0))
          if (clock64() - t0 > kWaitCycles) { atomicOr(tw.err, 2); break; }
      }
    }
  } else if (warp == 1) {
    // ================= MMA issuer =================
    if (lane == 0 && my_tiles > 0) {
      const uint32_t id256 = ptx::idesc_f16kind(kTile, kH, kF16);
      const uint32_t idj = ptx::idesc_f16kind(kTile, nj, kF16);
      long long g = 0;
      uint32_t ak = 0;
      bool ok = wait_bar(bar_addr(sh, B_J), 0, abort_flag, tw.err);
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int ph = 0; ph < n_phases && ok; ++ph) {
          if (!wait_bar(bar_addr(sh, B_AFULL), ak & 1u, abort_flag, tw.err)) { ok = false; break; }
          ++ak;
          ptx::tc_fence_after();
          if (ph < n_wphases) {
            for (int kc = 0; kc < 4; ++kc, ++g) {
              const int s = (int)(g % kStages);
              if (!wait_bar(bar_addr(sh, B_FULL(s)), (uint32_t)(g / kStages) & 1u, abort_flag, tw.err)) {
                ok = false;
                break;
              }
              ptx::tc_fence_after();
              const uint32_t aslab = sh.base + kOffA + kc * (kTile * 128);
              const uint32_t bslab = sh.base + kOffRing + s * kSlabBytes;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                ptx::mma_bf16(tmem, ptx::smem_desc_sw128(aslab + ks * 32, 1024),
                              ptx::smem_desc_sw128(bslab + ks * 32, 1024), id256, (kc | ks) != 0);
              ptx::mma_commit(bar_addr(sh, B_EMPTY(s)));
            }
            if (!ok) break;
          } else {
            for (int kc = 0; kc < 4; ++kc) {
              const uint32_t aslab = sh.base + kOffA + kc * (kTile * 128);
              const uint32_t bslab = sh.base + kOffJ + kc * nj * 128;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                ptx::mma_bf16(tmem, ptx::smem_desc_sw128(aslab + ks * 32, 1024),
                              ptx::smem_desc_sw128(bslab + ks * 32, 1024), idj, (kc | ks) != 0);
            }
          }
          ptx::mma_commit(bar_addr(sh, B_ACC));
        }
      }
      // all issued MMAs complete before TMEM is released
      ptx::mma_commit(bar_addr(sh, B_DONE));
      const long long t0 = clock64();
      while (!ptx::mbar_try_wait(bar_addr(sh, B_DONE), 0))
        if (clock64() - t0 > kWaitCycles) { atomicOr(tw.err, 2); break; }
    }
  } else {
    // ================= epilogue: 8 warps, one pair row per thread =================
    const int e = warp - 2;
    const int quad = warp & 3;
    const int hf = e >> 2;
    const int row = quad * 32 + lane;
    const int col0 = hf * 128;
    const int etid = e * 32 + lane;  // 0..255
    const uint32_t t_lane = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t a_base = sh.base + kOffA;
    const int n = w.n_dof;
    uint32_t acc_k = 0;
    bool ok = true;
    for (int it = 0; it < my_tiles && ok; ++it) {
      const int t = (int)blockIdx.x + it * (int)gridDim.x;
      int wp = 0, start = 0, len = 0;
      tile_lookup(w, t, wp, start, len);
      ptx::named_bar_sync(1, kEpiThreads);  // previous tile fully consumed
      s_ai[etid] = w.A[(size_t)wp * kH + etid];
      if (etid < kTile) {
        float4 pv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (etid < len) {
          int j;
          long long k;
          pair_at(w, wp, start + etid, j, k);
          pv = make_float4(w.p[3 * (size_t)j], w.p[3 * (size_t)j + 1], w.p[3 * (size_t)j + 2], 0.f);
        }
        s_pts[etid] = pv;
      }
      ptx::named_bar_sync(1, kEpiThreads);
      const float4 pt = s_pts[row];

      // ---- P1: h_1 = s(A_i + W_1p p) -> A --------------------------------------
      for (int c = col0; c < col0 + 128; c += 8) {
        uint32_t pk[4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
          float hv[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int cc = c + i + u;
            const float z = fmaf(s_w1p[3 * cc + 2], pt.z, fmaf(s_w1p[3 * cc + 1], pt.y, fmaf(s_w1p[3 * cc], pt.x, s_ai[cc])));
            hv[u] = z * silu_sig(z);
          }
          pk[i >> 1] = ptx::pack2<kF16>(hv[0], hv[1]);
        }
        ptx::st_shared_v4(a_base + a_offset(row, c), pk[0], pk[1], pk[2], pk[3]);
      }
      ptx::tc_fence_before();
      ptx::fence_proxy_async_smem();
      ptx::mbar_arrive(bar_addr(sh, B_AFULL));

      float fpart = 0.f;
      for (int ph = 0; ph < n_phases; ++ph) {
        if (!wait_bar(bar_addr(sh, B_ACC), acc_k & 1u, abort_flag, tw.err)) { ok = false; break; }
        ++acc_k;
        ptx::tc_fence_after();
        if (ph < L - 1) {
          // forward epilogue of layer l = ph + 2
          const int l = ph + 2;
          const float* bias = s_bias + (l - 2) * kH;
          for (int cc = 0; cc < 128; cc += 32) {
            const int c0 = col0 + cc;
            uint32_t v[32];
            ptx::tmem_ld32(t_lane + c0, v);
            ptx::tmem_wait_ld();
            uint32_t hp[16], dp[16];
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
              float hv[2], dv[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const float z = __uint_as_float(v[i + u]) + bias[c0 + i + u];
                const float sg = silu_sig(z);
                const float h = z * sg;
                const float d = sg * fmaf(z, 1.f - sg, 1.f);
                if (l == L) {
                  fpart = fmaf(s_wout[c0 + i + u], h, fpart);
                  hv[u] = s_wout[c0 + i + u] * d;  // g_L
                } else {
                  hv[u] = h;
                }
                dv[u] = d;
              }
              hp[i >> 1] = ptx::pack2<kF16>(hv[0], hv[1]);
              dp[i >> 1] = ptx::pack_f16x2(dv[0], dv[1]);  // stash is always FP16
            }
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              ptx::st_shared_v4(a_base + a_offset(row, c0 + 8 * q4), hp[4 * q4], hp[4 * q4 + 1], hp[4 * q4 + 2],
                                hp[4 * q4 + 3]);
            if (l < L) ptx::tmem_st16(t_lane + 256 + 128 * (l - 2) + (c0 >> 1), dp);
          }
          if (l < L) ptx::tmem_wait_st();
          if (l == L) s_f[hf * kTile + row] = fpart;
        } else if (ph < n_wphases) {
          // reverse epilogue: g_{l-1} = u * s'(z_{l-1}), l = 2L - 1 - ph
          const int lm1 = 2 * L - 2 - ph;
          for (int cc = 0; cc < 128; cc += 32) {
            const int c0 = col0 + cc;
            uint32_t v[32];
            uint32_t sd[16];
            ptx::tmem_ld32(t_lane + c0, v);
            if (lm1 >= 2) ptx::tmem_ld16(t_lane + 256 + 128 * (lm1 - 2) + (c0 >> 1), sd);
            ptx::tmem_wait_ld();
            uint32_t gp[16];
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
              float gv[2];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                float d;
                if (lm1 >= 2) {
                  d = u ? ptx::f16hi(sd[i >> 1]) : ptx::f16lo(sd[i >> 1]);
                } else {
                  const int c = c0 + i + u;
                  const float z = fmaf(s_w1p[3 * c + 2], pt.z, fmaf(s_w1p[3 * c + 1], pt.y, fmaf(s_w1p[3 * c], pt.x, s_ai[c])));
                  const float sg = silu_sig(z);
                  d = sg * fmaf(z, 1.f - sg, 1.f);
                }
                gv[u] = __uint_as_float(v[i + u]) * d;
              }
              gp[i >> 1] = ptx::pack2<kF16>(gv[0], gv[1]);
            }
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4)
              ptx::st_shared_v4(a_base + a_offset(row, c0 + 8 * q4), gp[4 * q4], gp[4 * q4 + 1], gp[4 * q4 + 2],
                                gp[4 * q4 + 3]);
          }
        } else {
          // input-Jacobian result: df/denc in accumulator columns [0, d_q)
          ptx::named_bar_sync(2, kEpiThreads);  // s_f written by both halves
          if (hf == 0) {
            uint32_t v[32];
            ptx::tmem_ld32(t_lane, v);
            ptx::tmem_wait_ld();
            const float fval = s_f[row] + s_f[kTile + row] + tw.bout;
            const float* tr = w.trig + (size_t)wp * 2 * w.n_ang;
            float dq[kMaxDof];
#pragma unroll
            for (int d = 0; d < kMaxDof; ++d) dq[d] = 0.f;
            dq[0] = __uint_as_float(v[0]);
            dq[1] = __uint_as_float(v[1]);
#pragma unroll
            for (int a = 0; a < kMaxAngles; ++a)
              if (a < w.n_ang)
                dq[2 + a] = tr[2 * a + 1] * __uint_as_float(v[2 + 2 * a]) - tr[2 * a] * __uint_as_float(v[3 + 2 * a]);
            const bool valid = row < len;
            int j = -1;
            long long k = 0;
            if (valid) pair_at(w, wp, start + row, j, k);
            if (w.mode == kQuery) {
              if (valid) {
                w.f_out[k] = fval;
                if (w.g_out)
                  for (int d = 0; d < n; ++d) w.g_out[(size_t)k * n + d] = dq[d];
              }
            } else {
              Partial pr = valid ? partial_of_pair(w.mode, w.param, fval, dq, n, j, start + row)
                                 : partial_identity(w.mode);
              pr = partial_warp_reduce(w.mode, w.param, pr);
              if (lane == 0) s_part[quad] = pr;
              ptx::named_bar_sync(3, 128);
              if (quad == 0 && lane == 0) {
                Partial a = s_part[0];
                for (int qq = 1; qq < 4; ++qq) a = partial_combine(w.mode, w.param, a, s_part[qq]);
                w.partials[t] = a;
              }
            }
          }
          break;  // no A write after the last chain of the tile
        }
        ptx::tc_fence_before();
        ptx::fence_proxy_async_smem();
        ptx::mbar_arrive(bar_addr(sh, B_AFULL));
      }
    }
  }

  // ---- teardown ---------------------------------------------------------------
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTmemCols);
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
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

int encode_2d(CUtensorMap* m, const void* base, int rows, int cols, int box_rows, bool f16) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return 1;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 2;
}

}  // namespace

int tc_tile_pairs() { return kTile; }

bool tc_supported(int H, int L, int n_dof) { return H == kH && L >= 2 && L <= 4 && n_dof >= 3 && n_dof <= kMaxDof; }

int tc_nj(int d_q) { return d_q <= 16 ? 16 : 32; }

// Image layout (BF16, row-major, 256 columns): rows [256 m, 256 m + 256) hold
// W_{m+2} for m = 0..L-2 (forward operands, row = output feature), then rows
// [256 (L-1+m), ...) hold W_{m+2}^T (reverse operands, row = input feature),
// then nj rows of W_1q^T (row d = input column 3 + d of layer 1; zero rows pad).
size_t tc_image_elems(int H, int L, int d_q) {
  return (size_t)2 * (L - 1) * H * H + (size_t)tc_nj(d_q) * H;
}

static uint16_t to_bits(float x, bool f16) {
  if (f16) {
    const __half h = __float2half_rn(x);
    return *reinterpret_cast<const uint16_t*>(&h);
  }
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&b);
}

void tc_build_image(const float* W, int H, int L, int d_q, int d_in, bool f16, uint16_t* out) {
  size_t off = (size_t)H * d_in + H;
  for (int m = 0; m < L - 1; ++m) {
    const float* Wl = W + off;
    uint16_t* fwd = out + (size_t)m * H * H;
    uint16_t* rev = out + (size_t)(L - 1 + m) * H * H;
    for (int o = 0; o < H; ++o)
      for (int i = 0; i < H; ++i) {
        const uint16_t b = to_bits(Wl[(size_t)o * H + i], f16);
        fwd[(size_t)o * H + i] = b;
        rev[(size_t)i * H + o] = b;
      }
    off += (size_t)H * H + H;
  }
  uint16_t* J = out + (size_t)2 * (L - 1) * H * H;
  const int nj = tc_nj(d_q);
  for (int d = 0; d < nj; ++d)
    for (int c = 0; c < H; ++c)
      J[(size_t)d * H + c] = to_bits(d < d_q ? W[(size_t)c * d_in + 3 + d] : 0.f, f16);
}

int tc_encode_maps(const uint16_t* image, int H, int L, int d_q, bool f16, TcWeights& tw) {
  int rc = encode_2d(&tw.map_w, image, 2 * (L - 1) * H, H, 256, f16);
  if (rc) return rc;
  return encode_2d(&tw.map_j, image + (size_t)2 * (L - 1) * H * H, tc_nj(d_q), H, tc_nj(d_q), f16);
}

template <bool kF16>
cudaError_t launch_tc_t(const WorkDesc& w, const TcWeights& tw, int num_sms, cudaStream_t s) {
  static int attr_done[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(tc_fused_kernel<kF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_done[dev] = 1;
  }
  const int grid = w.n_tiles < num_sms ? w.n_tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  tc_fused_kernel<kF16><<<grid, kThreads, kSmemBytes, s>>>(w, tw.map_w, tw.map_j, tw);
  return cudaGetLastError();
}

cudaError_t launch_tc(const WorkDesc& w, const TcWeights& tw, int num_sms, cudaStream_t s) {
  return tw.f16 ? launch_tc_t<true>(w, tw, num_sms, s) : launch_tc_t<false>(w, tw, num_sms, s);
}

}  // namespace gcdf
