// FP32 fused GCDF kernel on CUDA cores: value f(q_i, p_j) and df/dq for every
// pair of a tile, then per-pair outputs (query) or a per-tile partial record
// (collision-cost reductions).
//
// Per pair the network is (Sec. III-C; synthetic shape)
//   z_1 = A_i + W_1p p_j                 (first layer, split per waypoint/point)
//   h_l = s(z_l),  z_{l+1} = W_{l+1} h_l + b_{l+1}     l = 1..L-1
//   f   = w_o . s(z_L) + b_o
// and the reverse sweep for the configuration gradient (Sec. IV-A: the solver
// needs values and gradients of every constraint):
//   g_L = w_o * s'(z_L),  g_{l-1} = (W_l^T g_l) * s'(z_{l-1}),
//   df/denc = W_1q^T g_1,  then the sin/cos chain rule.
//
// A query without a gradient output runs the forward layers only.
//
// Layout.  A tile is TP = 8192 / H pairs of one waypoint.  256 threads; thread
// (pg, fg) owns pairs 4pg..4pg+3 and features fg + G f (f = 0..7, G = H / 8);
// a warp spans 2 pair groups and 16 feature groups (4 and 8 for H = 64).
// Activations live in shared memory feature-major, act[c][pair] (row stride
// TP + 4 floats); weight rows stream through a double-buffered shared chunk of
// KC rows with cp.async.  The weight images are pre-permuted on the host so a
// thread's 8 features are two 16-byte pieces of a row, at 4 fg and H / 2 + 4 fg:
// the feature groups of a warp read each half as one contiguous piece.
// s'(z_l) of layers 2..L-1 stays in shared memory for the reverse sweep;
// s'(z_1) is recomputed from A_i + W_1p p_j, which costs three FMAs.
#include "gcdf_internal.cuh"

namespace gcdf {

namespace {

__device__ __forceinline__ float sigmoid_acc(float z) { return 1.0f / (1.0f + expf(-z)); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

template <int H, int KC>
struct Cfg {
  static constexpr int TP = 8192 / H;
  static constexpr int G = H / 8;
  static constexpr int PG = TP / 4;
  static constexpr int AS = TP + 4;
  static constexpr int NCH = H / KC;  // chunks per matrix
  static_assert(PG * G == 256, "256 threads");
  static_assert(H % KC == 0, "chunking");
};

struct SmemLayout {
  size_t act, stash, wbuf, fpart, denc, pts, total;
};

template <int H, int KC>
__host__ __device__ constexpr size_t smem_floats_act() { return (size_t)H * Cfg<H, KC>::AS; }

template <int H, int KC>
__host__ __device__ inline SmemLayout smem_layout(int L) {
  using C = Cfg<H, KC>;
  SmemLayout s{};
  size_t o = 0;
  s.act = o;   o += (size_t)H * C::AS;
  s.stash = o; o += (size_t)(L - 2) * H * C::AS;
  s.wbuf = o;  o += (size_t)2 * KC * H;
  s.fpart = o; o += (size_t)C::G * C::TP;
  s.denc = o;  o += (size_t)C::TP * 24;
  s.pts = o;   o += (size_t)C::TP * 4;
  s.total = o * sizeof(float);
  return s;
}

// Chunk `c` of the per-tile weight sequence: forward layers 2..L then backward L..2.
template <int H, int KC>
__device__ __forceinline__ const float* chunk_src(const Fp32Weights& fw, int c) {
  using C = Cfg<H, KC>;
  const int phase = c / C::NCH;
  const int part = c - phase * C::NCH;
  const int nl = fw.L - 1;
  const float* base = (phase < nl) ? fw.BF + (size_t)phase * H * H
                                   : fw.BB + (size_t)(2 * nl - 1 - phase) * H * H;
  return base + (size_t)part * KC * H;
}

template <int H, int KC>
__device__ __forceinline__ void load_chunk(float* dst, const float* src) {
  constexpr int n16 = KC * H / 4;
#pragma unroll 4
  for (int k = threadIdx.x; k < n16; k += 256) cp_async16(dst + 4 * k, src + 4 * k);
  cp_async_commit();
}

template <int H, int KC>
__global__ void __launch_bounds__(256, 1)
fp32_fused_kernel(const WorkDesc w, const Fp32Weights fw) {
  using C = Cfg<H, KC>;
  extern __shared__ __align__(16) float smem[];
  const SmemLayout lay = smem_layout<H, KC>(fw.L);
  float* act = smem + lay.act;
  float* stash = smem + lay.stash;
  float* wbuf = smem + lay.wbuf;
  float* fpart = smem + lay.fpart;
  float* denc = smem + lay.denc;
  float* pts = smem + lay.pts;

  const int tid = threadIdx.x;
  // A warp covers WP pair groups x WF feature groups (2 x 16 where the tile
  // allows it, else 4 x 8), lanes running over the pair groups first
  // (lane = WP fg + pg within the warp): each of its two weight reads per K
  // step covers WF x 16 contiguous bytes, each read by WP lanes, and its
  // activation read WP distinct 16-byte pieces.  Against 4 x 8 with one pair
  // group per 8-lane phase this measured 1.1 % (2 x 16) and 2.6 % (4 x 8,
  // pair groups first) faster, the fully unrolled K chunk 3.4 % on top.
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int WF = C::G % 16 == 0 && C::PG % 2 == 0 ? 16 : 8;  // feature groups per warp
  constexpr int WP = 32 / WF;                                     // pair groups per warp
  static_assert(C::PG % WP == 0 && C::G % WF == 0, "warp tiling");
  const int pg = (warp / (C::G / WF)) * WP + (lane % WP);
  const int fg = (warp % (C::G / WF)) * WF + (lane / WP);
  const int L = fw.L;
  // value-only query (no gradient output): the forward layers alone
  const bool fwd_only = (w.mode == kQuery && w.g_out == nullptr);
  const int n_phases = fwd_only ? (L - 1) : 2 * (L - 1);
  const int nseq = n_phases * C::NCH;  // chunks per tile
  const int n = w.n_dof;
  const int d_q = fw.d_q;

  long long gchunk = 0;  // global chunk counter: buffer = gchunk & 1
  if (blockIdx.x < w.n_tiles) load_chunk<H, KC>(wbuf, chunk_src<H, KC>(fw, 0));

  for (int t = blockIdx.x; t < w.n_tiles; t += gridDim.x) {
    int wp, start, len;
    if (!tile_lookup(w, t, wp, start, len)) break;

    // ---- tile points ---------------------------------------------------------
    if (tid < C::TP) {
      float x = 0.f, y = 0.f, z = 0.f;
      if (tid < len) {
        int j;
        long long k;
        pair_at(w, wp, start + tid, j, k);
        x = w.p[3 * (size_t)j + 0];
        y = w.p[3 * (size_t)j + 1];
        z = w.p[3 * (size_t)j + 2];
      }
      pts[4 * tid + 0] = x;
      pts[4 * tid + 1] = y;
      pts[4 * tid + 2] = z;
    }
    __syncthreads();

    // ---- layer 1 (split): z1 = A_i + W1p p ------------------------------------
    const float* Ai = w.A + (size_t)wp * H;
    float a1[8], wpx[8], wpy[8], wpz[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      const int c = fg + C::G * f;
      a1[f] = Ai[c];
      wpx[f] = fw.W1[(size_t)c * fw.d_in + 0];
      wpy[f] = fw.W1[(size_t)c * fw.d_in + 1];
      wpz[f] = fw.W1[(size_t)c * fw.d_in + 2];
    }
    float px[4], py[4], pz[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      px[r] = pts[4 * (4 * pg + r) + 0];
      py[r] = pts[4 * (4 * pg + r) + 1];
      pz[r] = pts[4 * (4 * pg + r) + 2];
    }
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      float4 h;
      float* hv = reinterpret_cast<float*>(&h);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float z = fmaf(wpz[f], pz[r], fmaf(wpy[f], py[r], fmaf(wpx[f], px[r], a1[f])));
        hv[r] = z * sigmoid_acc(z);
      }
      *reinterpret_cast<float4*>(act + (size_t)(fg + C::G * f) * C::AS + 4 * pg) = h;
    }

    // ---- forward layers 2..L and reverse sweep L..2 ---------------------------
    float fsum[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ph = 0; ph < n_phases; ++ph) {
      float acc[4][8];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int f = 0; f < 8; ++f) acc[r][f] = 0.f;

      for (int part = 0; part < C::NCH; ++part, ++gchunk) {
        cp_async_wait_all();
        __syncthreads();  // chunk visible to all; previous buffer and act writes done
        {
          const int cnext = (int)((gchunk + 1) % nseq);
          const bool more = (cnext != 0) || (t + (int)gridDim.x < w.n_tiles);
          if (more) load_chunk<H, KC>(wbuf + ((gchunk + 1) & 1) * KC * H, chunk_src<H, KC>(fw, cnext));
        }
        const float* wb = wbuf + (gchunk & 1) * KC * H + 4 * fg;  // features f < 4; f >= 4 at + H / 2
        const float* ab = act + (size_t)(part * KC) * C::AS + 4 * pg;
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
          const float4 a = *reinterpret_cast<const float4*>(ab + (size_t)kk * C::AS);
          const float4 w0 = *reinterpret_cast<const float4*>(wb + (size_t)kk * H);
          const float4 w1 = *reinterpret_cast<const float4*>(wb + (size_t)kk * H + H / 2);
          const float av[4] = {a.x, a.y, a.z, a.w};
          const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int f = 0; f < 8; ++f) acc[r][f] = fmaf(av[r], wv[f], acc[r][f]);
        }
      }
      __syncthreads();  // everyone done reading act for this phase

      if (ph < L - 1) {
        // forward epilogue of layer l = ph + 2
        const int l = ph + 2;
        const float* bias = fw.bias + (size_t)(l - 2) * H + 8 * fg;
        float bv[8], wo[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) bv[f] = bias[f];
        if (l == L) {
#pragma unroll
          for (int f = 0; f < 8; ++f) wo[f] = fw.wout[8 * fg + f];
        }
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          float4 hv4, sv4;
          float* hv = reinterpret_cast<float*>(&hv4);
          float* sv = reinterpret_cast<float*>(&sv4);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float z = acc[r][f] + bv[f];
            const float s = sigmoid_acc(z);
            const float h = z * s;
            const float d = s * (1.f + z * (1.f - s));
            if (l == L) {
              fsum[r] = fmaf(wo[f], h, fsum[r]);
              hv[r] = wo[f] * d;  // g_L
            } else {
              hv[r] = h;
              sv[r] = d;
            }
          }
          const size_t row = (size_t)(fg + C::G * f) * C::AS + 4 * pg;
          *reinterpret_cast<float4*>(act + row) = hv4;
          if (l < L) *reinterpret_cast<float4*>(stash + (size_t)(l - 2) * H * C::AS + row) = sv4;
        }
        if (l == L) {
#pragma unroll
          for (int r = 0; r < 4; ++r) fpart[fg * C::TP + 4 * pg + r] = fsum[r];
        }
      } else {
        // reverse epilogue: g_{l-1} = u * s'(z_{l-1}) with l = L - (ph - (L - 1))
        const int l = 2 * L - 1 - ph;  // ph = L-1 -> l = L
        const int lm1 = l - 1;
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          const int c = fg + C::G * f;
          const size_t row = (size_t)c * C::AS + 4 * pg;
          float dv[4];
          if (lm1 >= 2) {
            const float4 s4 = *reinterpret_cast<const float4*>(stash + (size_t)(lm1 - 2) * H * C::AS + row);
            dv[0] = s4.x; dv[1] = s4.y; dv[2] = s4.z; dv[3] = s4.w;
          } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const float z = fmaf(wpz[f], pz[r], fmaf(wpy[f], py[r], fmaf(wpx[f], px[r], a1[f])));
              const float s = sigmoid_acc(z);
              dv[r] = s * (1.f + z * (1.f - s));
            }
          }
          float4 g4 = make_float4(acc[0][f] * dv[0], acc[1][f] * dv[1], acc[2][f] * dv[2], acc[3][f] * dv[3]);
          *reinterpret_cast<float4*>(act + row) = g4;
        }
      }
    }
    __syncthreads();  // act holds g_1 [c][pair]; fpart complete

    // ---- df/denc = W_1q^T g_1 ------------------------------------------------
    for (int o = tid; o < (fwd_only ? 0 : C::TP * d_q); o += 256) {
      const int pair = o % C::TP;
      const int d = o / C::TP;
      const float* wcol = fw.W1 + 3 + d;
      float s = 0.f;
#pragma unroll 8
      for (int c = 0; c < H; ++c) s = fmaf(act[(size_t)c * C::AS + pair], __ldg(wcol + (size_t)c * fw.d_in), s);
      denc[pair * 24 + d] = s;
    }
    __syncthreads();

    // ---- per pair: f, chain rule, outputs / partials ---------------------------
    if (tid < ((C::TP + 31) / 32) * 32) {
      const int pair = tid;
      const bool valid = pair < len;
      float fval = 0.f;
      float dq[kMaxDof];
#pragma unroll
      for (int d = 0; d < kMaxDof; ++d) dq[d] = 0.f;
      int j = -1;
      long long k = 0;
      if (pair < C::TP) {
        float s = fw.bout;
        for (int g = 0; g < C::G; ++g) s += fpart[g * C::TP + pair];
        fval = s;
        const float* de = denc + pair * 24;
        const float* tr = w.trig + (size_t)wp * 2 * w.n_ang;
        if (!fwd_only) {
          dq[0] = de[0];
          dq[1] = de[1];
          for (int a = 0; a < w.n_ang; ++a) dq[2 + a] = tr[2 * a + 1] * de[2 + 2 * a] - tr[2 * a] * de[3 + 2 * a];
        }
        if (valid) pair_at(w, wp, start + pair, j, k);
      }
      if (w.mode == kQuery) {
        if (valid) {
          w.f_out[k] = fval;
          if (w.g_out)
            for (int d = 0; d < n; ++d) w.g_out[(size_t)k * n + d] = dq[d];
        }
      } else {
        Partial pr = valid ? partial_of_pair(w.mode, w.param, fval, dq, n, j, start + pair)
                           : partial_identity(w.mode);
        pr = partial_warp_reduce(w.mode, w.param, pr);
        // TP <= 32 for H >= 256: one warp holds the tile.  Larger tiles merge warps in order.
        __shared__ Partial wpart[4];
        if ((tid & 31) == 0) wpart[warp] = pr;
        if (C::TP > 32) asm volatile("bar.sync 1, %0;\n" ::"r"(((C::TP + 31) / 32) * 32));
        if (tid == 0) {
          Partial acc = wpart[0];
          for (int q2 = 1; q2 < (C::TP + 31) / 32; ++q2) acc = partial_combine(w.mode, w.param, acc, wpart[q2]);
          w.partials[t] = acc;
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait_all();
}

template <int H, int KC>
cudaError_t launch_h(const WorkDesc& w, const Fp32Weights& fw, int num_sms, cudaStream_t s) {
  const SmemLayout lay = smem_layout<H, KC>(fw.L);
  // Opt in (per device) to the dynamic shared memory this L needs.
  static int attr_bytes[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || attr_bytes[dev] < (int)lay.total) {
    cudaError_t e = cudaFuncSetAttribute(fp32_fused_kernel<H, KC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_bytes[dev] = (int)lay.total;
  }
  const int grid = w.n_tiles < num_sms ? w.n_tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  fp32_fused_kernel<H, KC><<<grid, 256, lay.total, s>>>(w, fw);
  return cudaGetLastError();
}

}  // namespace

size_t fp32_smem_bytes(int H, int L) {
  switch (H) {
    case 64: return smem_layout<64, 64>(L).total;
    case 128: return smem_layout<128, 64>(L).total;
    case 256: return smem_layout<256, 32>(L).total;
    case 512: return smem_layout<512, 8>(L).total;
    default: return 0;
  }
}

int fp32_tile_pairs(int H) { return 8192 / H; }

cudaError_t launch_fp32(const WorkDesc& w, const Fp32Weights& fw, int num_sms, cudaStream_t s) {
  switch (fw.H) {
    case 64: return launch_h<64, 64>(w, fw, num_sms, s);
    case 128: return launch_h<128, 64>(w, fw, num_sms, s);
    case 256: return launch_h<256, 32>(w, fw, num_sms, s);
    case 512: return launch_h<512, 8>(w, fw, num_sms, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gcdf
