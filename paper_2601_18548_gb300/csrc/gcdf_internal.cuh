// Internal declarations shared by the libgcdf translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/gcdf.h"

namespace gcdf {

constexpr int kMaxDof = 12;
constexpr int kMaxAngles = kMaxDof - 2;
constexpr int kPartialFloats = 16;  // one per-tile partial record (see Partial)

// Reduction modes as seen by the kernels (query mode writes per-pair outputs).
enum Mode : int { kQuery = -1, kMin = GCDF_RED_MIN, kSoftmin = GCDF_RED_SOFTMIN, kHinge = GCDF_RED_HINGE };

// Per-tile partial result of a reduction, merged per waypoint in tile order.
//   MIN:     v0 = min f, idx = point index of the first minimising entry (-1 none),
//            g = df/dq at that entry.
//   SOFTMIN: v0 = running minimum m, v1 = sum exp(-(f - m)/T), g = sum exp(-(f - m)/T) df/dq,
//            idx as MIN.
//   HINGE:   v0 = sum max(0, delta - f), g = -sum_{f < delta} df/dq, idx as MIN (v1 = min f).
// Layout in memory: 16 floats = [v0, v1, idx (int bits), pos (int bits), g[0..11]].
struct Partial {
  float v0, v1;
  int idx, pos;
  float g[kMaxDof];
};
static_assert(sizeof(Partial) == kPartialFloats * 4, "partial record size");

// What one launch works on.  A tile is `tile` consecutive entries of one
// waypoint's point list; tiles are numbered waypoint-major.
struct WorkDesc {
  const float* q;        // (N, n)
  const float* p;        // (M, 3)
  const int* offsets;    // (N + 1) or nullptr (dense)
  const int* idx;        // (n_pairs) or nullptr
  const int* point_base; // range lists (internal): with offsets and no idx, list position r
                         // of waypoint i is point point_base[i] + r
  const float* A;        // (N, H) first-layer waypoint term, from the prep kernel
  const float* trig;     // (N, 2 * n_ang): sin, cos of every angle, from the prep kernel
  const int* tile_start; // (N + 1) tile prefix (CSR); nullptr for dense
  int N, M, n_pairs;
  int n_dof, n_ang;
  int tile;              // pairs per tile
  int tiles_per_wp;      // dense only
  int n_tiles;           // dense: exact; CSR: upper bound (tile_start[N] is exact)
  int mode;
  float param;
  float* f_out;          // query: (n_pairs)
  float* g_out;          // query: (n_pairs, n) or nullptr
  Partial* partials;     // reductions: (n_tiles)
  // tensor-core path with gradients: per-CTA stash of 2 s'(z_l), layers 1..L-1
  // (tc_stash_bytes); nullptr lets launch_tc take it from the library's pool
  void* stash;
};

// Locate tile t: its waypoint, first list position and valid length.
__device__ __forceinline__ bool tile_lookup(const WorkDesc& w, int t, int& wp, int& start, int& len) {
  if (w.tile_start == nullptr) {
    wp = t / w.tiles_per_wp;
    start = (t - wp * w.tiles_per_wp) * w.tile;
    len = min(w.tile, w.M - start);
    return wp < w.N;
  }
  if (t >= w.tile_start[w.N]) return false;
  int lo = 0, hi = w.N;  // largest i with tile_start[i] <= t
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (w.tile_start[mid] <= t) lo = mid; else hi = mid;
  }
  wp = lo;
  start = (t - w.tile_start[lo]) * w.tile;
  int m = w.offsets[lo + 1] - w.offsets[lo];
  len = min(w.tile, m - start);
  return true;
}

// Point index and global pair index of list position `pos` of waypoint `wp`.
__device__ __forceinline__ void pair_at(const WorkDesc& w, int wp, int pos, int& j, long long& k) {
  if (w.offsets == nullptr) {
    j = pos;
    k = (long long)wp * w.M + pos;
  } else {
    k = (long long)w.offsets[wp] + pos;
    j = w.idx ? w.idx[k] : w.point_base[wp] + pos;
  }
}

// ---- per-tile partial records -------------------------------------------------

__device__ __forceinline__ Partial partial_identity(int mode) {
  Partial r;
  r.v0 = (mode == kHinge) ? 0.f : __int_as_float(0x7f800000);
  r.v1 = (mode == kHinge) ? __int_as_float(0x7f800000) : 0.f;
  r.idx = -1;
  r.pos = 0x7fffffff;
#pragma unroll
  for (int d = 0; d < kMaxDof; ++d) r.g[d] = 0.f;
  return r;
}

// Partial record of a single pair at list position `pos` (point index `idx`).
__device__ __forceinline__ Partial partial_of_pair(int mode, float param, float f, const float* dq,
                                                   int n, int idx, int pos) {
  Partial r = partial_identity(mode);
  r.idx = idx;
  r.pos = pos;
  if (mode == kHinge) {
    r.v0 = fmaxf(0.f, param - f);
    if (f != f) r.v0 = f;  // NaN propagates
    r.v1 = f;
    const bool act = f < param;
    for (int d = 0; d < n; ++d) r.g[d] = act ? -dq[d] : 0.f;
  } else {
    r.v0 = f;
    r.v1 = 1.f;
    for (int d = 0; d < n; ++d) r.g[d] = dq[d];
  }
  return r;
}

// Smallest f tracked by a record (for argmin), NaN counting as smallest.
__device__ __forceinline__ float partial_minf(int mode, const Partial& a) {
  return mode == kHinge ? a.v1 : a.v0;
}

__device__ __forceinline__ bool first_is_better(float fa, int pa, float fb, int pb) {
  const bool na = fa != fa, nb = fb != fb;
  if (na || nb) return na && (!nb || pa < pb);
  return fa < fb || (fa == fb && pa < pb);
}

// Merge two records of the same waypoint.  Exact for MIN (a selection);
// fixed rounding for SOFTMIN / HINGE given a fixed merge tree.
__device__ __forceinline__ Partial partial_combine(int mode, float T, const Partial& a, const Partial& b) {
  if (a.pos == 0x7fffffff) return b;
  if (b.pos == 0x7fffffff) return a;
  const bool a_first = first_is_better(partial_minf(mode, a), a.pos, partial_minf(mode, b), b.pos);
  Partial r;
  if (mode == kMin) {
    return a_first ? a : b;
  }
  r.idx = a_first ? a.idx : b.idx;
  r.pos = a_first ? a.pos : b.pos;
  if (mode == kHinge) {
    r.v0 = a.v0 + b.v0;
    r.v1 = a_first ? a.v1 : b.v1;
#pragma unroll
    for (int d = 0; d < kMaxDof; ++d) r.g[d] = a.g[d] + b.g[d];
    return r;
  }
  // SOFTMIN: both records hold (m, s, G) relative to their own minimum m.
  const float m = a_first ? a.v0 : b.v0;
  const float ea = (a.v0 == m) ? 1.f : expf(-(a.v0 - m) / T);
  const float eb = (b.v0 == m) ? 1.f : expf(-(b.v0 - m) / T);
  r.v0 = m;
  r.v1 = a.v1 * ea + b.v1 * eb;
#pragma unroll
  for (int d = 0; d < kMaxDof; ++d) r.g[d] = a.g[d] * ea + b.g[d] * eb;
  return r;
}

__device__ __forceinline__ Partial partial_shfl_xor(const Partial& a, int lane_mask) {
  Partial r;
  r.v0 = __shfl_xor_sync(0xffffffffu, a.v0, lane_mask);
  r.v1 = __shfl_xor_sync(0xffffffffu, a.v1, lane_mask);
  r.idx = __shfl_xor_sync(0xffffffffu, a.idx, lane_mask);
  r.pos = __shfl_xor_sync(0xffffffffu, a.pos, lane_mask);
#pragma unroll
  for (int d = 0; d < kMaxDof; ++d) r.g[d] = __shfl_xor_sync(0xffffffffu, a.g[d], lane_mask);
  return r;
}

// Butterfly merge over the 32 lanes of a warp; every lane ends with the result.
// The merge tree depends only on lane numbers, so the result is deterministic.
__device__ __forceinline__ Partial partial_warp_reduce(int mode, float T, Partial a) {
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) {
    Partial o = partial_shfl_xor(a, m);
    const int lane = threadIdx.x & 31;
    a = (lane & m) ? partial_combine(mode, T, o, a) : partial_combine(mode, T, a, o);
  }
  return a;
}

// Stream-ordered device allocation of the library's temporaries, from a
// library-owned memory pool per device that keeps freed memory for reuse
// (defined in gcdf_api.cu); freed with cudaFreeAsync.
cudaError_t lib_malloc_async(void** out, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t lib_malloc_async(T** out, size_t bytes, cudaStream_t s) {
  return lib_malloc_async(reinterpret_cast<void**>(out), bytes, s);
}

// Host-side launchers (defined in the .cu files).
cudaError_t launch_prep(const WorkDesc& w, const float* W1, const float* b1, int H, int d_in,
                        const float* shift, float* A, float* trig, cudaStream_t s);
cudaError_t launch_tile_map(const int* offsets, int N, int tile, int* tile_start, cudaStream_t s);
cudaError_t launch_merge(const WorkDesc& w, int n_waypoints, float* cost, float* grad, int* argmin,
                         cudaStream_t s);
// Active lists of a HINGE / MIN reduction (w.mode, w.param) from the values f
// of every list position of w: out_off (N + 1) and point indices out_idx (at
// most w.n_pairs, or N for MIN); cnt, nact, amin (N) are temporaries.
cudaError_t launch_active_lists(const WorkDesc& w, const float* f, int* cnt, int* nact, int* amin, int* out_off,
                                int* out_idx, cudaStream_t s);

struct Fp32Weights {
  const float* BF;   // (L-1) x [H][H]: forward operand, row = input feature, columns permuted
  const float* BB;   // (L-1) x [H][H]: backward operand, row = output feature, columns permuted
  const float* bias; // (L-1) x [H]: biases of layers 2..L, permuted
  const float* W1;   // [H][d_in] first layer, original layout
  const float* wout; // [H] output weights, permuted
  float bout;
  int H, L, d_in, d_q;
};
cudaError_t launch_fp32(const WorkDesc& w, const Fp32Weights& fw, int num_sms, cudaStream_t s);
size_t fp32_smem_bytes(int H, int L);

struct TcWeights {
  CUtensorMap map_w;           // stacked 16-bit operands of layers 2..L (forward, then transposed)
  CUtensorMap map_j;           // 16-bit W_1q^T, padded to nj rows
  const float* bias;           // (L-1) x [H] biases of layers 2..L
  const float* W1p;            // [H][3] point columns of layer 1
  const float* wout;           // [H]
  float bout;
  int H, L, d_q, nj;
  int fmt;                     // operand format: 0 = BF16, 1 = FP16, 2 = FP8 E4M3
  float fp8_scale[8];          // FP8: weight scales, forward layers 2..L, reverse layers, W_1q
  int* err;                    // device status word (set when a bounded wait gives up)
};
cudaError_t launch_tc(const WorkDesc& w, const TcWeights& tw, int num_sms, cudaStream_t s);
// Bytes of the stash a launch with L layers uses on at most num_sms SMs (value-
// only queries use none).
size_t tc_stash_bytes(int L, int num_sms);
size_t tc_image_elems(int H, int L, int d_q);
// Operand image (16-bit elements, or bytes for FP8) and, for FP8, the scales.
void tc_build_image(const float* W, int H, int L, int d_q, int d_in, int fmt, void* out, float* scales);
int tc_encode_maps(const void* image, int H, int L, int d_q, int fmt, TcWeights& tw);
int tc_nj(int d_q);
cudaError_t launch_wait_expiry_probe(int* err, long long limit_cycles, int* seen, cudaStream_t s);
cudaError_t launch_fma_rate(int blocks, int threads, int iters, float* sink, cudaStream_t s);
long long fma_rate_flops_per_thread(int iters);

}  // namespace gcdf
