// Small kernels around the fused GCDF kernels:
//   prep      per-waypoint encoding and first-layer term A_i (the split of the
//             concatenated input of Sec. III-C; see below),
//   tile_map  tile prefix over CSR point lists (partitions I_{M,i}, Sec. IV-A),
//   merge     per-waypoint merge of per-tile partial records in a fixed order.
#include "gcdf_internal.cuh"

namespace gcdf {

// The first layer acts on v = [p', enc(q')].  Because it is affine, it splits
// exactly into a per-point and a per-waypoint term:
//   W_1 v + b_1 = W_1p p + (W_1q enc_i + b_1 - W_1p[:, 0:2] b_i) = W_1p p + A_i
// where W_1p are the three point columns, W_1q the encoding columns and b_i
// the waypoint's base shift.  A_i costs d_q * H multiply-adds per waypoint
// instead of per pair.
__global__ void prep_kernel(const float* __restrict__ q, const float* __restrict__ shift,
                            const float* __restrict__ W1, const float* __restrict__ b1,
                            int n_dof, int H, int d_in, float* __restrict__ A,
                            float* __restrict__ trig) {
  __shared__ float enc[3 + 2 + 2 * kMaxAngles];
  const int i = blockIdx.x;
  const int n_ang = n_dof - 2;
  const float* qi = q + (size_t)i * n_dof;
  if (threadIdx.x == 0) {
    const float bx = shift ? shift[2 * i + 0] : 0.f;
    const float by = shift ? shift[2 * i + 1] : 0.f;
    enc[0] = bx;
    enc[1] = by;
    enc[2] = 0.f;
    enc[3] = qi[0] - bx;
    enc[4] = qi[1] - by;
  }
  if (threadIdx.x < n_ang) {
    float s, c;
    sincosf(qi[2 + threadIdx.x], &s, &c);
    enc[5 + 2 * threadIdx.x] = s;
    enc[6 + 2 * threadIdx.x] = c;
    trig[(size_t)i * 2 * n_ang + 2 * threadIdx.x + 0] = s;
    trig[(size_t)i * 2 * n_ang + 2 * threadIdx.x + 1] = c;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < H; c += blockDim.x) {
    const float* w = W1 + (size_t)c * d_in;
    float acc = b1[c] - w[0] * enc[0] - w[1] * enc[1];
    for (int d = 3; d < d_in; ++d) acc = fmaf(w[d], enc[d + 0], acc);
    A[(size_t)i * H + c] = acc;
  }
}

cudaError_t launch_prep(const WorkDesc& w, const float* W1, const float* b1, int H, int d_in,
                        const float* shift, float* A, float* trig, cudaStream_t s) {
  if (w.N == 0) return cudaSuccess;
  prep_kernel<<<w.N, 256, 0, s>>>(w.q, shift, W1, b1, w.n_dof, H, d_in, A, trig);
  return cudaGetLastError();
}

// tile_start[i] = sum_{i' < i} ceil(m_i' / tile), one block.
__global__ void tile_map_kernel(const int* __restrict__ offsets, int N, int tile,
                                int* __restrict__ tile_start) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int lo = min(N, t * per), hi = min(N, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) {
    const int m = max(0, offsets[i + 1] - offsets[i]);
    sum += (m + tile - 1) / tile;
  }
  part[t] = sum;
  __syncthreads();
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    const int v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - sum;  // exclusive prefix of this thread's segment
  for (int i = lo; i < hi; ++i) {
    tile_start[i] = run;
    const int m = max(0, offsets[i + 1] - offsets[i]);
    run += (m + tile - 1) / tile;
  }
  if (t == blockDim.x - 1) tile_start[N] = part[t];
}

cudaError_t launch_tile_map(const int* offsets, int N, int tile, int* tile_start, cudaStream_t s) {
  tile_map_kernel<<<1, 1024, 0, s>>>(offsets, N, tile, tile_start);
  return cudaGetLastError();
}

// One warp per waypoint.  Lane l merges tiles l, l + 32, ... in increasing
// order, then the lanes merge in a fixed butterfly; the result therefore
// depends only on the waypoint's own tiles.
__global__ void merge_kernel(WorkDesc w, float* __restrict__ cost, float* __restrict__ grad,
                             int* __restrict__ argmin) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= w.N) return;
  int t0, t1;
  if (w.tile_start) {
    t0 = w.tile_start[warp];
    t1 = w.tile_start[warp + 1];
  } else {
    t0 = warp * w.tiles_per_wp;
    t1 = t0 + w.tiles_per_wp;
  }
  const float T = w.param;
  Partial acc = partial_identity(w.mode);
  for (int t = t0 + lane; t < t1; t += 32) acc = partial_combine(w.mode, T, acc, w.partials[t]);
  acc = partial_warp_reduce(w.mode, T, acc);
  const int n = w.n_dof;
  if (lane == 0) {
    float c;
    if (acc.pos == 0x7fffffff) {
      c = (w.mode == kHinge) ? 0.f : __int_as_float(0x7f800000);
    } else if (w.mode == kSoftmin) {
      c = acc.v0 - T * logf(acc.v1);
    } else {
      c = acc.v0;
    }
    cost[warp] = c;
    if (argmin) argmin[warp] = acc.idx;
  }
  if (lane < n) {
    float g = acc.g[0];
#pragma unroll
    for (int d = 1; d < kMaxDof; ++d)
      if (lane == d) g = acc.g[d];
    if (acc.pos == 0x7fffffff) g = 0.f;
    else if (w.mode == kSoftmin) g = g / acc.v1;
    grad[(size_t)warp * n + lane] = g;
  }
}

cudaError_t launch_merge(const WorkDesc& w, int n_waypoints, float* cost, float* grad, int* argmin,
                         cudaStream_t s) {
  if (n_waypoints == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (n_waypoints * 32 + threads - 1) / threads;
  merge_kernel<<<blocks, threads, 0, s>>>(w, cost, grad, argmin);
  return cudaGetLastError();
}

// ---- active sets of the HINGE and MIN reductions --------------------------------
//
// HINGE needs df/dq only for the pairs with f < delta (the l1 penalty of Eq. 12
// is zero and flat elsewhere) and MIN only at each waypoint's first minimising
// entry.  After a value-only pass has written f for every list position, these
// kernels build, per waypoint, the list of positions whose gradient the
// reduction needs, in list order:
//   HINGE  every position with f < delta or f NaN (a NaN value must reach the
//          cost); when there is none, the minimising position alone (it keeps
//          the argmin and adds max(0, delta - f) = 0 and no gradient);
//   MIN    the minimising position alone.
// The minimising position ranks NaN first, then the smallest f, then the lowest
// position (the fused kernels' rule).  Empty lists stay empty.  The reduction
// over these lists gives the full reduction's cost, gradient and argmin: the
// positions left out add exactly zero to the HINGE sums.

namespace {

constexpr int kActThreads = 256;
constexpr int kActPer = 8;  // consecutive positions per thread and round

__device__ __forceinline__ bool act_better(float fa, int pa, float fb, int pb) {
  return first_is_better(fa, pa, fb, pb);
}

__device__ __forceinline__ int list_len(const WorkDesc& w, int wp) {
  return w.offsets ? (w.offsets[wp + 1] - w.offsets[wp]) : w.M;
}

__device__ __forceinline__ long long list_pair(const WorkDesc& w, int wp, int pos) {
  return w.offsets ? (long long)w.offsets[wp] + pos : (long long)wp * w.M + pos;
}

}  // namespace

// One block per waypoint: cnt[i] = length of its active list, nact[i] = number
// of f < delta or NaN positions (HINGE), amin[i] = its minimising position.
__global__ void __launch_bounds__(kActThreads) active_count_kernel(WorkDesc w, const float* __restrict__ f,
                                                                  int* __restrict__ cnt, int* __restrict__ nact,
                                                                  int* __restrict__ amin) {
  __shared__ float sf[kActThreads / 32];
  __shared__ int sp[kActThreads / 32], sc[kActThreads / 32];
  const int wp = blockIdx.x;
  const int m = list_len(w, wp);
  const float delta = w.param;
  float bf = 0.f;
  int bp = 0x7fffffff, c = 0;
  for (int r = threadIdx.x; r < m; r += kActThreads) {
    const float v = f[list_pair(w, wp, r)];
    if (bp == 0x7fffffff || act_better(v, r, bf, bp)) { bf = v; bp = r; }
    c += (v < delta || v != v) ? 1 : 0;
  }
  // warp, then block: the best (f, position) and the count
  for (int o = 16; o > 0; o >>= 1) {
    const float of = __shfl_xor_sync(0xffffffffu, bf, o);
    const int op = __shfl_xor_sync(0xffffffffu, bp, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    if (op != 0x7fffffff && (bp == 0x7fffffff || act_better(of, op, bf, bp))) { bf = of; bp = op; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sf[warp] = bf; sp[warp] = bp; sc[warp] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float f0 = sf[0];
    int p0 = sp[0], c0 = sc[0];
    for (int k = 1; k < kActThreads / 32; ++k) {
      c0 += sc[k];
      if (sp[k] != 0x7fffffff && (p0 == 0x7fffffff || act_better(sf[k], sp[k], f0, p0))) { f0 = sf[k]; p0 = sp[k]; }
    }
    const int has = m > 0 ? 1 : 0;
    if (w.mode == kHinge) {
      nact[wp] = c0;
      cnt[wp] = c0 > 0 ? c0 : has;
    } else {
      nact[wp] = 0;
      cnt[wp] = has;
    }
    amin[wp] = has ? p0 : -1;
  }
}

// out[0] = 0, out[i + 1] = cnt[0] + ... + cnt[i] (one block).
__global__ void exclusive_scan_kernel(const int* __restrict__ cnt, int N, int* __restrict__ out) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int lo = min(N, t * per), hi = min(N, lo + per);
  long long sum = 0;
  for (int i = lo; i < hi; ++i) sum += cnt[i];
  part[t] = sum;
  __syncthreads();
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    const long long v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = part[t] - sum;
  if (t == 0) out[0] = 0;
  for (int i = lo; i < hi; ++i) {
    run += cnt[i];
    out[i + 1] = (int)run;
  }
}

// One block per waypoint: its active positions, in list order, written as point
// indices at out_idx[out_off[i] ...].
__global__ void __launch_bounds__(kActThreads) active_fill_kernel(WorkDesc w, const float* __restrict__ f,
                                                                 const int* __restrict__ out_off,
                                                                 const int* __restrict__ nact,
                                                                 const int* __restrict__ amin,
                                                                 int* __restrict__ out_idx) {
  __shared__ int warp_sum[kActThreads / 32];
  __shared__ int base_s;
  const int wp = blockIdx.x;
  const int m = list_len(w, wp);
  const int o = out_off[wp];
  if (m == 0) return;
  if (w.mode != kHinge || nact[wp] == 0) {
    if (threadIdx.x == 0) {
      int j;
      long long k;
      pair_at(w, wp, amin[wp], j, k);
      out_idx[o] = j;
    }
    return;
  }
  const float delta = w.param;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  for (int r0 = 0; r0 < m; r0 += kActThreads * kActPer) {
    // this thread's kActPer consecutive positions
    const int p0 = r0 + threadIdx.x * kActPer;
    unsigned keep = 0u;
#pragma unroll
    for (int u = 0; u < kActPer; ++u) {
      const int r = p0 + u;
      if (r < m) {
        const float v = f[list_pair(w, wp, r)];
        if (v < delta || v != v) keep |= 1u << u;
      }
    }
    const int c = __popc(keep);
    // block exclusive scan of the thread counts
    int incl = c;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < warp; ++k) before += warp_sum[k];
    int total = 0;
    for (int k = 0; k < kActThreads / 32; ++k) total += warp_sum[k];
    int pos = o + base_s + before + incl - c;
#pragma unroll
    for (int u = 0; u < kActPer; ++u) {
      if (keep & (1u << u)) {
        int j;
        long long k;
        pair_at(w, wp, p0 + u, j, k);
        out_idx[pos++] = j;
      }
    }
    __syncthreads();  // every thread has read warp_sum and base_s
    if (threadIdx.x == 0) base_s += total;
    __syncthreads();
  }
}

cudaError_t launch_active_lists(const WorkDesc& w, const float* f, int* cnt, int* nact, int* amin, int* out_off,
                                int* out_idx, cudaStream_t s) {
  if (w.N == 0) return cudaSuccess;
  active_count_kernel<<<w.N, kActThreads, 0, s>>>(w, f, cnt, nact, amin);
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(cnt, w.N, out_off);
  active_fill_kernel<<<w.N, kActThreads, 0, s>>>(w, f, out_off, nact, amin, out_idx);
  return cudaGetLastError();
}

}  // namespace gcdf
