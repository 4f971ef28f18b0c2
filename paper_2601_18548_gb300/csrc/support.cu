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

}  // namespace gcdf
