// Constraint-structure kernels around the fused GCDF pass (Sec. IV-A):
//   partition   per-waypoint lists I_{M,i} of the obstacle points within a
//               planar range R of the waypoint's reference base position
//               (count, scan, order-preserving fill);
//   jacobian    the dense (sum m_i) x n gradient block placed into the sparse
//               (sum m_i) x 2Nn Jacobian of Eq. (17): P_i of Eq. (18) puts the
//               n entries of a row of waypoint i at columns 2n(i-1) .. 2n(i-1)+n-1
//               (the columns of q_i in the state vector [x_1; ...; x_N],
//               x_i = [q_i, v_i]), written as CSR;
//   project     the single-step projection of Theorem 1,
//               q_z = q - f(p, q) M^{-1} grad_q f(p, q), for every pair.
#include <cstring>

#include "gcdf_internal.cuh"

namespace gcdf {

int set_error(int code, const char* fmt, ...);
void clear_error();
int net_n_dof(const gcdf_net* net);

namespace {

constexpr int kPartThreads = 256;
constexpr int kPerThread = 8;  // consecutive points per thread and tile of the fill

// Inside the planar range: FP64 on the FP32 inputs, each product and the sum
// rounded separately (no contraction), compared with R * R.
__device__ __forceinline__ bool in_range(const float* __restrict__ p, int j, double bx, double by, double r2) {
  const double dx = __dsub_rn((double)p[3 * (size_t)j], bx);
  const double dy = __dsub_rn((double)p[3 * (size_t)j + 1], by);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= r2;
}

// Row i tests points [begin_i, begin_i + len_i) of p (pbegin / plen NULL: all
// M points) against its base (x, y) at base + i * bstride; listed indices are
// indices into p.
struct RowRanges {
  const float* base;
  int bstride;
  const int* pbegin;
  const int* plen;
  int M;
  __device__ int begin(int i) const { return pbegin ? pbegin[i] : 0; }
  __device__ int len(int i) const { return plen ? plen[i] : M; }
};

__global__ void partition_count_kernel(RowRanges rr, const float* __restrict__ p, double r2,
                                       int* __restrict__ counts) {
  __shared__ int red[kPartThreads / 32];
  const int i = blockIdx.x;
  const double bx = rr.base[(size_t)i * rr.bstride], by = rr.base[(size_t)i * rr.bstride + 1];
  const int b0 = rr.begin(i), m = rr.len(i);
  int c = 0;
  for (int j = threadIdx.x; j < m; j += kPartThreads) c += in_range(p, b0 + j, bx, by, r2);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kPartThreads / 32; ++w) s += red[w];
    counts[i] = s;
  }
}

// out[0] = 0, out[k + 1] = in[0] + ... + in[k]; one block.
__global__ void exclusive_scan_kernel(const int* __restrict__ in, int N, int* __restrict__ out) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int lo = min(N, t * per), hi = min(N, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += in[i];
  part[t] = sum;
  __syncthreads();
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    const int v = (t >= d) ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - sum;
  if (t == 0) out[0] = 0;
  for (int i = lo; i < hi; ++i) {
    run += in[i];
    out[i + 1] = run;
  }
}

// One block per waypoint: tiles of kPartThreads * kPerThread points in order;
// thread t tests points tile + 8t .. tile + 8t + 7, the block scans the thread
// counts, so the list keeps increasing point order.
__global__ void partition_fill_kernel(RowRanges rr, const float* __restrict__ p, double r2,
                                      const int* __restrict__ offsets, int* __restrict__ idx) {
  __shared__ int wsum[kPartThreads / 32];
  __shared__ int s_total;
  const int i = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const double bx = rr.base[(size_t)i * rr.bstride], by = rr.base[(size_t)i * rr.bstride + 1];
  const int b0 = rr.begin(i), M = rr.len(i);
  int run = offsets[i];
  for (int tile = 0; tile < M; tile += kPartThreads * kPerThread) {
    const int j0 = tile + t * kPerThread;
    unsigned mask = 0;
#pragma unroll
    for (int u = 0; u < kPerThread; ++u)
      if (j0 + u < M && in_range(p, b0 + j0 + u, bx, by, r2)) mask |= 1u << u;
    const int c = __popc(mask);
    int x = c;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += v;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (t == 0) {
      int s = 0;
      for (int k = 0; k < kPartThreads / 32; ++k) {
        const int v = wsum[k];
        wsum[k] = s;
        s += v;
      }
      s_total = s;
    }
    __syncthreads();
    int pos = run + wsum[w] + x - c;
    for (int u = 0; u < kPerThread; ++u)
      if (mask & (1u << u)) idx[pos++] = b0 + j0 + u;
    run += s_total;
    __syncthreads();
  }
}

__device__ __forceinline__ int waypoint_of_row(const int* __restrict__ offsets, int N, int M, long long k) {
  if (offsets == nullptr) return k < 0x7fffffffLL ? (int)k / M : (int)(k / M);
  int lo = 0, hi = N;  // largest i with offsets[i] <= k
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offsets[mid] <= k) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int kRowsPerBlock = 256;  // rows of one block of the Jacobian / projection passes

// A block takes kRowsPerBlock consecutive rows: each thread looks up one row's
// waypoint, then the block streams the rows' n entries with coalesced loads
// and stores (element e of the block's range is row e / n, entry e % n).
__global__ void __launch_bounds__(kRowsPerBlock) jacobian_kernel(
    const float* __restrict__ grad, int N, int n, const int* __restrict__ offsets, int M, long long K,
    long long* __restrict__ row_ptr, int* __restrict__ col_idx, float* __restrict__ values) {
  __shared__ int s_col[kRowsPerBlock];
  for (long long k0 = (long long)blockIdx.x * kRowsPerBlock; k0 < K; k0 += (long long)gridDim.x * kRowsPerBlock) {
    const int rows = (int)min((long long)kRowsPerBlock, K - k0);
    if ((int)threadIdx.x < rows) {
      const long long k = k0 + threadIdx.x;
      s_col[threadIdx.x] = 2 * n * waypoint_of_row(offsets, N, M, k);
      row_ptr[k] = k * n;
    }
    __syncthreads();
    const long long e0 = k0 * n;
    for (int el = threadIdx.x; el < rows * n; el += kRowsPerBlock) {
      const int r = el / n, d = el - r * n;
      col_idx[e0 + el] = s_col[r] + d;
      if (values) values[e0 + el] = grad[e0 + el];
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[K] = K * n;
}

// g holds df/dq of every pair on entry and the projected configuration on exit.
__global__ void __launch_bounds__(kRowsPerBlock) project_kernel(
    const float* __restrict__ q, int N, int n, const int* __restrict__ offsets, int M, long long K,
    const float* __restrict__ f, const float* __restrict__ m_diag, float* __restrict__ g) {
  __shared__ int s_wp[kRowsPerBlock];
  __shared__ float s_f[kRowsPerBlock];
  __shared__ float s_minv[kMaxDof];
  if ((int)threadIdx.x < n) s_minv[threadIdx.x] = m_diag ? 1.0f / m_diag[threadIdx.x] : 1.0f;
  for (long long k0 = (long long)blockIdx.x * kRowsPerBlock; k0 < K; k0 += (long long)gridDim.x * kRowsPerBlock) {
    const int rows = (int)min((long long)kRowsPerBlock, K - k0);
    if ((int)threadIdx.x < rows) {
      const long long k = k0 + threadIdx.x;
      s_wp[threadIdx.x] = waypoint_of_row(offsets, N, M, k);
      s_f[threadIdx.x] = f[k];
    }
    __syncthreads();
    float* gb = g + k0 * n;
    for (int el = threadIdx.x; el < rows * n; el += kRowsPerBlock) {
      const int r = el / n, d = el - r * n;
      gb[el] = fmaf(-s_f[r], gb[el] * s_minv[d], q[(size_t)s_wp[r] * n + d]);
    }
    __syncthreads();
  }
}

int grid_for(long long work, int threads, int num_sms) {
  const long long b = (work + threads - 1) / threads;
  const long long cap = (long long)num_sms * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int check_partition(const float* base_xy, int N, const float* p, int M, float radius, const int* offsets) {
  if (N < 0 || M < 0) return set_error(GCDF_EINVAL, "negative size (n_waypoints %d, n_points %d)", N, M);
  if (N > 0 && (!base_xy || !al16(base_xy))) return set_error(GCDF_EINVAL, "base_xy NULL or not 16-byte aligned");
  if (M > 0 && (!p || !al16(p))) return set_error(GCDF_EINVAL, "p NULL or not 16-byte aligned");
  if (!offsets || !al16(offsets)) return set_error(GCDF_EINVAL, "part_offsets NULL or not 16-byte aligned");
  if (!(radius >= 0.f)) return set_error(GCDF_EINVAL, "radius must be >= 0 (got %g)", (double)radius);
  return GCDF_OK;
}

}  // namespace

// Partition of `rows` rows with per-row point ranges (planner): counts into
// `counts` (rows), offsets (rows + 1); then the indices.
cudaError_t launch_partition_offsets(const float* base, int bstride, int rows, const float* p, const int* pbegin,
                                     const int* plen, float radius, int* counts, int* offsets, cudaStream_t s) {
  if (rows == 0) return cudaMemsetAsync(offsets, 0, sizeof(int), s);
  const double r2 = (double)radius * (double)radius;
  partition_count_kernel<<<rows, kPartThreads, 0, s>>>(RowRanges{base, bstride, pbegin, plen, 0}, p, r2, counts);
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(counts, rows, offsets);
  return cudaGetLastError();
}

cudaError_t launch_partition_indices(const float* base, int bstride, int rows, const float* p, const int* pbegin,
                                     const int* plen, float radius, const int* offsets, int* idx, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  const double r2 = (double)radius * (double)radius;
  partition_fill_kernel<<<rows, kPartThreads, 0, s>>>(RowRanges{base, bstride, pbegin, plen, 0}, p, r2, offsets, idx);
  return cudaGetLastError();
}

// used by gcdf_project (gcdf_api.cu): the in-place projection of a query's output
cudaError_t launch_project(const float* q, int N, int n, const int* offsets, int M, long long K, const float* f,
                           const float* m_diag, float* g, cudaStream_t s) {
  if (K == 0) return cudaSuccess;
  project_kernel<<<grid_for(K, kRowsPerBlock, sms()), kRowsPerBlock, 0, s>>>(q, N, n, offsets, M, K, f, m_diag, g);
  return cudaGetLastError();
}

}  // namespace gcdf

using namespace gcdf;

extern "C" {

int gcdf_partition_offsets(const float* base_xy, int n_waypoints, const float* p, int n_points, float radius,
                           int* part_offsets, gcdf_stream_t stream) {
  int rc = check_partition(base_xy, n_waypoints, p, n_points, radius, part_offsets);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (n_waypoints == 0) {
    e = cudaMemsetAsync(part_offsets, 0, sizeof(int), s);
    if (e != cudaSuccess) return set_error(GCDF_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    clear_error();
    return GCDF_OK;
  }
  int* counts = nullptr;
  if ((e = cudaMallocAsync((void**)&counts, (size_t)n_waypoints * sizeof(int), s)))
    return set_error(e == cudaErrorMemoryAllocation ? GCDF_ENOMEM : GCDF_ECUDA, "cudaMallocAsync: %s",
                     cudaGetErrorString(e));
  const double r2 = (double)radius * (double)radius;
  partition_count_kernel<<<n_waypoints, kPartThreads, 0, s>>>(RowRanges{base_xy, 2, nullptr, nullptr, n_points}, p,
                                                              r2, counts);
  exclusive_scan_kernel<<<1, 1024, 0, s>>>(counts, n_waypoints, part_offsets);
  e = cudaGetLastError();
  cudaFreeAsync(counts, s);
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "partition launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}

int gcdf_partition_indices(const float* base_xy, int n_waypoints, const float* p, int n_points, float radius,
                           const int* part_offsets, int* part_idx, gcdf_stream_t stream) {
  int rc = check_partition(base_xy, n_waypoints, p, n_points, radius, part_offsets);
  if (rc) return rc;
  if (n_waypoints == 0 || n_points == 0) { clear_error(); return GCDF_OK; }
  if (!part_idx || !al16(part_idx)) return set_error(GCDF_EINVAL, "part_idx NULL or not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const double r2 = (double)radius * (double)radius;
  partition_fill_kernel<<<n_waypoints, kPartThreads, 0, s>>>(RowRanges{base_xy, 2, nullptr, nullptr, n_points}, p,
                                                             r2, part_offsets, part_idx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "partition launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}

int gcdf_jacobian_scatter(const float* grad, int n_waypoints, int n_dof, const int* part_offsets, int n_points,
                          int n_pairs, long long* row_ptr, int* col_idx, float* values, gcdf_stream_t stream) {
  if (n_waypoints < 0 || n_points < 0 || n_pairs < 0 || n_dof < 1 || n_dof > kMaxDof)
    return set_error(GCDF_EINVAL, "bad sizes");
  const long long K = part_offsets ? (long long)n_pairs : (long long)n_waypoints * n_points;
  if ((long long)2 * n_waypoints * n_dof > 0x7fffffffLL) return set_error(GCDF_EINVAL, "2 N n exceeds 2^31 - 1");
  if (!row_ptr || !al16(row_ptr)) return set_error(GCDF_EINVAL, "row_ptr NULL or not 16-byte aligned");
  if (K > 0 && (!col_idx || !al16(col_idx))) return set_error(GCDF_EINVAL, "col_idx NULL or not 16-byte aligned");
  if (K > 0 && values && (!grad || !al16(grad) || !al16(values)))
    return set_error(GCDF_EINVAL, "grad / values NULL or not 16-byte aligned");
  if (part_offsets && !al16(part_offsets)) return set_error(GCDF_EINVAL, "part_offsets not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  jacobian_kernel<<<grid_for(K, kRowsPerBlock, sms()), kRowsPerBlock, 0, s>>>(grad, n_waypoints, n_dof, part_offsets,
                                                                  n_points, K, row_ptr, col_idx, values);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "jacobian launch: %s", cudaGetErrorString(e));
  clear_error();
  return GCDF_OK;
}

}  // extern "C"
