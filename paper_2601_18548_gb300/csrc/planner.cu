// Trajectory optimisation with the GCDF collision cost (Sec. IV-A): the
// cost of Eq. (10) with the velocity controls eliminated through the
// integrator, the l1 penalty of the GCDF rows (Eq. 12), and a fixed number of
// Levenberg-Marquardt steps preconditioned by the exact Hessian of the smooth
// terms.  Every step is one batched HINGE collision-cost pass over all
// trajectories (the fused kernels, on range point lists) and one FP64 update
// launch with one block per trajectory.
//
// The Hessian of the smooth terms over the free waypoints q_2 .. q_N is, for
// every DOF d, tridiagonal with
//   diagonal  4 W_d / dt^2 (interior),  2 W_d / dt^2 + 2 w_goal (last),
//   off-diagonal  -2 W_d / dt^2,
// so the damped system (A_d + lambda diag A_d) s = g is solved per DOF by a
// tridiagonal Cholesky factorisation (one thread per DOF, sequential over
// the waypoints, FP64, reciprocal pivots from rsqrt).
#include <cstring>
#include <vector>

#include "gcdf_internal.cuh"
#include "planner.cuh"

namespace gcdf {

int set_error(int code, const char* fmt, ...);
void clear_error();
int net_n_dof(const gcdf_net* net);
int net_device(const gcdf_net* net);
int collision_ranges(gcdf_net* net, const float* q, int N, const float* p, int M, const int* offsets,
                     const int* point_base, const int* idx, int n_pairs, int reduction, float param, float* cost,
                     float* grad, cudaStream_t s);
cudaError_t launch_partition_offsets(const float* base, int bstride, int rows, const float* p, const int* pbegin,
                                     const int* plen, float radius, int* counts, int* offsets, cudaStream_t s);
cudaError_t launch_partition_indices(const float* base, int bstride, int rows, const float* p, const int* pbegin,
                                     const int* plen, float radius, const int* offsets, int* idx, cudaStream_t s);

namespace {

constexpr int kUpdThreads = 128;
constexpr int kChunk = 64;  // rows per shared-memory chunk of the tridiagonal solve

// Sum over the block in a fixed tree (deterministic for a fixed block size).
__device__ double block_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int m = kUpdThreads / 2; m > 0; m >>= 1) {
    if (t < m) red[t] += red[t + m];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void plan_init_kernel(const PlanTraj* __restrict__ trajs, PlanArrays a, PlanConsts c) {
  const PlanTraj tr = trajs[blockIdx.x];
  const int n = a.n;
  for (int d = threadIdx.x; d < n; d += blockDim.x) tr.goal[d] = (double)tr.q_goal[d];
  float* Qs = a.Qf + (size_t)tr.wp0 * n;
  for (int e = threadIdx.x; e < tr.N * n; e += blockDim.x) {
    const int i = e / n, d = e - i * n;
    double v;
    if (i == 0) {
      v = (double)tr.q_start[d];
    } else if (tr.q_init) {
      v = (double)tr.q_init[(size_t)i * n + d];
    } else {
      const double t = (double)i / (double)(tr.N - 1);
      v = (double)tr.q_start[d] + t * ((double)tr.q_goal[d] - (double)tr.q_start[d]);
    }
    tr.Qm[e] = v;
    tr.Qt[e] = v;
    tr.G[e] = 0.0;
    tr.Qf[e] = (float)v;
    Qs[e] = (float)v;
  }
  if (threadIdx.x == 0) {
    PlanState s;
    s.J = 0.0;
    s.lam = c.lam0;
    s.k = 0;
    s.accepted = 0;
    *tr.st = s;
  }
}

// One evaluation step of one trajectory: merit of the trial (its collision
// terms were just computed), accept or reject, gradient at the new iterate,
// next trial.
__global__ void __launch_bounds__(kUpdThreads) plan_update_kernel(const PlanTraj* __restrict__ trajs,
                                                                  PlanArrays a, PlanConsts c) {
  __shared__ double red[kUpdThreads];
  __shared__ int s_acc;
  __shared__ double s_lam;
  const PlanTraj tr = trajs[blockIdx.x];
  const int n = a.n, N = tr.N, t = threadIdx.x;
  const size_t r0 = (size_t)tr.wp0 * n;
  const double* goal = tr.goal;
  double* Qm = tr.Qm;
  double* Qt = tr.Qt;
  double* G = tr.G;
  double* Ls = tr.Ls;
  float* Qf = tr.Qf;
  float* Qs = a.Qf + r0;
  const float* cc = a.ccost + tr.wp0;
  const float* cg = a.cgrad + r0;

  // merit of the trial: control + tracking terms at the FP64 trial, penalty
  // from the collision costs of its FP32 rounding
  double part = 0.0;
  for (int e = t; e < N * n; e += kUpdThreads) {
    const int i = e / n, d = e - i * n;
    const double W = d < 2 ? c.w_trans : c.w_rot;
    if (i + 1 < N) {
      const double df = Qt[e + n] - Qt[e];
      part += c.dt2inv * W * df * df;
    } else {
      const double eg = Qt[e] - goal[d];
      part += c.w_goal * eg * eg;
    }
    if (d == 0) part += c.mu * (double)cc[i];
  }
  const double Jt = block_sum(part, red);

  if (t == 0) {
    PlanState s = *tr.st;
    const bool acc = (s.k == 0) || (Jt < s.J);
    if (acc) {
      s.J = Jt;
      if (s.k > 0) s.lam = fmax(s.lam * 0.5, c.lam_min);
      s.accepted += (s.k > 0);
    } else {
      s.lam = fmin(s.lam * 4.0, c.lam_max);
    }
    if (a.merit_hist && s.k < a.hist_len) {
      a.merit_hist[(size_t)tr.hist_row * a.hist_len + s.k] = s.J;
      a.acc_hist[(size_t)tr.hist_row * a.hist_len + s.k] = acc ? 1 : 0;
    }
    s.k += 1;
    *tr.st = s;
    s_acc = acc;
    s_lam = s.lam;
  }
  __syncthreads();
  const bool acc = s_acc;
  if (acc) {
    for (int e = t; e < N * n; e += kUpdThreads) Qm[e] = Qt[e];
    __syncthreads();
    // gradient at the new iterate: smooth terms + mu * collision gradient
    for (int e = t; e < N * n; e += kUpdThreads) {
      const int i = e / n, d = e - i * n;
      const double W = d < 2 ? c.w_trans : c.w_rot;
      const double s2 = 2.0 * c.dt2inv * W;
      double g = 0.0;
      if (i + 1 < N) g -= s2 * (Qm[e + n] - Qm[e]);
      if (i > 0) g += s2 * (Qm[e] - Qm[e - n]);
      if (i + 1 == N) g += 2.0 * c.w_goal * (Qm[e] - goal[d]);
      g += c.mu * (double)cg[e];
      G[e] = g;
    }
  }
  __syncthreads();

  // next trial: per DOF, (A_d (1 + lambda)) s = g over q_2 .. q_N by the
  // Cholesky factor with reciprocal pivots r_i = 1 / l_i (one rsqrt per row, no
  // divisions).  The rows go through shared memory in chunks loaded by the
  // whole block, so the per-DOF recurrences never wait on a global load.
  __shared__ double sg[kChunk][kMaxDof], sy[kChunk][kMaxDof], sr[kChunk][kMaxDof];
  const int d = t;
  const double W = d < 2 ? c.w_trans : c.w_rot;
  const double sc = 1.0 + s_lam;
  const double dint = 4.0 * c.dt2inv * W * sc;
  const double dlast = (2.0 * c.dt2inv * W + 2.0 * c.w_goal) * sc;
  const double off = -2.0 * c.dt2inv * W;
  const int m = N - 1;  // unknown rows 1 .. N-1
  // forward: l_i^2 = d_i - e_i^2, e_i = off r_{i-1};  y_i = (g_i - e_i y_{i-1}) r_i
  double rp = 0.0, yp = 0.0;
  for (int c0 = 0; c0 < m; c0 += kChunk) {
    const int cl = min(kChunk, m - c0);
    for (int e = t; e < cl * n; e += kUpdThreads) {
      const int i = e / n, dd = e - i * n;
      sg[i][dd] = G[(size_t)(c0 + i + 1) * n + dd];
    }
    __syncthreads();
    if (d < n) {
      for (int i = 0; i < cl; ++i) {
        const int gi = c0 + i;
        const double di = (gi + 1 == m) ? dlast : dint;
        const double e = (gi == 0) ? 0.0 : off * rp;
        const double r = rsqrt(fma(-e, e, di));
        const double y = fma(-e, yp, sg[i][d]) * r;
        sr[i][d] = r;
        sy[i][d] = y;
        rp = r;
        yp = y;
      }
    }
    __syncthreads();
    for (int e = t; e < cl * n; e += kUpdThreads) {
      const int i = e / n, dd = e - i * n;
      Ls[(size_t)(c0 + i + 1) * n + dd] = sr[i][dd];
      Qt[(size_t)(c0 + i + 1) * n + dd] = sy[i][dd];
    }
    __syncthreads();
  }
  // backward: x_i = (y_i - e_{i+1} x_{i+1}) r_i with e_{i+1} = off r_i; trial = q - x
  double xn = 0.0;
  for (int c1 = m; c1 > 0; c1 -= kChunk) {
    const int c0 = max(0, c1 - kChunk), cl = c1 - c0;
    for (int e = t; e < cl * n; e += kUpdThreads) {
      const int i = e / n, dd = e - i * n;
      sr[i][dd] = Ls[(size_t)(c0 + i + 1) * n + dd];
      sy[i][dd] = Qt[(size_t)(c0 + i + 1) * n + dd];
    }
    __syncthreads();
    if (d < n) {
      for (int i = cl - 1; i >= 0; --i) {
        const double r = sr[i][d];
        const double x = (c0 + i + 1 == m) ? sy[i][d] * r : fma(-off * r, xn, sy[i][d]) * r;
        sy[i][d] = x;
        xn = x;
      }
    }
    __syncthreads();
    for (int e = t; e < cl * n; e += kUpdThreads) {
      const int i = e / n, dd = e - i * n;
      const size_t r = (size_t)(c0 + i + 1) * n + dd;
      const double v = Qm[r] - sy[i][dd];
      Qt[r] = v;
      Qf[r] = (float)v;
      Qs[r] = (float)v;
    }
    __syncthreads();
  }
  if (d < n) {
    Qt[d] = Qm[d];
    Qf[d] = (float)Qm[d];
    Qs[d] = (float)Qm[d];
  }
}

__global__ void plan_output_kernel(const PlanTraj* __restrict__ trajs, int n, float* __restrict__ out,
                                   const int* __restrict__ out_row) {
  const PlanTraj tr = trajs[blockIdx.x];
  const size_t o = (size_t)out_row[blockIdx.x] * n;
  for (int e = threadIdx.x; e < tr.N * n; e += blockDim.x) out[o + e] = (float)tr.Qm[e];
}

}  // namespace

cudaError_t launch_plan_init(const PlanTraj* trajs, int n_traj, const PlanArrays& a, const PlanConsts& c,
                             cudaStream_t s) {
  if (n_traj == 0) return cudaSuccess;
  plan_init_kernel<<<n_traj, kUpdThreads, 0, s>>>(trajs, a, c);
  return cudaGetLastError();
}

cudaError_t launch_plan_update(const PlanTraj* trajs, int n_traj, const PlanArrays& a, const PlanConsts& c,
                               cudaStream_t s) {
  if (n_traj == 0) return cudaSuccess;
  plan_update_kernel<<<n_traj, kUpdThreads, 0, s>>>(trajs, a, c);
  return cudaGetLastError();
}

cudaError_t launch_plan_output(const PlanTraj* trajs, int n_traj, int n, float* out, const int* out_row,
                               cudaStream_t s) {
  if (n_traj == 0) return cudaSuccess;
  plan_output_kernel<<<n_traj, kUpdThreads, 0, s>>>(trajs, n, out, out_row);
  return cudaGetLastError();
}

size_t plan_state_bytes(int N, int n) {
  return (size_t)N * n * (5 * sizeof(double) + sizeof(float)) + (size_t)n * sizeof(double) + sizeof(PlanState) + 256;
}

int check_plan_params(const gcdf_plan_params* p) {
  if (!p) return set_error(GCDF_EINVAL, "params is NULL");
  if (!(p->dt > 0.f) || !(p->w_trans > 0.f) || !(p->w_rot > 0.f) || !(p->w_goal >= 0.f) || !(p->mu >= 0.f) ||
      !(p->delta == p->delta) || !(p->lambda0 >= 0.f) || !(p->lambda_min >= 0.f) ||
      !(p->lambda_max >= p->lambda_min) || p->iterations < 0 || !(p->partition_radius >= 0.f))
    return set_error(GCDF_EINVAL, "bad planner parameters");
  return GCDF_OK;
}

PlanConsts plan_consts(const gcdf_plan_params* p) {
  PlanConsts c;
  c.dt2inv = 1.0 / ((double)p->dt * (double)p->dt);
  c.w_trans = p->w_trans;
  c.w_rot = p->w_rot;
  c.w_goal = p->w_goal;
  c.mu = p->mu;
  c.lam0 = p->lambda0;
  c.lam_min = p->lambda_min;
  c.lam_max = p->lambda_max;
  return c;
}

int plan_partition(const float* base, int bstride, int rows, const float* points, const int* pbegin,
                   const int* plen, float radius, int* offsets, int** idx, long long* n_pairs, cudaStream_t s) {
  cudaError_t e;
  int* counts = nullptr;
  if ((e = lib_malloc_async((void**)&counts, (size_t)(rows > 0 ? rows : 1) * sizeof(int), s)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  e = launch_partition_offsets(base, bstride, rows, points, pbegin, plen, radius, counts, offsets, s);
  cudaFreeAsync(counts, s);
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "partition launch: %s", cudaGetErrorString(e));
  int total = 0;
  if ((e = cudaMemcpyAsync(&total, offsets + rows, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return set_error(GCDF_ECUDA, "partition read-back: %s", cudaGetErrorString(e));
  if ((e = lib_malloc_async((void**)idx, (size_t)(total > 0 ? total : 1) * sizeof(int), s)))
    return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
  if ((e = launch_partition_indices(base, bstride, rows, points, pbegin, plen, radius, offsets, *idx, s)))
    return set_error(GCDF_ECUDA, "partition launch: %s", cudaGetErrorString(e));
  *n_pairs = total;
  return GCDF_OK;
}

int plan_step(gcdf_net* net, const PlanStep& ps, const PlanArrays& a, const PlanConsts& c, float delta,
              cudaStream_t s) {
  int rc = collision_ranges(net, a.Qf, ps.n_rows, ps.points, ps.n_points, ps.offsets, ps.point_base, ps.idx,
                            ps.n_pairs, GCDF_RED_HINGE, delta, const_cast<float*>(a.ccost), const_cast<float*>(a.cgrad), s);
  if (rc) return rc;
  cudaError_t e = launch_plan_update(ps.trajs, ps.n_traj, a, c, s);
  if (e != cudaSuccess) return set_error(GCDF_ECUDA, "plan update launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

}  // namespace gcdf

using namespace gcdf;

namespace {

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  cudaError_t get(T** out, size_t count) {
    size_t bytes = count * sizeof(T);
    cudaError_t e = lib_malloc_async((void**)out, bytes < 16 ? 16 : bytes, s);
    if (e == cudaSuccess) ptrs.push_back(*out);
    return e;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

}  // namespace

namespace {

// Problems [0, n_problems) of a batch whose pair count fits one collision pass.
int solve_chunk(gcdf_net* net, const gcdf_plan_problem* problems, int n_problems, const gcdf_plan_params* params,
                float* q_out, double* merit_out, unsigned char* accepted_out, gcdf_stream_t stream) {
  int rc = GCDF_OK;
  const int n = net_n_dof(net);
  long long rows = 0, pts = 0, pairs = 0;
  for (int r = 0; r < n_problems; ++r) {
    rows += problems[r].n_waypoints;
    pts += problems[r].n_points;
    pairs += (long long)problems[r].n_waypoints * problems[r].n_points;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  cudaError_t e;
  const size_t rn = (size_t)rows * n;
  double *Qm, *Qt, *G, *Ls, *goal;
  float *Qf, *Qs, *ccost, *cgrad, *P;
  int *offsets, *pbase, *orow;
  PlanTraj* trajs;
  PlanState* st;
  if ((e = sc.get(&Qm, rn)) || (e = sc.get(&Qt, rn)) || (e = sc.get(&G, rn)) || (e = sc.get(&Ls, rn)) ||
      (e = sc.get(&goal, (size_t)n_problems * n)) || (e = sc.get(&Qf, rn)) || (e = sc.get(&Qs, rn)) ||
      (e = sc.get(&ccost, (size_t)rows)) || (e = sc.get(&cgrad, rn)) || (e = sc.get(&P, (size_t)pts * 3)) ||
      (e = sc.get(&offsets, (size_t)rows + 1)) || (e = sc.get(&pbase, (size_t)rows)) ||
      (e = sc.get(&orow, (size_t)n_problems)) || (e = sc.get(&trajs, (size_t)n_problems)) ||
      (e = sc.get(&st, (size_t)n_problems)))
    return set_error(e == cudaErrorMemoryAllocation ? GCDF_ENOMEM : GCDF_ECUDA, "cudaMallocAsync: %s",
                     cudaGetErrorString(e));
  std::vector<int> h_off((size_t)rows + 1), h_pb((size_t)rows), h_orow(n_problems);
  std::vector<PlanTraj> h_tr(n_problems);
  long long row = 0, pt = 0;
  h_off[0] = 0;
  for (int r = 0; r < n_problems; ++r) {
    const gcdf_plan_problem& pr = problems[r];
    PlanTraj& t = h_tr[r];
    memset(&t, 0, sizeof(t));
    t.wp0 = (int)row;
    t.N = pr.n_waypoints;
    t.hist_row = r;
    t.st = st + r;
    const size_t o = (size_t)row * n;
    t.Qm = Qm + o;
    t.Qt = Qt + o;
    t.G = G + o;
    t.Ls = Ls + o;
    t.Qf = Qf + o;
    t.goal = goal + (size_t)r * n;
    t.q_start = pr.q_start;
    t.q_goal = pr.q_goal;
    t.q_init = pr.q_init;
    h_orow[r] = (int)row;
    for (int i = 0; i < pr.n_waypoints; ++i) {
      h_off[row + i + 1] = h_off[row + i] + pr.n_points;
      h_pb[row + i] = (int)pt;
    }
    if (pr.n_points > 0 &&
        (e = cudaMemcpyAsync(P + pt * 3, pr.points, (size_t)pr.n_points * 12, cudaMemcpyDeviceToDevice, s)))
      return set_error(GCDF_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
    row += pr.n_waypoints;
    pt += pr.n_points;
  }
  if ((e = cudaMemcpyAsync(offsets, h_off.data(), h_off.size() * sizeof(int), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(pbase, h_pb.data(), h_pb.size() * sizeof(int), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(orow, h_orow.data(), h_orow.size() * sizeof(int), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(trajs, h_tr.data(), h_tr.size() * sizeof(PlanTraj), cudaMemcpyHostToDevice, s)))
    return set_error(GCDF_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
  PlanArrays a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.Qf = Qs;
  a.ccost = ccost;
  a.cgrad = cgrad;
  a.merit_hist = merit_out;
  a.acc_hist = accepted_out;
  a.hist_len = params->iterations + 1;
  const PlanConsts c = plan_consts(params);
  if ((e = launch_plan_init(trajs, n_problems, a, c, s)))
    return set_error(GCDF_ECUDA, "plan init launch: %s", cudaGetErrorString(e));
  PlanStep ps;
  ps.trajs = trajs;
  ps.n_traj = n_problems;
  ps.n_rows = (int)rows;
  ps.points = P;
  ps.n_points = (int)pts;
  ps.offsets = offsets;
  ps.point_base = pbase;
  ps.idx = nullptr;
  ps.n_pairs = (int)pairs;
  int* part_idx = nullptr;
  if (params->partition_radius > 0.f) {
    // lists around the reference bases: the (x, y) of the initial guess, which
    // the init kernel has just written (FP32) to the step rows
    std::vector<int> h_len((size_t)rows);
    for (long long i = 0; i < rows; ++i) h_len[i] = h_off[i + 1] - h_off[i];
    int *plen = nullptr, *poff = nullptr;
    if ((e = sc.get(&plen, (size_t)rows)) || (e = sc.get(&poff, (size_t)rows + 1)))
      return set_error(GCDF_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpyAsync(plen, h_len.data(), h_len.size() * sizeof(int), cudaMemcpyHostToDevice, s)))
      return set_error(GCDF_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
    long long np = 0;
    if ((rc = plan_partition(Qs, n, (int)rows, P, pbase, plen, params->partition_radius, poff, &part_idx, &np, s)))
      return rc;
    sc.ptrs.push_back(part_idx);
    ps.offsets = poff;
    ps.idx = part_idx;
    ps.n_pairs = (int)np;
  }
  for (int k = 0; k <= params->iterations; ++k) {
    if ((rc = plan_step(net, ps, a, c, params->delta, s))) return rc;
  }
  if ((e = launch_plan_output(trajs, n_problems, n, q_out, orow, s)))
    return set_error(GCDF_ECUDA, "plan output launch: %s", cudaGetErrorString(e));
  return GCDF_OK;
}

}  // namespace

extern "C" int gcdf_plan_solve(gcdf_net* net, const gcdf_plan_problem* problems, int n_problems,
                               const gcdf_plan_params* params, float* q_out, double* merit_out,
                               unsigned char* accepted_out, gcdf_stream_t stream) {
  if (!net) return set_error(GCDF_EINVAL, "net is NULL");
  int rc = check_plan_params(params);
  if (rc) return rc;
  if (n_problems < 0 || (n_problems > 0 && !problems)) return set_error(GCDF_EINVAL, "bad problem list");
  if (n_problems == 0) { clear_error(); return GCDF_OK; }
  if (!q_out || !al16(q_out)) return set_error(GCDF_EINVAL, "q_out NULL or not 16-byte aligned");
  if ((merit_out == nullptr) != (accepted_out == nullptr))
    return set_error(GCDF_EINVAL, "give both merit_out and accepted_out or neither");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != net_device(net)) return set_error(GCDF_EINVAL, "net belongs to device %d, current device is %d",
                                               net_device(net), dev);
  const int n = net_n_dof(net);
  const long long kLim = 0x7fffffffLL;
  for (int r = 0; r < n_problems; ++r) {
    const gcdf_plan_problem& pr = problems[r];
    if (pr.n_waypoints < 2) return set_error(GCDF_EINVAL, "problem %d: n_waypoints %d < 2", r, pr.n_waypoints);
    if (pr.n_points < 0) return set_error(GCDF_EINVAL, "problem %d: n_points < 0", r);
    if (!pr.q_start || !pr.q_goal) return set_error(GCDF_EINVAL, "problem %d: q_start / q_goal NULL", r);
    if (pr.n_points > 0 && (!pr.points || !al16(pr.points)))
      return set_error(GCDF_EINVAL, "problem %d: points NULL or not 16-byte aligned", r);
    if ((long long)pr.n_waypoints * pr.n_points > kLim)
      return set_error(GCDF_EINVAL, "problem %d has more than 2^31 - 1 pairs", r);
  }
  // consecutive chunks of problems whose pairs, points and rows each stay below
  // 2^31: one collision pass per step and chunk (problems are independent, so
  // the chunking changes no result)
  const int hl = params->iterations + 1;
  int r0 = 0;
  long long row0 = 0;
  while (r0 < n_problems) {
    long long cr = 0, cp = 0, cq = 0;
    int r1 = r0;
    while (r1 < n_problems) {
      const gcdf_plan_problem& pr = problems[r1];
      const long long q = (long long)pr.n_waypoints * pr.n_points;
      if (r1 > r0 && (cq + q > kLim || cp + pr.n_points > kLim || cr + pr.n_waypoints > kLim)) break;
      cr += pr.n_waypoints;
      cp += pr.n_points;
      cq += q;
      ++r1;
    }
    rc = solve_chunk(net, problems + r0, r1 - r0, params, q_out + row0 * n,
                     merit_out ? merit_out + (size_t)r0 * hl : nullptr,
                     accepted_out ? accepted_out + (size_t)r0 * hl : nullptr, stream);
    if (rc) return rc;
    row0 += cr;
    r0 = r1;
  }
  clear_error();
  return GCDF_OK;
}
