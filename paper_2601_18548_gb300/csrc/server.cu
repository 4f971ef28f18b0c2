// Planning server (gcdf_server_*, gcdf_plan_submit / gcdf_plan_poll): a host
// thread that runs the trajectory optimiser of planner.cu for every admitted
// request with continuous batching.
//
// Loop of the worker thread, one optimiser step per pass:
//   1. admission — waiting requests, first come first admitted, while a slot
//      and the device-memory budget allow: device copies of the inputs, state
//      arrays, one init launch;
//   2. when the admitted set changed, the step arrays of every net group (the
//      rows of all its trajectories back to back, their points, the range
//      lists) are rebuilt;
//   3. one step per group: the batched collision pass and the FP64 update;
//   4. after the step completes on the device, requests that made all their
//      evaluations are read back and release their memory.
// A request's trajectory is computed by the same launches whatever else is
// admitted with it, and every quantity of one trajectory depends only on its
// own rows (the fused kernels merge each waypoint's tiles in a fixed order),
// so its result does not depend on the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gcdf_internal.cuh"
#include "planner.cuh"

namespace gcdf {
int set_error(int code, const char* fmt, ...);
void clear_error();
int net_n_dof(const gcdf_net* net);
int net_device(const gcdf_net* net);
size_t net_step_bytes_per_row(const gcdf_net* net, int n_points);
}  // namespace gcdf

using namespace gcdf;

namespace {

struct Req {
  uint64_t ticket = 0;
  gcdf_net* net = nullptr;
  int N = 0, M = 0, n = 0;
  std::vector<float> qs, qg, pts;
  double t_submit = 0, t_admit = 0, t_done = 0;
  size_t bytes = 0;   // counted against the budget while admitted
  int k = 0;          // evaluations done
  // device memory (one block, carved)
  void* dmem = nullptr;
  PlanTraj tr{};      // host image of its table entry (wp0 set per rebuild)
  float* d_pts = nullptr;
  float* d_ref = nullptr;  // the initial trajectory (FP32): reference bases of the partition
  // result
  std::vector<float> q;
  double merit = 0;
  int accepted = 0;
};

struct Group {        // admitted requests that share a net
  gcdf_net* net = nullptr;
  std::vector<Req*> reqs;
  // step arrays
  void* dmem = nullptr;
  PlanTraj* trajs = nullptr;
  PlanArrays a{};
  PlanStep ps{};
  int* part_idx = nullptr;  // partition lists of the step (with partition_radius > 0)
  int* part_off = nullptr;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct gcdf_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  gcdf_server_desc desc{};
  PlanConsts consts{};
  std::chrono::steady_clock::time_point t0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  int fail_code = GCDF_OK;
  char fail_msg[256] = "";
  uint64_t next_ticket = 1;
  size_t used = 0;
  std::deque<std::unique_ptr<Req>> queue;   // waiting
  std::vector<std::unique_ptr<Req>> active; // admitted (worker only touches device parts)
  std::map<uint64_t, std::unique_ptr<Req>> done;
  std::vector<Group> groups;                // worker thread only
  bool dirty = false;                       // worker thread only
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;  // around each step's launches (worker thread only)
  gcdf_server_stats stats{};                // under mu

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Device bytes a request holds while admitted: its points, its persistent
// state, its rows of the step arrays and the fused pass's per-row temporaries.
size_t request_bytes(const gcdf_net* net, int N, int M, int n) {
  const size_t state = plan_state_bytes(N, n);
  const size_t pts = (size_t)M * 12 * 2 + (size_t)N * n * 4;  // own copy + step copy, reference trajectory
  const size_t rows = (size_t)N * (2 * n * 4 + 4 + 8);  // step Qf, cgrad, ccost, offsets, base
  const size_t pass = (size_t)N * net_step_bytes_per_row(net, M);
  return align256(state) + align256(pts) + rows + pass + 3 * 256;
}

int fail_server(gcdf_server* s, int code, const char* what, cudaError_t e) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fail_code == GCDF_OK) {
    s->fail_code = code;
    snprintf(s->fail_msg, sizeof(s->fail_msg), "%s: %s", what, e == cudaSuccess ? "" : cudaGetErrorString(e));
  }
  return code;
}

// Device copies and state for a newly admitted request; one init launch.
int admit(gcdf_server* s, Req* r) {
  const int n = r->n, N = r->N;
  const size_t b_state = align256(plan_state_bytes(N, n));
  const size_t b_in = align256((size_t)(2 * n) * 4) + align256((size_t)r->M * 12) + align256((size_t)N * n * 4);
  cudaError_t e = lib_malloc_async(&r->dmem, b_state + b_in + 256, s->stream);
  if (e != cudaSuccess) return fail_server(s, GCDF_ENOMEM, "cudaMallocAsync", e);
  char* p = (char*)r->dmem;
  PlanTraj& t = r->tr;
  memset(&t, 0, sizeof(t));
  t.N = N;
  t.hist_row = 0;
  t.Qm = (double*)p; p += (size_t)N * n * 8;
  t.Qt = (double*)p; p += (size_t)N * n * 8;
  t.G = (double*)p; p += (size_t)N * n * 8;
  t.Ls = (double*)p; p += (size_t)N * n * 8;
  t.goal = (double*)p; p += (size_t)n * 8;
  t.Qf = (float*)p; p += (size_t)N * n * 4;
  p = (char*)r->dmem + align256((size_t)(p - (char*)r->dmem));
  t.st = (PlanState*)p; p += 256;
  p = (char*)r->dmem + b_state;
  float* qsg = (float*)p;
  t.q_start = qsg;
  t.q_goal = qsg + n;
  t.q_init = nullptr;
  p += align256((size_t)(2 * n) * 4);
  r->d_pts = (float*)p;
  p += align256((size_t)r->M * 12);
  r->d_ref = (float*)p;
  if ((e = cudaMemcpyAsync(qsg, r->qs.data(), n * 4, cudaMemcpyHostToDevice, s->stream)) ||
      (e = cudaMemcpyAsync(qsg + n, r->qg.data(), n * 4, cudaMemcpyHostToDevice, s->stream)) ||
      (r->M > 0 && (e = cudaMemcpyAsync(r->d_pts, r->pts.data(), (size_t)r->M * 12, cudaMemcpyHostToDevice,
                                        s->stream))))
    return fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
  r->k = 0;
  return GCDF_OK;
}

void free_group(gcdf_server* s, Group& g) {
  if (g.dmem) cudaFreeAsync(g.dmem, s->stream);
  if (g.part_idx) cudaFreeAsync(g.part_idx, s->stream);
  if (g.part_off) cudaFreeAsync(g.part_off, s->stream);
  g.dmem = nullptr;
  g.part_idx = nullptr;
  g.part_off = nullptr;
}

// Step arrays of one group: rows of all its trajectories back to back.
int build_group(gcdf_server* s, Group& g, const gcdf_plan_params& prm) {
  const int n = net_n_dof(g.net);
  long long rows = 0, pts = 0, pairs = 0;
  for (Req* r : g.reqs) {
    rows += r->N;
    pts += r->M;
    pairs += (long long)r->N * r->M;
  }
  const size_t b_tr = align256(g.reqs.size() * sizeof(PlanTraj));
  const size_t b_qf = align256((size_t)rows * n * 4), b_cg = b_qf, b_cc = align256((size_t)rows * 4);
  const size_t b_p = align256((size_t)pts * 12), b_off = align256((size_t)(rows + 1) * 4), b_pb = b_cc;
  cudaError_t e = lib_malloc_async(&g.dmem, b_tr + b_qf + b_cg + b_cc + b_p + b_off + b_pb, s->stream);
  if (e != cudaSuccess) return fail_server(s, GCDF_ENOMEM, "cudaMallocAsync", e);
  char* p = (char*)g.dmem;
  g.trajs = (PlanTraj*)p; p += b_tr;
  float* Qs = (float*)p; p += b_qf;
  float* cg = (float*)p; p += b_cg;
  float* cc = (float*)p; p += b_cc;
  float* P = (float*)p; p += b_p;
  int* off = (int*)p; p += b_off;
  int* pb = (int*)p;
  std::vector<PlanTraj> h_tr;
  std::vector<int> h_off(1, 0), h_pb;
  long long row = 0, pt = 0;
  for (Req* r : g.reqs) {
    r->tr.wp0 = (int)row;
    h_tr.push_back(r->tr);
    for (int i = 0; i < r->N; ++i) {
      h_off.push_back(h_off.back() + r->M);
      h_pb.push_back((int)pt);
    }
    if (r->M > 0 &&
        (e = cudaMemcpyAsync(P + pt * 3, r->d_pts, (size_t)r->M * 12, cudaMemcpyDeviceToDevice, s->stream)))
      return fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
    // the trajectory's current trial (FP32) into its new rows
    if ((e = cudaMemcpyAsync(Qs + row * n, r->tr.Qf, (size_t)r->N * n * 4, cudaMemcpyDeviceToDevice, s->stream)))
      return fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
    row += r->N;
    pt += r->M;
  }
  if ((e = cudaMemcpyAsync(g.trajs, h_tr.data(), h_tr.size() * sizeof(PlanTraj), cudaMemcpyHostToDevice, s->stream)) ||
      (e = cudaMemcpyAsync(off, h_off.data(), h_off.size() * 4, cudaMemcpyHostToDevice, s->stream)) ||
      (e = cudaMemcpyAsync(pb, h_pb.data(), h_pb.size() * 4, cudaMemcpyHostToDevice, s->stream)))
    return fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
  memset(&g.a, 0, sizeof(g.a));
  g.a.Qf = Qs;
  g.a.ccost = cc;
  g.a.cgrad = cg;
  g.a.hist_len = prm.iterations + 1;
  g.a.n = n;
  g.ps.trajs = g.trajs;
  g.ps.n_traj = (int)g.reqs.size();
  g.ps.n_rows = (int)rows;
  g.ps.points = P;
  g.ps.n_points = (int)pts;
  g.ps.offsets = off;
  g.ps.point_base = pb;
  g.ps.idx = nullptr;
  g.ps.n_pairs = (int)pairs;
  if (prm.partition_radius > 0.f) {
    // the reference bases of every row (each request's initial trajectory) and
    // each row's point count, then the lists over the rows' point ranges
    float* base = nullptr;
    int* plen = nullptr;
    if ((e = lib_malloc_async(&base, (size_t)(rows > 0 ? rows : 1) * n * 4, s->stream)) ||
        (e = lib_malloc_async(&plen, (size_t)(rows > 0 ? rows : 1) * 4, s->stream)) ||
        (e = lib_malloc_async(&g.part_off, (size_t)(rows + 1) * 4, s->stream)))
      return fail_server(s, GCDF_ENOMEM, "cudaMallocAsync", e);
    std::vector<int> h_len;
    long long r0 = 0;
    for (Req* r : g.reqs) {
      if ((e = cudaMemcpyAsync(base + r0 * n, r->d_ref, (size_t)r->N * n * 4, cudaMemcpyDeviceToDevice, s->stream)))
        return fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
      for (int i = 0; i < r->N; ++i) h_len.push_back(r->M);
      r0 += r->N;
    }
    if ((e = cudaMemcpyAsync(plen, h_len.data(), h_len.size() * 4, cudaMemcpyHostToDevice, s->stream)))
      return fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
    long long np = 0;
    const int rc = plan_partition(base, n, (int)rows, P, pb, plen, prm.partition_radius, g.part_off, &g.part_idx, &np,
                                  s->stream);
    cudaFreeAsync(base, s->stream);
    cudaFreeAsync(plen, s->stream);
    if (rc) return fail_server(s, rc, "partition", cudaGetLastError());
    g.ps.offsets = g.part_off;
    g.ps.idx = g.part_idx;
    g.ps.n_pairs = (int)np;
  }
  return GCDF_OK;
}

void worker_loop(gcdf_server* s) {
  cudaSetDevice(s->device);
  const gcdf_plan_params prm = s->desc.params;
  const int evals = prm.iterations + 1;
  std::vector<Req*> fresh;
  auto pass_start = std::chrono::steady_clock::now();
  bool stepped = false;
  for (;;) {
    {
      const auto now = std::chrono::steady_clock::now();
      if (stepped) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.pass_s += std::chrono::duration<double>(now - pass_start).count();
      }
      pass_start = now;
      stepped = false;
    }
    fresh.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop || s->fail_code) break;
      // 1. admission, first come first admitted
      while (!s->queue.empty() && (int)s->active.size() < s->desc.max_active &&
             s->used + s->queue.front()->bytes <= s->desc.hbm_budget_bytes) {
        std::unique_ptr<Req> r = std::move(s->queue.front());
        s->queue.pop_front();
        s->used += r->bytes;
        r->t_admit = s->now();
        fresh.push_back(r.get());
        s->active.push_back(std::move(r));
      }
      if (s->active.empty()) {
        s->cv.wait_for(lk, std::chrono::milliseconds(50));
        continue;
      }
    }
    for (Req* r : fresh) {
      if (admit(s, r)) return;
      // one init launch per admitted request (a one-entry table)
      PlanTraj* d_tr = nullptr;
      cudaError_t e = lib_malloc_async(&d_tr, sizeof(PlanTraj), s->stream);
      if (e != cudaSuccess) { fail_server(s, GCDF_ENOMEM, "cudaMallocAsync", e); return; }
      if ((e = cudaMemcpyAsync(d_tr, &r->tr, sizeof(PlanTraj), cudaMemcpyHostToDevice, s->stream))) {
        fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
        return;
      }
      // the init kernel also writes the step rows (row wp0 = 0 of a0.Qf): point
      // them at the persistent copy, from which the rebuild below copies
      PlanArrays a0{};
      a0.Qf = r->tr.Qf;
      a0.n = r->n;
      if ((e = launch_plan_init(d_tr, 1, a0, s->consts, s->stream))) {
        fail_server(s, GCDF_ECUDA, "plan init launch", e);
        return;
      }
      cudaFreeAsync(d_tr, s->stream);
      // the initial trajectory, whose (x, y) are the partition's reference bases
      if ((e = cudaMemcpyAsync(r->d_ref, r->tr.Qf, (size_t)r->N * r->n * 4, cudaMemcpyDeviceToDevice, s->stream))) {
        fail_server(s, GCDF_ECUDA, "cudaMemcpyAsync", e);
        return;
      }
      s->dirty = true;
    }
    // 2. step arrays
    if (s->dirty) {
      for (Group& g : s->groups) free_group(s, g);
      s->groups.clear();
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& up : s->active) {
          Req* r = up.get();
          auto it = std::find_if(s->groups.begin(), s->groups.end(), [&](const Group& g) { return g.net == r->net; });
          if (it == s->groups.end()) {
            s->groups.emplace_back();
            s->groups.back().net = r->net;
            it = s->groups.end() - 1;
          }
          it->reqs.push_back(r);
        }
      }
      for (Group& g : s->groups)
        if (build_group(s, g, prm)) return;
      s->dirty = false;
    }
    // 3. one step per group; host time from the first launch to the return of
    // the synchronisation against the device time between two events
    const auto h0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaEventRecord(s->ev_a, s->stream);
    if (e != cudaSuccess) { fail_server(s, GCDF_ECUDA, "cudaEventRecord", e); return; }
    for (Group& g : s->groups) {
      const int rc = plan_step(g.net, g.ps, g.a, s->consts, prm.delta, s->stream);
      if (rc) { fail_server(s, rc, "plan step", cudaGetLastError()); return; }
    }
    if ((e = cudaEventRecord(s->ev_b, s->stream)) != cudaSuccess) { fail_server(s, GCDF_ECUDA, "cudaEventRecord", e); return; }
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) { fail_server(s, GCDF_ECUDA, "step", e); return; }
    {
      const double host_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - h0).count();
      float dev_ms = 0.f;
      cudaEventElapsedTime(&dev_ms, s->ev_a, s->ev_b);
      std::lock_guard<std::mutex> lk(s->mu);
      s->stats.steps += 1;
      s->stats.step_host_s += host_s;
      s->stats.step_device_s += 1e-3 * dev_ms;
      s->stats.active_sum += (uint64_t)s->active.size();
    }
    stepped = true;
    // 4. finished requests
    std::vector<Req*> fin;
    for (auto& up : s->active)
      if (++up->k == evals) fin.push_back(up.get());
    for (Req* r : fin) {
      std::vector<double> qd((size_t)r->N * r->n);
      PlanState st{};
      if ((e = cudaMemcpy(qd.data(), r->tr.Qm, qd.size() * 8, cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(&st, r->tr.st, sizeof(st), cudaMemcpyDeviceToHost))) {
        fail_server(s, GCDF_ECUDA, "cudaMemcpy", e);
        return;
      }
      r->q.resize(qd.size());
      for (size_t i = 0; i < qd.size(); ++i) r->q[i] = (float)qd[i];
      r->merit = st.J;
      r->accepted = st.accepted;
      cudaFreeAsync(r->dmem, s->stream);
      r->dmem = nullptr;
    }
    if (!fin.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      for (Req* r : fin) {
        auto it = std::find_if(s->active.begin(), s->active.end(), [&](const std::unique_ptr<Req>& u) { return u.get() == r; });
        std::unique_ptr<Req> up = std::move(*it);
        s->active.erase(it);
        s->used -= up->bytes;
        up->t_done = s->now();
        up->pts.clear();
        up->pts.shrink_to_fit();
        s->done[up->ticket] = std::move(up);
      }
      s->dirty = true;
    }
  }
}

}  // namespace

extern "C" {

int gcdf_server_create(const gcdf_server_desc* desc, gcdf_server** out) {
  if (!desc || !out) return set_error(GCDF_EINVAL, "desc or out is NULL");
  int rc = check_plan_params(&desc->params);
  if (rc) return rc;
  if (desc->max_active < 1 || desc->max_queued < 0 || desc->hbm_budget_bytes == 0)
    return set_error(GCDF_EINVAL, "bad server descriptor (max_active %d, max_queued %d, budget %zu)",
                     desc->max_active, desc->max_queued, desc->hbm_budget_bytes);
  gcdf_server* s = new (std::nothrow) gcdf_server();
  if (!s) return set_error(GCDF_ENOMEM, "host allocation failed");
  s->desc = *desc;
  s->consts = plan_consts(&desc->params);
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_a);
  if (e == cudaSuccess) e = cudaEventCreate(&s->ev_b);
  if (e != cudaSuccess) {
    if (s->ev_a) cudaEventDestroy(s->ev_a);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return set_error(GCDF_ECUDA, "server stream: %s", cudaGetErrorString(e));
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  clear_error();
  return GCDF_OK;
}

int gcdf_plan_submit(gcdf_server* s, const gcdf_plan_request* rq, uint64_t* ticket) {
  if (!s || !rq || !ticket) return set_error(GCDF_EINVAL, "server, request or ticket is NULL");
  if (!rq->net) return set_error(GCDF_EINVAL, "request net is NULL");
  if (net_device(rq->net) != s->device) return set_error(GCDF_EINVAL, "net and server are on different devices");
  if (rq->n_waypoints < 2) return set_error(GCDF_EINVAL, "n_waypoints %d < 2", rq->n_waypoints);
  if (rq->n_points < 0 || (rq->n_points > 0 && !rq->points)) return set_error(GCDF_EINVAL, "bad points");
  if (!rq->q_start || !rq->q_goal) return set_error(GCDF_EINVAL, "q_start / q_goal NULL");
  if ((long long)rq->n_waypoints * rq->n_points > 0x7fffffffLL)
    return set_error(GCDF_EINVAL, "request has more than 2^31 - 1 pairs");
  const int n = net_n_dof(rq->net);
  std::unique_ptr<Req> r(new (std::nothrow) Req());
  if (!r) return set_error(GCDF_ENOMEM, "host allocation failed");
  r->net = rq->net;
  r->N = rq->n_waypoints;
  r->M = rq->n_points;
  r->n = n;
  r->bytes = request_bytes(rq->net, r->N, r->M, n);
  if (r->bytes > s->desc.hbm_budget_bytes)
    return set_error(GCDF_EINVAL, "request needs %zu bytes, budget is %zu", r->bytes, s->desc.hbm_budget_bytes);
  r->qs.assign(rq->q_start, rq->q_start + n);
  r->qg.assign(rq->q_goal, rq->q_goal + n);
  r->pts.assign(rq->points, rq->points + (size_t)r->M * 3);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fail_code) return set_error(s->fail_code, "server failed: %s", s->fail_msg);
    if ((int)s->queue.size() >= s->desc.max_queued) return set_error(GCDF_EAGAIN, "queue full (%d waiting)", (int)s->queue.size());
    r->ticket = s->next_ticket++;
    r->t_submit = s->now();
    *ticket = r->ticket;
    s->queue.push_back(std::move(r));
  }
  s->cv.notify_one();
  clear_error();
  return GCDF_OK;
}

int gcdf_plan_poll(gcdf_server* s, uint64_t ticket, gcdf_plan_result* res) {
  if (!s || !res) return set_error(GCDF_EINVAL, "server or result is NULL");
  std::unique_ptr<Req> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
      const bool waiting = std::any_of(s->queue.begin(), s->queue.end(), [&](const std::unique_ptr<Req>& u) { return u->ticket == ticket; });
      const bool running = std::any_of(s->active.begin(), s->active.end(), [&](const std::unique_ptr<Req>& u) { return u->ticket == ticket; });
      if (s->fail_code) return set_error(s->fail_code, "server failed: %s", s->fail_msg);
      if (waiting || running) { clear_error(); return GCDF_PENDING; }
      return set_error(GCDF_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    }
    r = std::move(it->second);
    s->done.erase(it);
  }
  if (res->q) memcpy(res->q, r->q.data(), r->q.size() * sizeof(float));
  res->merit = r->merit;
  res->accepted_steps = r->accepted;
  res->submit_s = r->t_submit;
  res->admit_s = r->t_admit;
  res->done_s = r->t_done;
  clear_error();
  return GCDF_OK;
}

double gcdf_server_clock(gcdf_server* s) { return s ? s->now() : 0.0; }

int gcdf_server_stats_get(gcdf_server* s, gcdf_server_stats* out) {
  if (!s || !out) return set_error(GCDF_EINVAL, "server or out is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  clear_error();
  return GCDF_OK;
}

size_t gcdf_plan_request_bytes(gcdf_net* net, int n_waypoints, int n_points) {
  if (!net || n_waypoints < 0 || n_points < 0) return 0;
  return request_bytes(net, n_waypoints, n_points, net_n_dof(net));
}

int gcdf_server_destroy(gcdf_server* s) {
  if (!s) return GCDF_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (Group& g : s->groups) free_group(s, g);
  for (auto& r : s->active)
    if (r->dmem) cudaFreeAsync(r->dmem, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaEventDestroy(s->ev_a);
  cudaEventDestroy(s->ev_b);
  cudaStreamDestroy(s->stream);
  delete s;
  return GCDF_OK;
}

}  // extern "C"
