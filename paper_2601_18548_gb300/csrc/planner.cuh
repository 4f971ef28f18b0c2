// Internal declarations of the trajectory optimiser (planner.cu) shared with
// the planning server (server.cu).
#pragma once

#include "gcdf_internal.cuh"

namespace gcdf {

// Per-trajectory scalars, kept across steps.
struct PlanState {
  double J;               // merit of the current iterate
  double lam;             // damping for the next step
  int k;                  // evaluations done
  int accepted;           // accepted trials
};

// One trajectory of a step (device table entry).  Its state arrays (N rows of
// n values each) persist across steps; its rows of the step arrays (the
// collision pass's input and outputs) start at row wp0.
struct PlanTraj {
  int wp0;                // first row in the step arrays
  int N;                  // waypoints
  int hist_row;           // row of the merit / accepted history (if recorded)
  int pad;
  PlanState* st;
  double* Qm;             // current iterate
  double* Qt;             // trial (also the forward-substitution scratch)
  double* G;              // gradient of J at the current iterate
  double* Ls;             // Cholesky factor scratch
  double* goal;           // (n)
  float* Qf;              // trial rounded to FP32 (persistent copy)
  const float* q_start;   // (n) device, read by the init kernel only
  const float* q_goal;    // (n) device, read by the init kernel only
  const float* q_init;    // (N, n) device or nullptr (straight line)
};

// Arrays of one step, rows of all its trajectories back to back.
struct PlanArrays {
  float* Qf;              // trials rounded to FP32: the field's input
  const float* ccost;     // collision cost of every row (HINGE)
  const float* cgrad;     // its gradient (n per row)
  double* merit_hist;     // (rows of history, hist_len) or nullptr
  unsigned char* acc_hist;
  int hist_len;
  int n;
};

struct PlanConsts {
  double dt2inv, w_trans, w_rot, w_goal, mu, lam0, lam_min, lam_max;
};

// What one step works on.
struct PlanStep {
  const PlanTraj* trajs;  // device table of n_traj entries
  int n_traj;
  int n_rows;             // waypoint rows covered by the collision pass (idle rows have empty lists)
  const float* points;    // (n_points, 3) device
  int n_points;
  const int* offsets;     // (n_rows + 1) pair offsets of the rows' point ranges
  const int* point_base;  // (n_rows) first point of each row's range
  const int* idx;         // partition lists (CSR with offsets) or nullptr: the ranges above
  int n_pairs;
};

cudaError_t launch_plan_init(const PlanTraj* trajs, int n_traj, const PlanArrays& a, const PlanConsts& c,
                             cudaStream_t s);
cudaError_t launch_plan_update(const PlanTraj* trajs, int n_traj, const PlanArrays& a, const PlanConsts& c,
                               cudaStream_t s);
// Final iterates in FP32: trajectory r's rows go to out + out_row[r] * n.
cudaError_t launch_plan_output(const PlanTraj* trajs, int n_traj, int n, float* out, const int* out_row,
                               cudaStream_t s);
// Device bytes one trajectory's persistent state takes (arrays and scalars).
size_t plan_state_bytes(int N, int n);
int check_plan_params(const gcdf_plan_params* p);
PlanConsts plan_consts(const gcdf_plan_params* p);
// Partition lists of the step's rows around their reference bases (row i at
// base + i * bstride), each over its own point range; fills ps.offsets-like
// arrays: offsets (n_rows + 1) on the device, returns the list length.
int plan_partition(const float* base, int bstride, int rows, const float* points, const int* pbegin,
                   const int* plen, float radius, int* offsets, int** idx, long long* n_pairs, cudaStream_t s);
// One evaluation + update of every trajectory of the step.
int plan_step(gcdf_net* net, const PlanStep& ps, const PlanArrays& a, const PlanConsts& c, float delta,
              cudaStream_t s);

}  // namespace gcdf
