/*
 * gcdf.h — C ABI of libgcdf: batched neural GCDF value + configuration
 * gradient on one GB300 (sm_103a), fused with per-waypoint collision-cost
 * reductions.
 *
 * The method (arXiv 2601.18548).  The Generalized Configuration Space
 * Distance Field f(p, q) (Definition 1, Sec. III-B) of a mobile manipulator
 * with configuration q = [x, y, yaw, arm joints] is approximated by a
 * coordinate MLP over the concatenation of the point p and q (Sec. III-C).
 * The trajectory optimizer (Sec. IV-A) imposes f(p_j, q_i) - delta >= 0 for
 * every waypoint q_i and every obstacle point p_j of that waypoint's
 * partition (Eq. 11), queries all values and their gradients in one
 * GPU batch, and stacks them waypoint-major (Eq. 14) with a dense gradient
 * block of shape (sum_i m_i) x n (Eq. 15).
 *
 * Network (fixed by this library): input v = [p', x', y', sin a_1, cos a_1,
 * ..., sin a_k, cos a_k] with k = n_dof - 2 angles (base yaw, then the arm
 * joints), p' = p - (b, 0) and (x', y') = (x, y) - b for the optional
 * per-waypoint base shift b (Sec. IV-A: points are moved into the waypoint's
 * base frame before the query; b is a constant and carries no gradient);
 * L hidden layers of width H with SiLU activation; a scalar output.
 *
 * Conventions for every entry point below.
 *  - Arrays are row-major FP32 (int32 for indices) in DEVICE memory, owned by
 *    the caller, never freed or retained by the library, and 16-byte aligned
 *    (cudaMalloc and PyTorch allocations are).  Exception: weights_host.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) and return once the work is enqueued.  Outputs are valid
 *    after the stream reaches that point.  Temporary device memory is taken,
 *    stream-ordered on the same stream, from a memory pool per device that the
 *    library owns and that keeps freed memory for the next call (so the pool
 *    holds the largest temporaries used so far; gcdf_release_cached_memory
 *    returns the unused part to the driver).
 *  - Return value: GCDF_OK or an error code; gcdf_last_error() gives a
 *    message (per calling thread).  Argument errors are detected before any
 *    work is enqueued.
 *  - NaN or Inf inputs propagate to the affected outputs; nothing traps.
 *  - One net may be used from several streams at once; every call owns its
 *    temporaries.
 */
#ifndef GCDF_H
#define GCDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GCDF_API __attribute__((visibility("default")))
#else
#define GCDF_API
#endif

/* A CUDA stream handle, layout-compatible with cudaStream_t. */
typedef struct CUstream_st *gcdf_stream_t;

/* Opaque network: device copies of the weights in the layouts the kernels use. */
typedef struct gcdf_net gcdf_net;

enum gcdf_status {
  GCDF_OK = 0,
  GCDF_EINVAL = 1,       /* bad shape, NULL or misaligned pointer, bad enum */
  GCDF_ENOMEM = 2,       /* device allocation failed */
  GCDF_ECUDA = 3,        /* a CUDA call or kernel launch failed */
  GCDF_EUNSUPPORTED = 4, /* valid request the library does not implement */
  GCDF_EAGAIN = 5,       /* planning server: the queue is full, try again later */
  GCDF_PENDING = 6,      /* planning server: the request is not finished yet (poll only) */
  GCDF_ETIMEOUT = 7      /* a device wait gave up (see gcdf_device_status) */
};

enum gcdf_precision {
  GCDF_FP32 = 0, /* FP32 weights and activations on CUDA cores */
  GCDF_BF16 = 1, /* BF16 weights and activations, FP32 accumulation, tcgen05 tensor cores */
  GCDF_FP16 = 2, /* FP16 weights and activations, FP32 accumulation, same tensor-core kernel;
                    three more mantissa bits than BF16 at the same throughput, range +-65504 */
  GCDF_FP8 = 3   /* FP8 E4M3 weights (one scale per layer: max |W_l| / 448) and activations, FP32
                    accumulation, tcgen05 kind::f8f6f4; reverse-sweep operands carry a factor 64;
                    the epilogue arithmetic and the stash stay FP16 */
};

enum gcdf_reduction {
  GCDF_RED_MIN = 0,     /* c_i = min_j f_ij; grad = df/dq at the first minimising list entry */
  GCDF_RED_SOFTMIN = 1, /* c_i = -T log sum_j exp(-f_ij / T); grad = softmax-weighted df/dq */
  GCDF_RED_HINGE = 2    /* c_i = sum_j max(0, delta - f_ij); grad = -sum_{f_ij < delta} df/dq */
};

typedef struct gcdf_net_desc {
  int n_dof;           /* n: x, y, then n - 2 angles; 3 <= n <= 12 */
  int hidden;          /* H: hidden width; FP32: 64, 128, 256 or 512; BF16/FP16/FP8: 256 */
  int n_hidden_layers; /* L: number of SiLU layers, >= 2 (FP32: <= 5, BF16/FP16/FP8: <= 4) */
  int precision;       /* enum gcdf_precision */
} gcdf_net_desc;

/*
 * Number of FP32 weights a net of this shape takes: for every affine layer,
 * input to output, W (fan_out x fan_in, row-major) followed by b.  Layer 1 is
 * H x (3 + 2 + 2 (n - 2)) with input columns [p_x, p_y, p_z, x, y, sin a_1,
 * cos a_1, ..., sin a_k, cos a_k]; layers 2..L are H x H; the output layer is
 * 1 x H.  Returns 0 for an invalid shape.
 */
GCDF_API size_t gcdf_weight_count(const gcdf_net_desc *desc);

/*
 * Build a net from HOST weights (layout of gcdf_weight_count).  The weights
 * are copied (and, for GCDF_BF16 / GCDF_FP16, rounded to 16 bits and re-laid out for the
 * tensor cores) onto the current CUDA device; the host buffer may be freed
 * on return.  Synchronous.  *out receives the net; it is bound to the device
 * that was current at creation and must be used with that device current.
 * Errors: EINVAL (NULL pointer, n_weights mismatch, shape outside the limits
 * above), EUNSUPPORTED (shape valid but not built for this precision),
 * ENOMEM, ECUDA.
 */
GCDF_API int gcdf_create_net(const gcdf_net_desc *desc, const float *weights_host,
                    size_t n_weights, gcdf_net **out);

/* Free a net's device memory.  Synchronises the device first.  NULL is a no-op. */
GCDF_API int gcdf_destroy_net(gcdf_net *net);

/*
 * Value and configuration gradient for every (waypoint, point) pair — the
 * stacked constraint vector c_gcdf (Eq. 14, without the constant delta) and
 * its dense Jacobian block (Eq. 15), computed on the GPU in one batch
 * (Sec. IV-A, "GPU-parallel querying").
 *
 *   q      (n_waypoints, n)    configurations q_i
 *   p      (n_points, 3)       obstacle points p_j
 *   part_offsets (n_waypoints + 1) and part_idx (n_pairs): per-waypoint point
 *          lists I_{M,i} (Sec. IV-A partitions) in CSR form; waypoint i uses
 *          points part_idx[part_offsets[i] .. part_offsets[i+1]-1].  Both
 *          NULL = every point for every waypoint (n_pairs is then ignored and
 *          taken as n_waypoints * n_points).  part_offsets must start at 0,
 *          be non-decreasing and end at n_pairs; every index must be in
 *          [0, n_points).  Entries may repeat across or within waypoints.
 *   shift  (n_waypoints, 2) or NULL: per-waypoint base shift b_i.
 *   f      (n_pairs,)        out: f for pair k in stacked order
 *                            (dense: k = i * n_points + j)
 *   grad   (n_pairs, n) or NULL  out: df/dq for pair k; NULL runs the forward
 *          layers alone (no reverse sweep: about half the work)
 * n_waypoints == 0 or n_pairs == 0 enqueues nothing and returns GCDF_OK.
 */
GCDF_API int gcdf_query(gcdf_net *net, const float *q, int n_waypoints,
               const float *p, int n_points, const int *part_offsets,
               const int *part_idx, int n_pairs, const float *shift,
               float *f, float *grad, gcdf_stream_t stream);

/*
 * Per-waypoint collision cost and its gradient with respect to q_i, reduced
 * over that waypoint's points (all points, or its CSR list as in gcdf_query)
 * without writing any per-pair value to device memory.  The reduction turns
 * the N x M constraints f(p_j, q_i) - delta >= 0 of Eq. (11) into one cost per
 * waypoint for the optimizer:
 *   GCDF_RED_MIN      param unused.  cost_i = min_j f_ij; argmin_i = the point
 *                     index of the first list entry attaining it; grad_i its df/dq.
 *   GCDF_RED_SOFTMIN  param = temperature T > 0.  cost_i = -T log sum_j
 *                     exp(-f_ij / T); grad_i = sum_j w_ij df_ij/dq with
 *                     w = softmax(-f_i / T); argmin_i as for MIN.
 *   GCDF_RED_HINGE    param = margin delta.  cost_i = sum_j max(0, delta - f_ij)
 *                     (the l1 penalty of Eq. 12 on the GCDF rows);
 *                     grad_i = -sum_{f_ij < delta} df_ij/dq; argmin_i as for MIN.
 *   cost (n_waypoints,), grad (n_waypoints, n) out; argmin (n_waypoints,) out
 *   or NULL.  An empty list gives cost +inf (MIN, SOFTMIN) or 0 (HINGE), a
 *   zero gradient and argmin -1.
 * The result does not depend on the stream, the launch order or what else
 * runs on the device: partial results are merged in a fixed order.
 */
GCDF_API int gcdf_collision_cost(gcdf_net *net, const float *q, int n_waypoints,
                        const float *p, int n_points, const int *part_offsets,
                        const int *part_idx, int n_pairs, const float *shift,
                        int reduction, float param, float *cost, float *grad,
                        int *argmin, gcdf_stream_t stream);

/*
 * gcdf_collision_cost without any device allocation.  The paper has no
 * counterpart: this is a deployment variant of the same computation for
 * callers that must not allocate once running (for example a trajectory
 * optimizer inside a real-time control loop, where an allocation can block,
 * synchronise or fail at an unpredictable moment, or an application whose GPU
 * memory is budgeted up front).  Arguments, outputs and results are those of
 * gcdf_collision_cost.
 *
 * Every temporary comes from one 96 MiB array that is part of the library's
 * image on each device (every GPU that loads the library holds it until the
 * process exits).  A request needing more — per-waypoint terms
 * (n_waypoints x (hidden + 2 (n_dof - 2)) floats), the tile prefix of point
 * lists, one 64-byte record per tile (tiles: 128 pairs on BF16/FP16,
 * 8192 / hidden pairs on FP32) and, on BF16/FP16/FP8 nets, the tensor-core
 * kernel's stash of 2 s'(z_l) for the hidden layers 1..L-1 (128 KiB per SM
 * and layer) — is rejected with GCDF_EINVAL before any work is
 * enqueued.  Nothing in the array needs to start at zero: each call writes
 * every word it later reads.
 *
 * All calls on a device share the array, so calls whose GPU work overlaps in
 * time (on different streams, or from different threads) race and corrupt
 * each other's results; serialise them (one stream, or events).  Every call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress; the first call on a device may also load the
 * library's device code there), so the address stays right after the context
 * is destroyed and recreated; make the first call on each device before any
 * stream capture.  Calls no cudaMalloc, cudaMallocAsync or cudaFree.
 */
GCDF_API int gcdf_collision_cost_noalloc(gcdf_net *net, const float *q, int n_waypoints,
                                         const float *p, int n_points, const int *part_offsets,
                                         const int *part_idx, int n_pairs, const float *shift,
                                         int reduction, float param, float *cost, float *grad,
                                         int *argmin, gcdf_stream_t stream);

/*
 * HINGE and MIN need df/dq only where the reduction uses it: HINGE on the pairs
 * with f < delta (the active set of the l1 penalty, Eq. 12), MIN at each
 * waypoint's first minimising entry.  With the active set on (the default for
 * every net), gcdf_collision_cost and gcdf_plan_solve / the planning server
 * evaluate HINGE and MIN in two passes: every pair's value without the reverse
 * sweep, then value and gradient of the active pairs alone (NaN values count
 * as active, so they still reach the cost).  The cost, gradient and argmin are
 * those of the one-pass reduction; the HINGE sums are added in another order.
 * Temporaries grow by 8 bytes per pair (the values and the active lists).
 * gcdf_collision_cost_noalloc always runs in one pass.  enable 0 selects the
 * one-pass evaluation.  Not thread-safe against calls in flight on the same
 * net.  Errors: EINVAL (net NULL).
 */
GCDF_API int gcdf_set_active_set(gcdf_net *net, int enable);

/*
 * Device-side status of a net's kernels since the last call: 0 when every
 * bounded wait inside the tensor-core kernel completed; bit 0 set when a wait
 * gave up (the kernel then stopped issuing work, drained its copies, released
 * its tensor memory and returned; that call's outputs are not valid); bit 1
 * set when the drain itself timed out.  Synchronises the device, then clears
 * the word.  Errors: EINVAL (NULL argument), ECUDA.
 */
GCDF_API int gcdf_device_status(gcdf_net *net, int *status);

/*
 * Self-test of the device-side failure detection (no counterpart in the
 * paper).  Launches, on the net's device and synchronously, one block whose
 * two warps wait with the tensor-core kernel's own bounded-wait routines (the
 * producer/MMA wait and the epilogue's warp-wide wait) on an mbarrier that
 * nothing ever arrives on, with a limit of limit_cycles clock cycles instead of
 * the kernel's ~1 s.  Both waits must give up, raise the kernel's abort flag
 * and set bit 0 of the net's status word, exactly as a wait of the fused
 * kernel would; no copy, MMA or tensor memory is in flight, so the context
 * stays usable.  seen (3 ints, HOST) out: [producer wait expired (1/0),
 * epilogue wait expired (1/0), abort flag raised (1/0)].  Read and clear the
 * status word with gcdf_device_status.  Errors: EINVAL (NULL argument,
 * limit_cycles outside [1e3, 4e9], net of another device), ECUDA.
 */
GCDF_API int gcdf_selftest_wait_expiry(gcdf_net *net, long long limit_cycles, int *seen);

/*
 * FP32 fused-multiply-add rate loop (no counterpart in the paper): the
 * measured roofline denominator of the FP32 CUDA-core paths.  Enqueues one
 * launch of `blocks` x `threads` threads (threads a multiple of 32, at most
 * 1024), each running 8 independent FMA chains for 4 x iters steps and writing
 * one float to sink (blocks x threads floats, DEVICE).  Returns the FLOPs the
 * launch performs (2 per FMA) — time it with events on `stream` — or minus an
 * error code (EINVAL for bad arguments, ECUDA).
 */
GCDF_API long long gcdf_diag_fp32_fma(int blocks, int threads, int iters, float *sink, gcdf_stream_t stream);

/*
 * Profiling hook: while set, every gcdf_query / gcdf_collision_cost call on
 * this net records `start_event` on its stream immediately before launching
 * the fused value+gradient kernel and `stop_event` immediately after it, so
 * cudaEventElapsedTime gives that kernel's device time alone.  Both are
 * cudaEvent_t handles owned by the caller; NULL, NULL turns the hook off.
 * Errors: EINVAL (net NULL, or exactly one event NULL).
 */
GCDF_API int gcdf_set_profile_events(gcdf_net *net, void *start_event, void *stop_event);

/*
 * Single-step projection (Theorem 1, property 2): for every (waypoint, point)
 * pair, q_z = q_i - f(p_j, q_i) M^{-1} df/dq(p_j, q_i), the configuration on
 * the point's zero-level set nearest to q_i when f is the exact GCDF.
 * Arguments as gcdf_query; m_diag (n) DEVICE: the diagonal of M, or NULL for
 * the identity.  q_out (n_pairs, n) out, stacked order of Eq. (14).
 */
GCDF_API int gcdf_project(gcdf_net *net, const float *q, int n_waypoints, const float *p, int n_points,
                          const int *part_offsets, const int *part_idx, int n_pairs, const float *shift,
                          const float *m_diag, float *q_out, gcdf_stream_t stream);

/*
 * Spatial partition (Sec. IV-A): waypoint i considers the obstacle points
 * within a range of its reference base position b_i.  The paper does not give
 * the range's shape; here it is planar: I_{M,i} = { j : (p_jx - b_ix)^2 +
 * (p_jy - b_iy)^2 <= radius^2 }, evaluated in FP64 on the FP32 inputs (each
 * product and the sum rounded separately), in increasing point order — the
 * CSR lists gcdf_query and gcdf_collision_cost take.
 *   base_xy (n_waypoints, 2) DEVICE, p (n_points, 3) DEVICE, radius >= 0
 *   (INFINITY keeps every point).
 * gcdf_partition_offsets writes part_offsets (n_waypoints + 1) DEVICE;
 * part_offsets[n_waypoints] is the list length the caller then allocates for
 * part_idx, filled by gcdf_partition_indices with the same arguments.
 * Errors: EINVAL (NULL or misaligned pointer, negative size or radius), ECUDA.
 */
GCDF_API int gcdf_partition_offsets(const float *base_xy, int n_waypoints, const float *p, int n_points,
                                    float radius, int *part_offsets, gcdf_stream_t stream);
GCDF_API int gcdf_partition_indices(const float *base_xy, int n_waypoints, const float *p, int n_points,
                                    float radius, const int *part_offsets, int *part_idx, gcdf_stream_t stream);

/*
 * Dense -> sparse GCDF Jacobian (Eq. 17): row k of the dense gradient block
 * grad (n_pairs, n) (the Eq. 15 output of gcdf_query) belongs to waypoint i_k;
 * in the Jacobian of the stacked constraints with respect to the state vector
 * [x_1; ...; x_N], x_i = [q_i, v_i] in R^{2n}, its n entries sit at columns
 * 2n i_k .. 2n i_k + n - 1 (P_i of Eq. 18 places I_n at the columns of q_i;
 * the printed offset 2Nn(i-1) would exceed the 2Nn columns for i >= 2, so the
 * state stride 2n is used).  Writes the (n_pairs x 2Nn) Jacobian as CSR:
 * row_ptr (n_pairs + 1, int64) DEVICE, col_idx (n_pairs n) DEVICE, and values
 * (n_pairs n) DEVICE (a copy of grad; NULL writes the structure only).
 * part_offsets (N + 1) as for gcdf_query, or NULL for dense lists
 * (n_pairs = n_waypoints n_points).  Errors: EINVAL, ECUDA.
 */
GCDF_API int gcdf_jacobian_scatter(const float *grad, int n_waypoints, int n_dof, const int *part_offsets,
                                   int n_points, int n_pairs, long long *row_ptr, int *col_idx, float *values,
                                   gcdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Differentiable fit (Sec. III-C; distance loss of Table I).  An FP32 net
 * given by its flat weights in DEVICE memory (layout of gcdf_weight_count,
 * e.g. FP32 master weights being trained), evaluated per SAMPLE (q_b, p_b)
 * rather than over a waypoint x point grid, with the vector-Jacobian products
 * a training step needs.  Every product is a hand-written GEMM (FP32 on CUDA
 * cores, or BF16 operands with FP32 accumulation on tcgen05 tensor cores, by
 * gcdf_fit_desc.precision); the reductions over the batch (weight and bias
 * gradients) are summed in a fixed order, so results are deterministic.
 * Temporaries: the activations and s'(z) of every layer (2 L batch x hidden
 * floats), a 64-chunk partials array and, for BF16, two operand images of
 * about batch x max(hidden, input width) BF16 values, from cudaMallocAsync on
 * the stream.  A tensor-core wait that gives up (about a second) sets the
 * status that gcdf_fit_device_status reads; the call itself cannot see it.
 * ------------------------------------------------------------------------- */

typedef struct gcdf_fit_desc {
  int n_dof;            /* n, 3 .. 12 */
  int hidden;           /* H, 1 .. 4096 */
  int n_hidden_layers;  /* L, 1 .. 16 */
  int precision;        /* GCDF_FP32 (SIMT FP32 GEMMs) or GCDF_BF16 (the matrix products on
                           tcgen05 tensor cores with BF16 operands and FP32 accumulation; the
                           weights, activations and element-wise steps stay FP32) */
} gcdf_fit_desc;

/* f (batch,) DEVICE out: f(q_b, p_b) for q (batch, n) and p (batch, 3) DEVICE. */
/* Synchronises the current device, then *status = the fit kernels' device
 * status word since the last call (0: every tensor-core wait completed; bit 1:
 * one gave up and its product is incomplete) and clears it.  Errors: ECUDA. */
GCDF_API int gcdf_fit_device_status(int *status);

GCDF_API int gcdf_fit_forward(const gcdf_fit_desc *desc, const float *weights, const float *q, const float *p,
                              int batch, float *f, gcdf_stream_t stream);

/* For g_f (batch,) DEVICE = dL/df_b: dweights (gcdf_weight_count) DEVICE out =
 * sum_b g_b df_b/dweights (written, not accumulated) and, unless NULL,
 * dq (batch, n) DEVICE out = g_b df_b/dq_b. */
GCDF_API int gcdf_fit_vjp(const gcdf_fit_desc *desc, const float *weights, const float *q, const float *p,
                          int batch, const float *g_f, float *dweights, float *dq, gcdf_stream_t stream);

/* f (batch,) and dq (batch, n) DEVICE out: f(q_b, p_b) and its gradient
 * grad_q f(q_b, p_b) (the per-sample field and gradient that the regularisers
 * of Table I — gradient direction, eikonal, tension — are built from). */
GCDF_API int gcdf_fit_value_grad(const gcdf_fit_desc *desc, const float *weights, const float *q, const float *p,
                                 int batch, float *f, float *dq, gcdf_stream_t stream);

/* Second-order vector-Jacobian product for a loss of f and grad_q f: with
 * g_f (batch,) = dL/df_b and G_q (batch, n) = dL/d(grad_q f_b), both DEVICE,
 * dweights (gcdf_weight_count) DEVICE out = sum_b [g_b df_b/dweights +
 * G_b . d(grad_q f_b)/dweights] (written, not accumulated).  The gradient of
 * such a loss with respect to q itself is not provided.  Temporaries: about
 * 5 L + 3 batch x hidden floats (activations, s', s'', the reverse sweep) and
 * the partials array. */
GCDF_API int gcdf_fit_vjp2(const gcdf_fit_desc *desc, const float *weights, const float *q, const float *p,
                           int batch, const float *g_f, const float *G_q, float *dweights, gcdf_stream_t stream);

/* A training step that computes f and then its weight gradient can keep what
 * the reverse sweep of gcdf_fit_vjp needs instead of recomputing the forward
 * pass (BF16 precision only): the transposed BF16 images of the input
 * encoding and of h_1 .. h_{L-1}, s'(z_1) .. s'(z_L) and h_L in FP32, in a
 * caller-owned DEVICE buffer (the "tape").
 * gcdf_fit_tape_bytes: *bytes = the tape size for `batch` samples (0 for
 *   batch 0).  Errors: EINVAL (bad shape, FP32 precision, bytes NULL).
 * gcdf_fit_forward_tape: gcdf_fit_forward that also fills the tape (tape 256-
 *   byte aligned, at least gcdf_fit_tape_bytes long; EINVAL otherwise).
 * gcdf_fit_vjp_tape: gcdf_fit_vjp from a tape filled by gcdf_fit_forward_tape
 *   with the SAME desc, weights, q, p and batch (nothing checks that; another
 *   tape gives the gradient of that other forward pass).  The tape is only
 *   read.  Results equal gcdf_fit_vjp's bit for bit; the forward pass's
 *   products are not repeated.  Temporaries: the delta images and the weight
 *   images (about 4 batch x hidden BF16 values) and the partials array. */
GCDF_API int gcdf_fit_tape_bytes(const gcdf_fit_desc *desc, int batch, size_t *bytes);
GCDF_API int gcdf_fit_forward_tape(const gcdf_fit_desc *desc, const float *weights, const float *q, const float *p,
                                   int batch, float *f, void *tape, size_t tape_bytes, gcdf_stream_t stream);
GCDF_API int gcdf_fit_vjp_tape(const gcdf_fit_desc *desc, const float *weights, const float *q, const float *p,
                               int batch, const float *g_f, const void *tape, size_t tape_bytes, float *dweights,
                               float *dq, gcdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Trajectory optimisation with the GCDF collision cost (Sec. IV-A).
 *
 * Problem (Eq. 10 with the velocity controls eliminated through the
 * integrator; the base velocity's norm is |q^t_{i+1} - q^t_i| / dt whatever the
 * yaw, because a rotation keeps lengths): waypoints q_1 .. q_N, q_1 = q_start
 * fixed, minimise
 *   J = (1/dt^2) sum_{i<N} sum_d W_d (q_{i+1,d} - q_{i,d})^2        (control cost)
 *     + w_goal |q_N - q_goal|^2                                      (tracking cost)
 *     + mu sum_i sum_j max(0, delta - f(p_j, q_i))                   (l1 GCDF rows, Eq. 12)
 * with W_d = w_trans for x, y and w_rot for the yaw and the arm joints.
 * The paper solves its nonlinear program with an external SCP package; this
 * library replaces it with a fixed number of Levenberg-Marquardt steps
 * preconditioned by the exact Hessian A of the smooth terms (block-diagonal
 * over DOFs, tridiagonal over waypoints):
 *   (A_d + lambda diag(A_d)) s_d = g_d   (FP64 tridiagonal Cholesky, per DOF),
 *   trial = q - s; accepted when it lowers J (lambda /= 2, floor lambda_min),
 *   otherwise rejected (lambda *= 4, cap lambda_max).
 * Each step costs one HINGE collision-cost evaluation of every waypoint over
 * all points of its problem (or its partition, see partition_radius); the first
 * evaluation is the initial guess (the straight line from q_start to q_goal).  J and every step are computed in
 * FP64; the field is queried at the FP32 rounding of the trial.
 * ------------------------------------------------------------------------- */

typedef struct gcdf_plan_params {
  float dt;              /* time step (> 0) */
  float w_trans, w_rot;  /* control-cost weights (> 0) */
  float w_goal;          /* tracking weight (>= 0) */
  float mu;              /* penalty weight of the GCDF rows (>= 0) */
  float delta;           /* safety margin of Eq. (11) */
  float lambda0, lambda_min, lambda_max;  /* damping: start, floor, cap (>= 0) */
  int iterations;        /* Levenberg-Marquardt steps (>= 0); iterations + 1 evaluations */
  float partition_radius; /* > 0: waypoint i only considers the points within this planar range of
                             its reference base position, the (x, y) of the initial guess (the
                             partitions of Sec. IV-A, as gcdf_partition_*); 0: every point */
} gcdf_plan_params;

typedef struct gcdf_plan_problem {
  int n_waypoints;       /* N >= 2 */
  const float *q_start;  /* (n)      DEVICE */
  const float *q_goal;   /* (n)      DEVICE */
  const float *q_init;   /* (N, n)   DEVICE initial guess, or NULL for the straight line */
  const float *points;   /* (M, 3)   DEVICE obstacle points of this problem */
  int n_points;          /* M >= 0 */
} gcdf_plan_problem;

/*
 * Optimise n_problems trajectories together with one net: every step is one
 * batched collision-cost launch over all problems' (waypoint, point) pairs and
 * one FP64 update launch (one block per problem).  Problems do not interact:
 * each problem's result is bit-identical to solving it alone.
 *   q_out     (sum_r N_r, n) DEVICE out: the final iterates, problems in order
 *   merit_out (n_problems, iterations + 1) DEVICE out or NULL: J of the current
 *             iterate after each evaluation
 *   accepted_out (n_problems, iterations + 1) DEVICE out or NULL: 1 where the
 *             evaluation's trial was accepted (always 1 for the first)
 * Asynchronous on `stream`, except that with partition_radius > 0 the list
 * length is read back once per 2^31-pair chunk.  The problems' point arrays are
 * copied into one temporary array first; batches above 2^31 pairs are split
 * into chunks.  Errors: EINVAL (NULL or misaligned pointer, N < 2, bad parameter),
 * ENOMEM, ECUDA.
 */
GCDF_API int gcdf_plan_solve(gcdf_net *net, const gcdf_plan_problem *problems, int n_problems,
                             const gcdf_plan_params *params, float *q_out, double *merit_out,
                             unsigned char *accepted_out, gcdf_stream_t stream);

/*
 * Planning server: a host thread that owns a CUDA stream on the device that
 * was current at creation and runs the optimisation above for every admitted
 * request, with continuous batching — requests that arrive while others are
 * on the GPU are admitted at the next step boundary when a slot and enough of
 * the device-memory budget are free, and every step processes all admitted
 * requests (grouped by net) in the same launches.  Requests keep their place
 * in the queue (first come, first admitted).  A request's result does not
 * depend on what else runs with it.
 */
typedef struct gcdf_server gcdf_server;

typedef struct gcdf_server_desc {
  size_t hbm_budget_bytes;  /* device memory for admitted requests' points and state */
  int max_active;           /* requests optimised together at most (>= 1) */
  int max_queued;           /* submissions waiting for admission at most (>= 0) */
  gcdf_plan_params params;  /* used for every request */
} gcdf_server_desc;

typedef struct gcdf_plan_request {
  gcdf_net *net;            /* the robot's field; nets may differ between requests */
  int n_waypoints;          /* N >= 2 */
  const float *q_start;     /* (n)    HOST, copied at submission */
  const float *q_goal;      /* (n)    HOST, copied at submission */
  const float *points;      /* (M, 3) HOST, copied at submission */
  int n_points;             /* M >= 0 */
} gcdf_plan_request;

typedef struct gcdf_plan_result {
  float *q;                 /* (N, n) HOST, caller-provided: receives the final iterate */
  double merit;             /* out: J of the final iterate */
  int accepted_steps;       /* out: accepted trials */
  double submit_s, admit_s, done_s;  /* out: server clock (seconds) at submission,
                                        admission and completion */
} gcdf_plan_result;

/* Device bytes a request of this size counts against the server's budget
 * while admitted (its points, optimiser state, its rows of the step arrays and
 * the fused pass's temporaries).  0 for a NULL net or negative sizes. */
GCDF_API size_t gcdf_plan_request_bytes(gcdf_net *net, int n_waypoints, int n_points);

/* Start a server.  Errors: EINVAL (bad descriptor), ENOMEM, ECUDA. */
GCDF_API int gcdf_server_create(const gcdf_server_desc *desc, gcdf_server **out);

/*
 * Queue a request (non-blocking; the inputs are copied).  *ticket identifies
 * it.  Errors: EAGAIN (max_queued requests already waiting), EINVAL (bad
 * request, or one that alone needs more than the budget), ECUDA.
 */
GCDF_API int gcdf_plan_submit(gcdf_server *server, const gcdf_plan_request *request, uint64_t *ticket);

/*
 * GCDF_OK and the result (the ticket is then retired) when the request is
 * finished; GCDF_PENDING while it waits or runs; EINVAL for an unknown ticket;
 * ECUDA or ETIMEOUT when the server's device work failed.
 */
GCDF_API int gcdf_plan_poll(gcdf_server *server, uint64_t ticket, gcdf_plan_result *result);

/* Server clock in seconds (the clock of gcdf_plan_result). */
GCDF_API double gcdf_server_clock(gcdf_server *server);

/* Counters of a server's worker loop since creation (no counterpart in the
 * paper: they show what the host-driven loop costs).  A step is one
 * optimiser step of every admitted request.
 *   steps          steps run
 *   step_device_s  device time of the steps' launches (CUDA events around them)
 *   step_host_s    host time from a step's first launch to the return of the
 *                  synchronisation that ends it (includes step_device_s)
 *   pass_s         host time of the loop passes that ran a step, including
 *                  admission, rebuilding the step arrays and reading back
 *                  finished requests (includes step_host_s)
 *   active_sum     sum over steps of the admitted requests (mean batch =
 *                  active_sum / steps) */
typedef struct gcdf_server_stats {
  uint64_t steps;
  double step_device_s;
  double step_host_s;
  double pass_s;
  uint64_t active_sum;
} gcdf_server_stats;

/* Copy the counters above.  Errors: EINVAL (NULL argument). */
GCDF_API int gcdf_server_stats_get(gcdf_server *server, gcdf_server_stats *out);

/* Stop the server thread (after the step in progress) and free its memory.
 * Unfinished requests are dropped.  NULL is a no-op. */
GCDF_API int gcdf_server_destroy(gcdf_server *server);

/* Return the unused memory of the library's temporary-memory pool on the
 * current device to the driver (cudaMemPoolTrimTo 0).  Memory of calls still
 * in flight stays; synchronise first to release everything.  Errors: ECUDA. */
GCDF_API int gcdf_release_cached_memory(void);

/* Message for the last error returned on the calling thread ("" if none). */
GCDF_API const char *gcdf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GCDF_H */
