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
 *    after the stream reaches that point.  Temporary device memory is taken
 *    with cudaMallocAsync on the same stream and released on it.
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
  GCDF_EUNSUPPORTED = 4  /* valid request this build does not implement */
};

enum gcdf_precision {
  GCDF_FP32 = 0, /* FP32 weights and activations on CUDA cores */
  GCDF_BF16 = 1, /* BF16 weights and activations, FP32 accumulation, tcgen05 tensor cores */
  GCDF_FP16 = 2  /* FP16 weights and activations, FP32 accumulation, same tensor-core kernel;
                    three more mantissa bits than BF16 at the same throughput, range +-65504 */
};

enum gcdf_reduction {
  GCDF_RED_MIN = 0,     /* c_i = min_j f_ij; grad = df/dq at the first minimising list entry */
  GCDF_RED_SOFTMIN = 1, /* c_i = -T log sum_j exp(-f_ij / T); grad = softmax-weighted df/dq */
  GCDF_RED_HINGE = 2    /* c_i = sum_j max(0, delta - f_ij); grad = -sum_{f_ij < delta} df/dq */
};

typedef struct gcdf_net_desc {
  int n_dof;           /* n: x, y, then n - 2 angles; 3 <= n <= 12 */
  int hidden;          /* H: hidden width; FP32: 64, 128, 256 or 512; BF16/FP16: 256 */
  int n_hidden_layers; /* L: number of SiLU layers, >= 2 (FP32: <= 5, BF16/FP16: <= 4) */
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
 *   grad   (n_pairs, n) or NULL  out: df/dq for pair k
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
 * Every temporary comes from one 16 MiB array that is part of the library's
 * image on each device (every GPU that loads the library holds it until the
 * process exits).  A request needing more — per-waypoint terms
 * (n_waypoints x (hidden + 2 (n_dof - 2)) floats), the tile prefix of point
 * lists and one 64-byte record per tile (tiles: 128 pairs on BF16/FP16,
 * 8192 / hidden pairs on FP32) — is rejected with GCDF_EINVAL before any work
 * is enqueued.  Nothing in the array needs to start at zero: each call writes
 * every word it later reads.
 *
 * All calls on a device share the array, so calls whose GPU work overlaps in
 * time (on different streams, or from different threads) race and corrupt
 * each other's results; serialise them (one stream, or events).  The first
 * call on each device looks up the array's device address (under a lock);
 * make that first call before any stream capture.  Calls no cudaMalloc,
 * cudaMallocAsync or cudaFree.
 */
GCDF_API int gcdf_collision_cost_noalloc(gcdf_net *net, const float *q, int n_waypoints,
                                         const float *p, int n_points, const int *part_offsets,
                                         const int *part_idx, int n_pairs, const float *shift,
                                         int reduction, float param, float *cost, float *grad,
                                         int *argmin, gcdf_stream_t stream);

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
 * Profiling hook: while set, every gcdf_query / gcdf_collision_cost call on
 * this net records `start_event` on its stream immediately before launching
 * the fused value+gradient kernel and `stop_event` immediately after it, so
 * cudaEventElapsedTime gives that kernel's device time alone.  Both are
 * cudaEvent_t handles owned by the caller; NULL, NULL turns the hook off.
 * Errors: EINVAL (net NULL, or exactly one event NULL).
 */
GCDF_API int gcdf_set_profile_events(gcdf_net *net, void *start_event, void *stop_event);

/* Message for the last error returned on the calling thread ("" if none). */
GCDF_API const char *gcdf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GCDF_H */
