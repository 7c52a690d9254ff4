/*
 * dpvo_ba.h -- C ABI of the B300-native differentiable Gauss-Newton bundle
 * adjustment over the DPVO patch graph (Deep Patch Visual Odometry, Sec. 3.1
 * "Differentiable Bundle Adjustment", Eq. 6; reprojection Eq. 2-3; damping in
 * the Appendix "Bundle Adjustment Layer"; optimisation window Sec. 3.3).
 *
 * The layer minimises, over camera poses T (world->camera, SE(3)) and one
 * inverse depth d_k per patch (its pixel centre held fixed),
 *
 *     sum_{(k,j) in edges}  || target_kj - omega_ij(T, P_k) ||^2_{diag(weight_kj)}
 *
 * where patch k is anchored in frame i = anchor[k] and omega_ij reprojects its
 * centre (x_k, y_k) at inverse depth d_k from frame i into frame j (Eq. 2).
 * Every iteration linearises the residuals, eliminates the inverse depths with
 * the Schur complement, solves the reduced pose system by Cholesky with poses
 * [0, t0) held fixed, back-substitutes the inverse depths and retracts
 * T_a <- Exp(dxi_a) T_a (left increment, dxi = (v, w), translation first),
 * d_k <- d_k + dd_k.  A damping lambda is added to every inverse-depth diagonal
 * entry.  An edge takes part iff the third homogeneous coordinate of the
 * reprojected centre exceeds z_min.
 *
 * Conventions for every entry point
 *   - Return value: DPVO_BA_OK (0) or a negative DPVO_BA_E* code.  No call aborts,
 *     traps or waits without a bound.
 *   - Pointers inside dpvo_ba_problem are DEVICE pointers owned by the caller;
 *     the library never frees them.  Arrays are dense, row-major, float32 or
 *     int32 as stated, and must stay valid until the work on `stream` is done.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are asynchronous on that stream unless stated otherwise.
 *   - The handle owns its device workspace; calls that need more than it holds
 *     grow it (a cudaMalloc outside any kernel).  dpvo_ba_reserve() grows it
 *     ahead of time so that later solves allocate nothing.
 *   - A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef DPVO_BA_H
#define DPVO_BA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define DPVO_BA_OK            0
#define DPVO_BA_EINVAL      (-1)   /* bad argument (NULL, negative size, limit exceeded) */
#define DPVO_BA_ENOMEM      (-2)   /* device allocation failed or memory budget exceeded */
#define DPVO_BA_ECUDA       (-3)   /* a CUDA runtime call failed                         */
#define DPVO_BA_ETIMEOUT    (-4)   /* a bounded wait ran out                             */
#define DPVO_BA_EBUSY       (-5)   /* serving: no slot free and the call may not block   */
#define DPVO_BA_ENOTFOUND   (-6)   /* serving: unknown session or ticket                 */

/* ---- per-problem status bits (written to dpvo_ba_problem.status) -------- */
#define DPVO_BA_STATUS_OK          0
#define DPVO_BA_STATUS_NOT_SPD     1  /* reduced pose system not positive definite: pivot <= 0 or NaN */
#define DPVO_BA_STATUS_BAD_INPUT   2  /* index out of range, unsorted edges, or a capacity exceeded   */
#define DPVO_BA_STATUS_NONFINITE   4  /* a non-finite increment was produced                          */
#define DPVO_BA_STATUS_TIMEOUT     8  /* a bounded device-side wait (tensor-core completion) ran out  */
/* A problem whose status is not OK leaves its poses and patches as it found them. */

/* ---- capacities of this build ------------------------------------------- */
#define DPVO_BA_MAX_FRAMES       128  /* N per problem                                   */
#define DPVO_BA_MAX_FREE          32  /* N - t0 per problem (reduced system <= 192 x 192) */
#define DPVO_BA_MAX_ITERS         16  /* Gauss-Newton iterations per solve               */

/* Sizes of one problem. */
typedef struct {
    int32_t n_frames;   /* N >= 1                                                  */
    int32_t n_patches;  /* P >= 0                                                  */
    int32_t n_edges;    /* E >= 0                                                  */
    int32_t t0;         /* poses [0, t0) fixed, [t0, N) free; 0 <= t0 <= N          */
    int32_t n_iters;    /* Gauss-Newton iterations (2 in the paper, Sec. 3.3)       */
    float fx, fy, cx, cy; /* pinhole intrinsics (Eq. 3)                             */
} dpvo_ba_dims;

/* Layer constants (Appendix "Bundle Adjustment Layer": damping 1e-4). */
typedef struct {
    float damping;          /* lambda added to each inverse-depth diagonal entry (1e-4)   */
    float z_min;            /* edge active iff reprojected homogeneous depth > z_min (0.1)*/
    size_t mem_budget_bytes;/* serving: device bytes sessions may hold (0 = 8 GiB)        */
    int32_t max_sessions;   /* serving: resident sessions (0 = 256)                       */
    int32_t schur_tf32;     /* Where sum_k E_k C_k^-1 E_k^T accumulates.  Up to 15 free
                             * poses (the Schur sums fused into the linearisation):
                             * mode 0 (default) and 2 in FP32 with compensated sums on the
                             * CUDA cores; mode 1, when every problem of the batch has at
                             * most 10 free poses, on the tensor cores, each term as three
                             * TF32 products (hi.hi + hi.lo + lo.hi).  Beyond 15 free poses
                             * (a separate assembly launch): modes 0 and 1 on the tensor
                             * cores (three TF32 products, the FP32 accumulation in TMEM
                             * over at most 2048 patches, the ranges added in FP64), mode
                             * 2 in compensated FP32 on the CUDA cores.  The tensor cores'
                             * FP32 accumulation truncates: on the fused path's
                             * ill-conditioned systems the pose update error grows about
                             * 5x (measured up to 1e-5 relative end to end, vs 1e-6 in
                             * FP32); on the wide windows both assemblies meet 1e-4 per
                             * iteration against the FP64 oracle                           */
    int32_t reduced_solve_f64; /* 0 (default): the reduced pose system is factored in FP32
                             * and its solution refined against the FP64 system, with
                             * FP64 elimination where an FP32 pivot fails or the
                             * refinement stalls.  1: FP64 elimination always (slower;
                             * the reference mode of the fallback path)                  */
} dpvo_ba_config;

/* One problem's device arrays (caller-owned).
 *   poses   [N][7]  tx ty tz qx qy qz qw, world->camera, unit quaternion.  IN/OUT.
 *   patches [P][3]  x y d: pixel centre and inverse depth.  d is IN/OUT, x y are read.
 *   anchor  [P]     source frame i_k of each patch, non-decreasing in k.
 *   kk      [E]     patch of each edge, non-decreasing (edges grouped by patch).
 *   jj      [E]     frame of each edge; strictly increasing within one patch.
 *   target  [E][2]  2-D target pixel (the reprojection centre plus the flow revision).
 *   weight  [E][2]  per-component confidence weight (the paper's Sigma, in (0,1)).
 *   status  [1]     int32 DPVO_BA_STATUS_* bits written by solve (may be NULL).   */
typedef struct {
    float *poses;
    float *patches;
    const int32_t *anchor;
    const int32_t *kk;
    const int32_t *jj;
    const float *target;
    const float *weight;
    int32_t *status;
} dpvo_ba_problem;

typedef struct dpvo_ba_handle dpvo_ba_handle;

/* Create a handle on the current CUDA device.  cfg may be NULL (defaults above).
 * Errors: EINVAL (out NULL), ECUDA, ENOMEM. */
int dpvo_ba_create(const dpvo_ba_config *cfg, dpvo_ba_handle **out);

/* Release the handle and its workspace (waits for the handle's own work). */
int dpvo_ba_destroy(dpvo_ba_handle *h);

/* Grow the workspace so that a solve of up to n_problems problems, none larger
 * than *max_dims (frames, patches, edges, iterations; t0 is ignored), needs no
 * further allocation.  Synchronous.  Errors: EINVAL, ENOMEM. */
int dpvo_ba_reserve(dpvo_ba_handle *h, const dpvo_ba_dims *max_dims, int n_problems);

/* Solve n_problems independent problems (dims[b], probs[b] host arrays of
 * structs describing device data), n_iters Gauss-Newton iterations each (Sec.
 * 3.1, Eq. 6).  n_problems == 1 is the plain form; larger batches are packed
 * into the same launches.  Poses and inverse depths are updated in place;
 * status bits written per problem.  Asynchronous on stream.
 * Errors: EINVAL (NULL, sizes out of range, more than DPVO_BA_MAX_FREE free
 * poses), ENOMEM, ECUDA.  Input-content errors (indices, ordering) are reported
 * per problem as DPVO_BA_STATUS_BAD_INPUT, not as a return code. */
int dpvo_ba_solve(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *probs,
                  int n_problems, void *stream);

/* The same solve with every array in HOST memory (pageable or pinned): copies
 * the inputs to the handle's device staging area, solves, copies poses,
 * patches and status back, and synchronises before returning.  The pointers in
 * hprobs are host pointers with the layouts above.  A call of at least 64
 * problems goes in up to 8 sub-batches of at least 32: each sub-batch's
 * descriptors and inputs are copied on a stream of the handle's own (after the
 * caller's prior work on `stream`), and each is solved on `stream` once its
 * inputs have landed, so the solves run under the later copies.  Afterwards
 * dpvo_ba_iterate sees the last sub-batch's problems only (index 0 = its
 * first).  Errors: as dpvo_ba_solve. */
int dpvo_ba_solve_host(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *hprobs,
                       int n_problems, void *stream);

/* Gradient buffers of one problem for dpvo_ba_backward (DEVICE pointers, caller-owned).
 *   dL_dposes  [N][7]  dL/d(final poses), same layout as the poses      (read)
 *   dL_ddepth  [P]     dL/d(final inverse depths)                        (read)
 *   dL_dtarget [E][2]  dL/d(targets)                                     (written)
 *   dL_dweight [E][2]  dL/d(weights)                                     (written)            */
typedef struct {
    const float *dL_dposes;
    const float *dL_ddepth;
    float *dL_dtarget;
    float *dL_dweight;
} dpvo_ba_grads;

/* Backward pass of the layer (Sec. 3.1: gradients are propagated through the
 * Gauss-Newton iterations).  probs[b] describes the problem's state at the
 * START of the forward solve; it is read, never modified.  The forward
 * iterations are recomputed (only the small per-iteration states, increments
 * and FP64 reduced-system factors are kept in the workspace), then the
 * adjoint runs back through every iteration: retraction (SE(3) left
 * Jacobian), linear solve (Schur complement with the kept factor), and the
 * per-edge residual and Jacobian terms including the Jacobian's own
 * derivative.  Inactive edges and self edges get zero gradient; a problem
 * whose status is not OK gets zero gradients.  Up to DPVO_BA_MAX_FREE free
 * poses: beyond 15 the forward's reduced systems are eliminated in FP64 (their
 * factors kept, n (n + 1) / 2 doubles per iteration) and the adjoint's
 * right-hand side sum_k E_k C_k^-1 dbar_k is assembled from the rows of each
 * adjoint linearisation, in the forward's Schur mode.  Asynchronous on stream.
 * Errors: EINVAL (as dpvo_ba_solve, a NULL gradient buffer), ENOMEM, ECUDA. */
int dpvo_ba_backward(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *probs,
                     const dpvo_ba_grads *grads, int n_problems, void *stream);

/* ---- serving: many concurrent VO sessions, continuously batched ----------
 * (The paper's VO system runs one bundle adjustment per frame, Sec. 3.3; these
 * calls serve many such streams from one GPU.)  A session keeps one problem's
 * graph and state resident in device memory owned by the library; each request
 * brings new targets and weights (host memory) for one session and runs
 * n_iters Gauss-Newton iterations on the session's current state.  A
 * scheduler thread packs every pending request into the next batched solve as
 * soon as one of max_in_flight launch slots is free, so requests that arrive
 * while a batch runs join the next batch and batches overlap on the device.
 * Sessions are admitted against cfg.mem_budget_bytes (their resident arrays;
 * the slots' workspaces are reserved at start and not counted).  A session
 * takes one request at a time.  Every wait is bounded; none traps. */

/* Start the scheduler.  max_dims bounds every session's sizes (as for
 * dpvo_ba_reserve); max_batch requests per launch; 1..8 launch slots.
 * Errors: EINVAL, EBUSY (already started), ENOMEM. */
int dpvo_ba_serve_start(dpvo_ba_handle *h, const dpvo_ba_dims *max_dims, int max_batch, int max_in_flight);

/* Stop the scheduler, wait for the launches in flight, close every session.
 * Also done by dpvo_ba_destroy. */
int dpvo_ba_serve_stop(dpvo_ba_handle *h);

/* Open a session from HOST arrays (layouts of dpvo_ba_problem; status unused).
 * The data are copied; the caller may free them on return.  EBUSY when the
 * session does not fit in the remaining memory budget (not admitted: retry
 * after closing another).  Errors: EINVAL, EBUSY, ENOMEM, ECUDA. */
int dpvo_ba_session_open(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *host_problem,
                         int64_t *session_id);

/* Close a session once its request (if any) has finished (waits up to 10 s:
 * ETIMEOUT) and release its memory.  Errors: EINVAL, ENOTFOUND, ETIMEOUT. */
int dpvo_ba_session_close(dpvo_ba_handle *h, int64_t session_id);

/* Copy a session's current poses [N][7] and patches [P][3] to HOST memory (either
 * may be NULL); waits up to 10 s for its request to finish.  Synchronous. */
int dpvo_ba_session_read(dpvo_ba_handle *h, int64_t session_id, float *poses_out, float *patches_out);

/* Queue a request on a session: target and weight are HOST arrays [E][2].
 * Pageable buffers are copied before the call returns; page-locked ones
 * (cudaMallocHost, cudaHostAlloc, cudaHostRegister) are read in place by the
 * device when the batch runs, so they must stay unchanged until the request
 * completes.  EBUSY if the session's previous request has not finished.
 * Errors: EINVAL (also for a window session: see dpvo_ba_submit_frame),
 * ENOTFOUND, EBUSY. */
int dpvo_ba_submit(dpvo_ba_handle *h, int64_t session_id, const float *target, const float *weight,
                   uint64_t *ticket);

/* Non-blocking: DPVO_BA_OK and the request's status bits and latency (submit to
 * completion on the device, milliseconds) when done -- a ticket is collected
 * once; EBUSY while pending; ENOTFOUND for an unknown or collected ticket. */
int dpvo_ba_poll(dpvo_ba_handle *h, uint64_t ticket, int32_t *status, double *latency_ms);

/* Blocking form of dpvo_ba_poll, bounded by timeout_ms (ETIMEOUT). */
int dpvo_ba_wait(dpvo_ba_handle *h, uint64_t ticket, int timeout_ms, int32_t *status, double *latency_ms);

/* Diagnostic: the reduced pose system of ONE linearisation at the given state
 * (no update).  S_out [n][n] and v_out [n] are DEVICE float64 arrays with
 * n = 6 (N - t0): S = B - E C^-1 E^T and v' = v - E C^-1 w (Sec. 3.1, Schur
 * complement).  Asynchronous.  Errors: EINVAL, ENOMEM, ECUDA. */
int dpvo_ba_reduced_system(dpvo_ba_handle *h, const dpvo_ba_dims *dims, const dpvo_ba_problem *prob,
                           double *S_out, double *v_out, void *stream);

/* Diagnostic: after a solve on this handle (and before the next call on it),
 * copy problem `index`'s state after iteration `iter` (0 = the input state,
 * n_iters = the output) into HOST buffers: poses_out [N][7] float32 and
 * depth_out [P] float32; and, for iter < n_iters, the FP64 pose increment of
 * that iteration, dxi_out [N - t0][6] (v then w).  Any output may be NULL.
 * Synchronises the device.  Errors: EINVAL (no such problem or iteration). */
int dpvo_ba_iterate(dpvo_ba_handle *h, int index, int iter, float *poses_out, float *depth_out,
                    double *dxi_out);

/* Diagnostic timing.  While enabled (enable != 0), every solve records a CUDA
 * event on its own stream before and after each kernel launch.
 * dpvo_ba_timing() waits for the recorded events and writes, for each launch
 * since the previous read (all solves, in order), the elapsed milliseconds
 * (ms_out[i]) and the kernel (kind_out[i]: 0 plan, 1 linearise/Schur,
 * 2 reduce/Cholesky/retract, 3 Schur assembly, 4 last depth back-substitution);
 * it returns the number of launches written
 * (<= cap) or a negative code, and starts a new record.  The record grows
 * while enabled: read it regularly. */
int dpvo_ba_set_timing(dpvo_ba_handle *h, int enable);
int dpvo_ba_timing(dpvo_ba_handle *h, float *ms_out, int *kind_out, int cap);

/* Failure-detection self-test (the paper has no counterpart).  Every
 * pipelined kernel (TF32 Schur, assembly, correlation) waits on mbarriers with
 * a bounded number of polls and reports DPVO_BA_STATUS_TIMEOUT instead of
 * hanging.  This launches one thread that initialises an mbarrier expecting
 * one arrival, arrives on it if `arrive` != 0, and then waits for the phase
 * with the same bounded wait, at most `polls` polls.  *status (device int32,
 * caller-owned) receives DPVO_BA_STATUS_TIMEOUT if the wait gave up (the phase
 * never completes when arrive == 0), else 0.  Asynchronous on `stream`; the
 * context stays usable.  Errors: EINVAL (NULL status, polls < 1), ECUDA. */
int dpvo_ba_selftest_bounded_wait(int32_t *status, int arrive, int polls, void *stream);

/* Allocation-free solve of ONE problem (the paper has no counterpart: this is
 * a deployment entry point).  For callers that may not allocate device memory
 * while running -- fixed-budget embedded pipelines, processes whose device
 * memory is owned by another allocator, real-time loops that cannot take
 * cudaMalloc's device synchronisation -- it needs no handle and makes no host
 * or device allocation.  Its workspace is a fixed 8 MiB device array inside
 * this library, held by every GPU that loads the library until the process
 * exits.  Arguments as for dpvo_ba_solve with n_problems == 1 (cfg may be NULL
 * for the defaults); results are the same as dpvo_ba_solve's.
 *   - Every call looks up the array's device address in the current context
 *     and sets the kernels' attributes: host-side calls that allocate nothing
 *     once this library's module is loaded on the device.  The first call on a
 *     device loads it, so make that first call before any stream capture, with
 *     the device current.  An error left pending on the calling thread by
 *     earlier, unrelated CUDA work is cleared, not reported as this call's.
 *   - All calls in the process share the one array and it keeps the previous
 *     call's contents (every call rewrites what it reads).  Calls whose work
 *     overlaps on the GPU -- on different streams, or from several host
 *     threads -- race on it and corrupt each other: serialise them.
 *   - Returns DPVO_BA_EINVAL, launching nothing, when the problem's workspace
 *     exceeds the array, or when it has more than 15 free poses (this entry
 *     point has no separate Schur-assembly pass).  The workspace grows with
 *     the patch count (one chunk of up to 64 patches per work item, up to two
 *     CTAs per SM, each with its own partial reduced system; one stored Schur
 *     row per patch) and with the square of the free-pose count: an 8-frame
 *     problem of 512 patches needs about 0.4 MiB, a 22-frame window of 2112
 *     patches with 10 free poses about 1.9 MiB, a 32-frame window of 3072
 *     patches with 10 free poses about 3.4 MiB.
 * Errors: EINVAL, ECUDA. */
int dpvo_ba_solve_noalloc(const dpvo_ba_config *cfg, const dpvo_ba_dims *dims, const dpvo_ba_problem *prob,
                          void *stream);

/* ---- pose supervision (Sec. 3.4, Eq. 7) -----------------------------------
 * The training loss on the poses, L = sum over ordered frame pairs (i, j),
 * i != j, of || Log_SE(3)[ (G_i^-1 G_j)^-1 (T_i^-1 T_j) ] || (the Euclidean norm
 * of the twist (rho, phi), translation first), with T the predicted and G the
 * ground-truth poses, and its gradient dL/dT in the layout dpvo_ba_grads takes,
 * so that dpvo_ba_backward carries it to the targets and weights.  The
 * predicted translations are first multiplied by `scale` (the Umeyama scale
 * alignment of the paper, computed by the caller and held constant).  One
 * problem per descriptor; all pointers DEVICE, caller-owned:
 *   poses      [N][7]  predicted poses (t, q xyzw), world -> camera   (read)
 *   gt_poses   [N][7]  ground-truth poses, same layout                (read)
 *   loss       [1]     L                                              (written)
 *   dL_dposes  [N][7]  dL/d(t, q): the translation gradient, and the
 *                      quaternion gradient of L(t, q / |q|) (orthogonal to q)
 *                      (written)
 * A pair whose twist is shorter than 1e-5 adds its length to L but nothing to
 * the gradient (the norm is not differentiable at zero, and below that length
 * the twist's direction is FP32 rounding of the relative poses).  FP32 arithmetic; J_l^-1 of the twist by its
 * Bernoulli series in ad (converges for rotation angles up to pi, which Log
 * returns).  Asynchronous on stream; no workspace.
 * Errors: EINVAL (NULL pointers, n_frames outside [1, DPVO_BA_MAX_FRAMES],
 * n_problems < 0), ECUDA. */
typedef struct {
    const float *poses;
    const float *gt_poses;
    float *loss;
    float *dL_dposes;
    int32_t n_frames;
    float scale;
} dpvo_ba_pose_loss_problem;

int dpvo_ba_pose_loss(const dpvo_ba_pose_loss_problem *probs, int n_problems, void *stream);

/* ---- window maintenance (Sec. 3.3 "Expansion" and "Optimization") -------
 * A sliding optimisation window kept on the device: frames are appended one at
 * a time and, once the window holds max_frames frames, the oldest frame leaves
 * with every patch extracted from it.  Appending a frame (one kernel launch):
 *   - its pose from the constant-velocity model T_n = T_{n-1} T_{n-2}^-1 T_{n-1}
 *     (T_n = T_{n-1} for the second frame, identity for the first; FP64
 *     composition, stored FP32);
 *   - its patches at the caller's pixel centres, all with the median inverse
 *     depth of the patches extracted from the previous 3 frames (the lower
 *     median: rank floor((K - 1) / 2) of the K values; 1 when K = 0);
 *   - the edges regenerated from the patch graph rule: patch k connects to
 *     every frame j of the window with |j - anchor_k| <= radius, edges grouped
 *     by patch, frames increasing (the layout dpvo_ba_solve requires);
 *   - targets set to the reprojection at the current state (Eq. 2; the patch
 *     centre for self edges and for points behind the camera), weights to 1:
 *     the caller overwrites both (the update operator's output) before a solve;
 *   - t0 = min(n_frames, max(2, n_frames - free_poses)): the last free_poses
 *     poses are free, but the first two always stay fixed (gauge and
 *     monocular scale; with fewer fixed poses S is singular).
 * The host keeps the per-frame patch counts, so the new sizes are known without
 * reading the device.  The window's arrays are library-owned device memory;
 * dpvo_ba_window_problem returns them, valid until the next append or destroy
 * (poses, inverse depths, targets and weights may be written through them). */
typedef struct dpvo_ba_window dpvo_ba_window;

typedef struct {
    int32_t max_frames;       /* frames kept, 1 .. DPVO_BA_MAX_FRAMES                     */
    int32_t max_new_patches;  /* patches per appended frame, at most (0 .. 8192)          */
    int32_t radius;           /* graph radius in frames (>= 0)                            */
    int32_t free_poses;       /* the last free_poses poses are free (>= 0)                */
    int32_t n_iters;          /* Gauss-Newton iterations recorded in the window's dims    */
    float fx, fy, cx, cy;     /* pinhole intrinsics (Eq. 3)                               */
} dpvo_ba_window_params;

/* Create an empty window (device memory for its maximum sizes).
 * Errors: EINVAL (a parameter out of range), ENOMEM, ECUDA. */
int dpvo_ba_window_create(const dpvo_ba_window_params *params, dpvo_ba_window **out);

/* Free the window's memory (after the work queued on its arrays). */
int dpvo_ba_window_destroy(dpvo_ba_window *w);

/* Append a frame with n_new patches at DEVICE pixel centres new_xy [n_new][2]
 * (read).  Asynchronous on stream; the window's earlier work must be ordered
 * before it (same stream).  Every argument is checked before the window
 * changes: an EINVAL leaves it as it was.  If a launch fails (ECUDA) after the
 * window's sizes have moved on, the window is marked unusable and every later
 * call on it returns ECUDA.  Errors: EINVAL (NULL, n_new outside
 * [0, max_new_patches]), ECUDA. */
int dpvo_ba_window_append(dpvo_ba_window *w, const float *new_xy, int n_new, void *stream);

/* Append one frame to each of n distinct windows (ws[b] with n_new[b] patches
 * at DEVICE new_xy[b]); host arrays of length n.  Two launches per 128
 * windows.  Errors: EINVAL (as dpvo_ba_window_append, or a window listed
 * twice), ECUDA. */
int dpvo_ba_window_append_batch(dpvo_ba_window *const *ws, const float *const *new_xy, const int *n_new, int n,
                                void *stream);

/* The window's current problem: sizes (with t0, n_iters, intrinsics) and its
 * device arrays (status included).  Errors: EINVAL (NULL, empty window). */
int dpvo_ba_window_problem(const dpvo_ba_window *w, dpvo_ba_dims *dims, dpvo_ba_problem *prob);

/* ---- sliding-window serving sessions (Sec. 3.3 "Expansion" and
 * "Optimization", served as in the calls above) ------------------------------
 * A window session owns a window (semantics of dpvo_ba_window above, created
 * empty) instead of a fixed graph.  Each request appends a frame and then
 * solves the window: the VO system's per-frame step.  Requests of window and
 * fixed-graph sessions are batched together.  dpvo_ba_poll, dpvo_ba_wait,
 * dpvo_ba_session_read and dpvo_ba_session_close take window sessions too. */

/* Open a window session.  Admitted against the memory budget by the window's
 * device bytes; its largest problem (max_frames frames, max_frames x
 * max_new_patches patches, the graph's edges, n_iters) must fit the max_dims
 * given to dpvo_ba_serve_start.  Errors: EINVAL (parameters out of range or
 * beyond max_dims), EBUSY (over the budget: not admitted), ENOMEM, ECUDA. */
int dpvo_ba_session_open_window(dpvo_ba_handle *h, const dpvo_ba_window_params *params, int64_t *session_id);

/* The number of edges E the session's window holds after appending a frame of
 * n_new patches (from the host's frame counts; nothing runs on the device):
 * the length of the arrays dpvo_ba_submit_frame takes.  Errors: EINVAL (not a
 * window session, n_new out of range), ENOTFOUND, EBUSY (a request is pending:
 * the count changes when it runs). */
int dpvo_ba_session_frame_edges(dpvo_ba_handle *h, int64_t session_id, int n_new, int32_t *n_edges);

/* The session's current sizes (a window's frames, patches, edges and t0; the
 * fixed graph's dims).  Waits up to 10 s for its pending request.
 * Errors: EINVAL, ENOTFOUND, ETIMEOUT. */
int dpvo_ba_session_dims(dpvo_ba_handle *h, int64_t session_id, dpvo_ba_dims *dims);

/* Queue a frame request on a window session (HOST arrays):
 *   new_xy [n_new][2]  the new frame's patch centres (pixels), 0 <= n_new <= max_new_patches;
 *   delta  [E][2]      revision of each edge's target, E = dpvo_ba_session_frame_edges(n_new):
 *                      the target becomes the edge's reprojection at the window's
 *                      current state plus delta (the flow revision of Eq. 5-6);
 *   weight [E][2]      the edges' confidence weights.
 * delta and weight are both given or both NULL (then targets stay the
 * reprojections and weights 1).  When it runs: the frame is appended (as
 * dpvo_ba_window_append), the factors set, and the window solved with its
 * n_iters iterations.  Pageable buffers are copied before the call returns;
 * page-locked ones are read in place when the batch runs (keep them unchanged
 * until the request completes).  Errors: EINVAL (not a window session, bad
 * sizes, one of delta / weight NULL), ENOTFOUND, EBUSY. */
int dpvo_ba_submit_frame(dpvo_ba_handle *h, int64_t session_id, const float *new_xy, int n_new, const float *delta,
                         const float *weight, uint64_t *ticket);

/* ---- correlation features (Sec. 3.2 "Correlation", Eq. 4; Appendix
 * "Correlation Operation") -----------------------------------------------------
 * For every edge (k, j) and every pixel (u, v) of patch k's p x p grid, the
 * inner products of its feature vector g_uv with frame j's features bilinearly
 * sampled on the 7 x 7 integer grid around the pixel's reprojection, at both
 * pyramid levels:
 *   C[e][l][uv][a][b] = < g_uv , f_l( P'_kj(u, v) / s_l + (a - 3, b - 3) ) >
 * with s_0 = 1, s_1 = level1_scale.  Coordinates are in level-0 feature-map
 * pixels (x along the width), pixel centres at integers; bilinear sampling
 * reads zero outside the map.  By linearity each 7 x 7 grid is a bilinear
 * combination of the 8 x 8 integer-pixel inner products around it; those are
 * computed for the bounding box of the patch's 9 windows as one small GEMM on
 * the tensor cores (tcgen05, BF16 operands, FP32 accumulators in TMEM).
 * All pointers DEVICE, caller-owned:
 *   fmap0   [N][H0][W0][128] bf16  level-0 matching features            (read)
 *   fmap1   [N][H1][W1][128] bf16  level 1, H1 = H0 / s, W1 = W0 / s     (read)
 *   gpatch  [P][9][128] bf16       patch features, pixel uv = 3 u + v      (read)
 *   kk, jj  [E] int32              patch and frame of each edge            (read)
 *   coords  [E][9][2] float        P'_kj(u, v) as (x, y), level-0 pixels  (read)
 *   corr    [E][2][9][7][7] float  the correlation features               (written)
 *   status  [1] int32              bits OR-ed in: DPVO_BA_STATUS_BAD_INPUT for an
 *                                  edge whose kk or jj is out of range (its
 *                                  output is zero), DPVO_BA_STATUS_TIMEOUT if
 *                                  a bounded wait ran out (the outputs from
 *                                  then on are zero)                       (read, OR-ed)
 * An edge-level whose coordinates are not finite or beyond 1e4 gets zeros;
 * one whose 9 windows span more than 4 x 128 pixels is computed on the CUDA
 * cores instead.  fmap0, fmap1 and gpatch must start on 16-byte boundaries
 * (features are read in 16-byte pieces: tensor-map box loads, copies).
 * Asynchronous on stream.
 * Errors: EINVAL (NULL, a feature array not 16-byte aligned, sizes out of
 * range: maps of 1 .. 4096 pixels per side, level1_scale >= 1, at least one
 * frame), ECUDA. */
#define DPVO_BA_CORR_DIM 128
typedef struct {
    int32_t n_frames, n_patches, n_edges;
    int32_t height, width;       /* level-0 map H0 x W0                                  */
    int32_t level1_scale;        /* level 1 = level 0 average-pooled by this factor (4)  */
} dpvo_ba_corr_dims;

int dpvo_ba_correlation(const dpvo_ba_corr_dims *dims, const void *fmap0, const void *fmap1, const void *gpatch,
                        const int32_t *kk, const int32_t *jj, const float *coords, float *corr, int32_t *status,
                        void *stream);

/* Human-readable name of a return code. */
const char *dpvo_ba_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* DPVO_BA_H */
