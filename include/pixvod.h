/*
 * pixvod.h - C ABI of the GB300 (sm_103a) PixVOD GBP sweep library.
 *
 * PixVOD (Kim, Alzugaray, Rhodes, Kelly, Davison; arxiv 2606.03989) tracks the
 * 6-DoF motion of a camera relative to a keyframe and the keyframe's log-depth
 * with synchronous Gaussian Belief Propagation over the pixel grid. Every pixel
 * holds a 7-D belief (se(3) pose [theta; rho] and log-depth) in information form
 * (Sec. 3.3, Sec. 3.4); factors are the photometric factor (Eq. 3, warp of Eq. 2,
 * Huber by covariance weighting, Sec. 4.1), a pose prior (Eq. 4), a log-depth
 * prior (Sec. 3.3), camera-motion identity factors between 4-neighbours (Eq. 5,
 * grid pattern) and normal-integration factors between 4-neighbours (Eq. 6).
 * One sweep linearises every factor at the current means, sends all
 * factor-to-variable messages at once, damps them, updates the beliefs and
 * moves the linearisation point, projecting stored messages onto the new
 * tangent space (Sec. 4.1). A frame's pose is the pixel average of the pose
 * components (App. C.2, estimator equation); keyframes are re-anchored by a
 * count rule (Sec. 3.5, App. A).
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers (CUDA global memory of the device
 *    that was current when the handle was created); h_* and plain arrays are
 *    host pointers. The library never takes ownership of caller memory.
 *  - Images are row-major, width x height, no padding, float32.
 *  - Work is enqueued on the handle's stream; only calls documented as
 *    synchronising wait for it. Device input buffers must stay valid and
 *    unmodified until the enqueued work has consumed them.
 *  - The library allocates no device memory: all device state lives in the
 *    caller-provided workspace. It launches only its own kernels and plain
 *    cudaMemcpyAsync / cudaMemsetAsync on the handle's stream.
 *  - A handle is not thread-safe; use one handle per host thread or serialise.
 *  - Errors: calls return a pixvod_status. PIXVOD_EINVAL leaves the handle
 *    unchanged. PIXVOD_ECUDA reports a CUDA runtime error (the handle may then
 *    be unusable). Numerical trouble inside kernels never traps: it sets sticky
 *    flags read by pixvod_get_status.
 */
#ifndef PIXVOD_H
#define PIXVOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIXVOD_ABI_VERSION 1

typedef enum {
    PIXVOD_OK = 0,
    PIXVOD_EINVAL = 1,   /* bad argument: null or misaligned pointer, bad size, sigma <= 0 ... */
    PIXVOD_ECUDA = 2,    /* a CUDA runtime call failed */
    PIXVOD_ENUMERIC = 3, /* device flags report a numerical failure (see flags below) */
    PIXVOD_ESTATE = 4,   /* call not valid in the handle's current state */
    PIXVOD_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    PIXVOD_ENOMEM = 6    /* workspace smaller than pixvod_workspace_bytes */
} pixvod_status;

/* Sticky device flags (bitwise OR), read with pixvod_get_status. */
#define PIXVOD_FLAG_NONPOS_PIVOT 0x1u /* a Cholesky pivot was <= 0; that pixel skipped its update */
#define PIXVOD_FLAG_NONFINITE    0x2u /* a non-finite mean was produced */
#define PIXVOD_FLAG_TIMEOUT      0x4u /* a bounded spin-wait gave up */
#define PIXVOD_FLAG_BOUNDS       0x10u /* checked build only: an index left its buffer (access skipped) */

/* Checked build. libpixvod_checked.so is the same library compiled with
 * PIXVOD_CHECKED: every index the sweep computes (neighbour state, input
 * planes, bilinear taps, shared-memory message slots) is tested against its
 * buffer, a violation sets PIXVOD_FLAG_BOUNDS and skips the access (nothing
 * traps), and the lanes of ragged state tiles outside the image are filled with
 * NaN at creation so that any read of them shows as PIXVOD_FLAG_NONFINITE. It is
 * meant for tests; results can differ from the plain build by FP32 rounding. */

/* Pinhole intrinsics (Eq. 2): pixel centres at integer coordinates. */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
} pixvod_intrinsics;

/* Factor strengths and schedule. Each sigma enters as Lambda = I / sigma^2
 * (Sec. 4.2). Defaults (pixvod_params_default): the paper's leaf values
 * sigma_D = 5e-3, sigma_P = 1, sigma_R = 4e-4, sigma_N = 1e-3, t_huber = 400
 * (Sec. 4.2); sigma_Z = 1 (log-depth prior, not given by the paper);
 * damping = 0.5 (pairwise message damping, not in the paper); kf_interval = 10
 * (frames per keyframe segment; the paper uses 150-300 on its 10x-upsampled
 * sequences, App. A); precision = 32. */
typedef struct {
    float sigma_D;     /* photometric noise (intensities in [0, 1]) */
    float sigma_P;     /* pose prior */
    float sigma_R;     /* camera-motion identity factor */
    float sigma_N;     /* normal-integration factor */
    float sigma_Z;     /* log-depth prior */
    float t_huber;     /* Huber threshold on |r| / sigma_D */
    float damping;     /* beta in m <- (1 - beta) m_new + beta m_old, in [0, 1) */
    int32_t kf_interval; /* frame k > 0 with k % kf_interval == 0 becomes a keyframe; 0 = never */
    int32_t precision;   /* arithmetic and state precision: 32 (float) or 64 (double) */
    int32_t topology;    /* identity factors: PIXVOD_TOPOLOGY_GRID (0, default) or _QUADTREE (1) */
    int32_t reserved[6]; /* must be zero */
} pixvod_params;

/* Camera-motion identity factor patterns (Eq. 5).
 * GRID: between every pair of horizontally or vertically adjacent pixels.
 * QUADTREE: the hierarchical pattern of the paper's main experiments (Sec. 3.3
 *   factor graph): a pose node per 2x2 block of pixels (level 1), per 2x2 block
 *   of level-1 nodes (level 2), ... up to one root; each pixel or node is joined
 *   to its parent only, the factor between levels l - 1 and l with sigma_R / 2^(l-1),
 *   and a level-l node carries a pose prior with sigma_P / 2^l (Sec. 4.2: both
 *   halved per level). An image of w x h has ceil(w / 2^l) x ceil(h / 2^l) nodes at
 *   level l. The normal-integration factors stay on the pixel grid. A quadtree
 *   handle stores its pixel state in the same layout (identity slot 0 holds the
 *   message from the parent, slots 1..3 are zero); its checkpoints append the
 *   node states (pixvod_save_state). The adjoint (pixvod_set_recording) returns
 *   ESTATE for a quadtree handle, and batches take grid handles only. */
#define PIXVOD_TOPOLOGY_GRID 0
#define PIXVOD_TOPOLOGY_QUADTREE 1

typedef struct pixvod_handle pixvod_handle;

/* Timing collected while profiling is enabled (pixvod_set_profiling). */
typedef struct {
    int64_t sweep_launches;   /* sweep-kernel launches timed */
    double sweep_ms;          /* summed CUDA-event time of those launches */
    int64_t kernel_launches;  /* all kernels this handle launched since enabling */
} pixvod_profile;

/* Static description of the library (no CUDA calls). */
const char* pixvod_status_string(pixvod_status s);
int pixvod_abi_version(void);
pixvod_params pixvod_params_default(void);

/* Bytes of device workspace a handle needs for these intrinsics and params
 * (no CUDA calls). EINVAL for invalid intrinsics or params. */
pixvod_status pixvod_workspace_bytes(const pixvod_intrinsics* K, const pixvod_params* p,
                                     size_t* out_bytes);

/* Bytes per pixel of the per-sweep state the sweep kernel reads and writes
 * (one copy), for the given precision (32 or 64). No CUDA calls. */
size_t pixvod_state_bytes_per_pixel(int32_t precision);

/* Create a handle. d_workspace: caller-owned device buffer of at least
 * pixvod_workspace_bytes, 256-byte aligned; it must outlive the handle and is not
 * freed by pixvod_destroy. stream: a cudaStream_t (NULL = legacy default
 * stream). Enqueues a memset of the workspace. EINVAL on null or misaligned
 * workspace, invalid intrinsics (fx, fy <= 0, width or height < 2) or params
 * (any sigma <= 0, damping outside [0, 1), precision not 32/64, nonzero
 * reserved, topology not 0/1); ENOMEM if ws_bytes is too small. */
pixvod_status pixvod_create(const pixvod_intrinsics* K, const pixvod_params* p, void* d_workspace,
                            size_t ws_bytes, void* stream, pixvod_handle** out);

/* Release the host-side handle (frees nothing the caller owns). NULL is a no-op. */
pixvod_status pixvod_destroy(pixvod_handle* h);

/* Consume one frame (Sec. 3.5, Sec. 4.3). d_frame: width*height float32 device
 * intensities in [0, 1]. Frame 0 becomes the keyframe (no sweeps). A later
 * frame is the target: n_iters synchronous sweeps run from the previous frame's
 * state, then the pose average is reduced on the device. If the frame index is
 * a multiple of kf_interval, the frame then becomes the next keyframe: the
 * device composes T_cam<-world, resets poses and messages, and sets the log-depth
 * and its prior mean to the segment's mean log-depth. d_normals (width*height*3
 * float32 camera-frame unit normals of this frame, or NULL) is required exactly
 * when the frame becomes a keyframe (EINVAL otherwise, nothing enqueued).
 * n_iters >= 0. Asynchronous; capturable in a CUDA graph (no host sync). */
pixvod_status pixvod_track(pixvod_handle* h, const float* d_frame, const float* d_normals,
                           int32_t n_iters);

/* As pixvod_track, with host inputs: the frame (and normals, when given) are
 * copied into the workspace's staging buffers with cudaMemcpyAsync first. Host
 * buffers must stay valid until the stream has passed the copies (pinned host
 * memory makes the copies asynchronous). */
pixvod_status pixvod_track_host(pixvod_handle* h, const float* h_frame, const float* h_normals,
                                int32_t n_iters);

/* Run n_iters more sweeps on the current target frame and reduce the pose again
 * (no new frame, no keyframe decision). ESTATE before the first target frame. */
pixvod_status pixvod_sweep(pixvod_handle* h, int32_t n_iters);

/* xi_est of the last frame relative to the keyframe it was tracked against,
 * [theta; rho] (App. C.2). Synchronises the stream. */
pixvod_status pixvod_get_pose(pixvod_handle* h, double xi[6]);

/* T_cam<-world of the last frame, 4x4 row-major; the world frame is the first
 * keyframe's camera. Synchronises the stream. */
pixvod_status pixvod_get_pose_global(pixvod_handle* h, double T[16]);

/* Asynchronous copy of xi_est (6 doubles) to device memory. */
pixvod_status pixvod_get_pose_device(pixvod_handle* h, double* d_xi);

/* Depth exp(mu_6) (resp. inverse depth exp(-mu_6)) of every keyframe pixel,
 * width*height float32 into caller device memory. Asynchronous. */
pixvod_status pixvod_get_depth(pixvod_handle* h, float* d_depth);
pixvod_status pixvod_get_inv_depth(pixvod_handle* h, float* d_inv_depth);

/* Sticky device flags (PIXVOD_FLAG_*). Synchronises the stream. Returns
 * ETIMEOUT when PIXVOD_FLAG_TIMEOUT is set (a bounded wait gave up: the sweep
 * that set it stopped early, so the state is not a sweep result and should be
 * reloaded from a checkpoint or re-anchored), else ENUMERIC when any other flag
 * is set, OK otherwise. */
pixvod_status pixvod_get_status(pixvod_handle* h, uint32_t* flags);

/* Checkpoint of the full sweep state: a 256-byte header, the state planes, the
 * input planes and the device scalars. Header (little-endian int64 words):
 *   [0] magic 0x50495856  [1] version 1  [2] precision (32/64)  [3] width
 *   [4] height  [5] pitch (elements per plane row)  [6] state planes (151)
 *   [7] frame index  [8] byte offset of the planes  [9] byte offset of the scalars
 *   [10] input planes (6)  [11] 1 if a target frame is loaded
 *   [12] quadtree nodes n (0 for the grid topology)  [13] node planes (162 for
 *   the quadtree topology, else 0)  [14] byte offset of the node planes (0 for
 *   the grid topology); words 15..31 are zero
 * Each plane is height*pitch elements of the state precision. State planes:
 *   0..6     mu: xi_0..xi_5 (theta, rho), log-depth
 *   7..27    M_p: pose information of the belief without the photometric factor
 *            (pose prior plus identity messages), 6x6 lower triangle packed row
 *            by row ((0,0),(1,0),(1,1),(2,0),...)
 *   28..33   u: the depth-marginalised pose information of the belief is
 *            P = M_p + u u^T
 *   34       s: pose-marginalised log-depth information of the belief
 *   35+27k.. identity-factor message into the pixel from slot k (k = 0 left,
 *            1 right, 2 up, 3 down): 21 packed Lambda then 6 eta
 *   143+2k.. normal-integration message from slot k: Lambda, eta
 * Input planes: keyframe intensity I_s, target intensity I_t, its gradients
 * g_x, g_y, normal-integration edge measurements m_x (to the right neighbour),
 * m_y (to the lower neighbour).
 * Scalars (doubles): xi_est[6], T_kf[16] (T_kf<-world), T_cur[16], d_prior,
 * d_mean.
 * Quadtree handles then hold 162 node planes of n elements each (state
 * precision), nodes numbered level by level from level 1, row-major within a
 * level. Node planes:
 *   0..5     pose of the node (theta, rho)
 *   6..26    belief information: level prior plus the damped messages, packed
 *   27+27k.. identity-factor message into the node from slot k (k = 0..3 the
 *            children, 2 (row % 2) + col % 2; k = 4 the parent): 21 packed
 *            Lambda then 6 eta
 * pixvod_state_size returns the byte count. save and load synchronise the
 * stream (the library's internal state layout differs from this format and is
 * converted on the host); load restores the frame index. EINVAL on a size,
 * magic or geometry mismatch. */
pixvod_status pixvod_state_size(pixvod_handle* h, size_t* bytes);
pixvod_status pixvod_save_state(pixvod_handle* h, void* h_buf, size_t bytes);
pixvod_status pixvod_load_state(pixvod_handle* h, const void* h_buf, size_t bytes);

/* Per-kernel timing: when enabled, CUDA events are recorded around every sweep
 * launch on the handle's stream; pixvod_get_profile synchronises and returns
 * the totals since enabling. */
pixvod_status pixvod_set_profiling(pixvod_handle* h, int32_t enable);
pixvod_status pixvod_get_profile(pixvod_handle* h, pixvod_profile* out);

/* Number of kernels this handle has launched since creation. */
pixvod_status pixvod_launch_count(pixvod_handle* h, int64_t* out);

/* ---------------------------------------------------------------------------
 * Adjoint of the unrolled sweeps of one frame (reverse-mode derivative).
 *
 * With recording on, pixvod_track of a target frame also stores the state every
 * `checkpoint_every` sweeps. pixvod_backward then differentiates a loss
 * L(xi_est, inverse depth) of that frame's result through its n_iters sweeps
 * (Eqs. 2-6 with relinearisation, damping, the belief solve, the mean update
 * and the tangent projection of Sec. 3.4), recomputing each segment of sweeps
 * from its checkpoint with the sweep kernel, which then also records each
 * pixel's discrete decisions (warp validity, Huber branch, skipped update) so
 * that the derivative follows the branches the forward took. Gradients are
 * truncated at the frame start: the state carried from earlier frames is a
 * constant.
 * Two reverse passes exist (pixvod_set_backward_method):
 *   PIXVOD_ADJOINT_HANDWRITTEN (default): the hand-written reverse pass, in the
 *     handle's precision (FP32 or FP64), no tape, in stages with one thread per
 *     pixel or per pixel and direction;
 *   PIXVOD_ADJOINT_TAPE: a reverse-mode tape of the same update in FP64 (about
 *     230 KB of tape per pixel and sweep, a 10 GB workspace at 320x240), kept to
 *     cross-check the hand-written pass.
 * ------------------------------------------------------------------------- */
#define PIXVOD_ADJOINT_HANDWRITTEN 0
#define PIXVOD_ADJOINT_TAPE 1

/* Device bytes of the recording workspace for frames of at most max_iters
 * sweeps (>= 1) with a checkpoint every checkpoint_every (>= 1) sweeps, for the
 * hand-written reverse pass (no CUDA calls). checkpoint_every = 1 keeps every
 * intermediate state of the frame (max_iters - 1 states, written by the sweeps
 * themselves, no copies) and every sweep's decisions, so that pixvod_backward
 * recomputes nothing; larger values keep one state per checkpoint_every sweeps
 * and pixvod_backward recomputes each segment from its checkpoint (the same
 * bits). */
pixvod_status pixvod_backward_workspace_bytes(const pixvod_intrinsics* K, const pixvod_params* p,
                                              int32_t max_iters, int32_t checkpoint_every, size_t* out_bytes);

/* The same for the tape reverse pass (its tapes are sized by the device's SM
 * count, which this queries). */
pixvod_status pixvod_backward_tape_workspace_bytes(const pixvod_intrinsics* K, const pixvod_params* p,
                                                   int32_t max_iters, int32_t checkpoint_every, size_t* out_bytes);

/* Choose the reverse pass (PIXVOD_ADJOINT_*). Call before pixvod_set_recording,
 * whose workspace must then be sized by the matching query; ESTATE while
 * recording is on, EINVAL for an unknown method. */
pixvod_status pixvod_set_backward_method(pixvod_handle* h, int32_t method);

/* Turns recording on (d_workspace: 256-byte aligned caller device memory of at
 * least pixvod_backward_workspace_bytes, owned by the caller and valid while
 * recording is on) or off (d_workspace NULL). While on, pixvod_track of a
 * target frame with more than max_iters sweeps returns EINVAL. */
pixvod_status pixvod_set_recording(pixvod_handle* h, void* d_workspace, size_t ws_bytes, int32_t max_iters,
                                   int32_t checkpoint_every);

/* Gradients of L through the last tracked frame's sweeps. Inputs (device,
 * FP64): d_grad_xi = dL/dxi_est (6, or NULL for 0), d_grad_invdepth =
 * dL/d(exp(-mu_6)) per keyframe pixel (width*height row-major, or NULL for 0).
 * Outputs (device, FP64, overwritten): d_grad_sigmas = dL/d(sigma_D, sigma_N)
 * (2), d_grad_Is = dL/d(keyframe intensities) and d_grad_It = dL/d(target
 * frame intensities) (width*height row-major each). check (host, optional,
 * 2 doubles): the largest difference between the reverse pass's own
 * recomputation of a pixel update and the sweep kernel's result, relative to
 * the magnitude of the output (at least 1; for the hand-written pass, also
 * against its block's scale, that of a 6 x 6 solve's rounding: sqrt(|A_rr A_cc|)
 * for entry (r, c) of M_p or of a message's Lambda, the largest stored entry for
 * an entry of xi, u or a message's eta; and the projected messages
 * eta - Lambda tau against |eta| + |Lambda tau|, whose rounding they carry), and
 * (tape pass) the longest tape. Synchronises the stream.
 * ESTATE if recording is off or the last call was not a non-anchoring target
 * frame tracked with recording on; ENUMERIC if a pixel's tape overflowed, or if
 * that recomputation differs by more than PIXVOD_RECOMPUTE_TOL_FP32 (FP32
 * arithmetic) or PIXVOD_RECOMPUTE_TOL_FP64 (FP64): the gradients then belong to
 * a different update than the one the forward ran. In FP64 the recomputation
 * is exact to rounding (about 1e-12 at 320x240); in FP32 two evaluations of the
 * same update differ by rounding (measured up to about 1e-3 at 320x240). */
#define PIXVOD_RECOMPUTE_TOL_FP32 1e-2
#define PIXVOD_RECOMPUTE_TOL_FP64 1e-9
pixvod_status pixvod_backward(pixvod_handle* h, const double* d_grad_xi, const double* d_grad_invdepth,
                              double* d_grad_sigmas, double* d_grad_Is, double* d_grad_It, double* check);

/* Differentiate only the last `last_sweeps` sweeps of a recorded frame in
 * pixvod_backward (0, the default, = all of them): the state before them is
 * treated as a constant, a truncation of the unrolled derivative. On inputs where
 * the sweep map expands, the full unrolled derivative grows roughly geometrically
 * with the number of sweeps and a short window keeps it bounded. EINVAL if
 * last_sweeps < 0. */
pixvod_status pixvod_set_backward_window(pixvod_handle* h, int32_t last_sweeps);

/* ---------------------------------------------------------------------------
 * Batches: many independent sequences (each with its own intrinsics, image size
 * and state, all with the same params) advanced together, one frame per call.
 * Each sequence's results are bit-identical to tracking it alone with
 * pixvod_track; only the scheduling of the work differs:
 *   PIXVOD_SCHED_PLAIN       every sequence runs its own launches in turn;
 *   PIXVOD_SCHED_BATCHED     one launch per sweep covers the tiles of all
 *                            sequences;
 *   PIXVOD_SCHED_PERSISTENT  one cooperative launch per frame runs all sweeps of
 *                            all sequences, blocks meeting at a bounded grid
 *                            barrier between sweeps (blocks_per_sm resident
 *                            blocks per SM, 1..4).
 * Sequences of the quadtree topology (params.topology) batch too: under
 * PIXVOD_SCHED_BATCHED a sweep is one launch of each of the three quadtree
 * kernels (pixels, node messages, node beliefs) for all sequences; the
 * persistent schedule is for the grid only (a quadtree sweep is three dependent
 * launches).
 * The keyframe count rule applies to the batch's frame index.
 * --------------------------------------------------------------------------- */
typedef struct pixvod_batch pixvod_batch;

#define PIXVOD_SCHED_PLAIN 0
#define PIXVOD_SCHED_BATCHED 1
#define PIXVOD_SCHED_PERSISTENT 2

/* Device workspace bytes for n sequences with intrinsics K[0..n-1]. No CUDA calls. */
pixvod_status pixvod_batch_workspace_bytes(int32_t n, const pixvod_intrinsics* K, const pixvod_params* p,
                                           size_t* out_bytes);

/* Create a batch on a caller-owned 256-byte aligned workspace (as pixvod_create).
 * The schedule starts as PIXVOD_SCHED_PERSISTENT with 4 blocks per SM (grid
 * sequences, where the device supports cooperative launches), else
 * PIXVOD_SCHED_BATCHED.
 * Synchronises the stream. EINVAL / ENOMEM as pixvod_create; n >= 1. */
pixvod_status pixvod_batch_create(int32_t n, const pixvod_intrinsics* K, const pixvod_params* p, void* d_workspace,
                                  size_t ws_bytes, void* stream, pixvod_batch** out);
pixvod_status pixvod_batch_destroy(pixvod_batch* b);

/* Register the input buffers: d_frames[i] (width_i*height_i float32) and
 * d_normals[i] (width_i*height_i*3 float32, read at keyframes) are device
 * pointers, arrays of n host entries. Every pixvod_batch_track call reads them
 * (so a captured CUDA graph of pixvod_batch_track can be replayed after the
 * caller writes new frames into the same buffers). May be called again to point
 * at other buffers. EINVAL on a null or misaligned pointer. */
pixvod_status pixvod_batch_set_inputs(pixvod_batch* b, const float* const* d_frames, const float* const* d_normals);

/* Advance every sequence by one frame from the registered buffers (semantics of
 * pixvod_track). Asynchronous; ESTATE before pixvod_batch_set_inputs. */
pixvod_status pixvod_batch_track(pixvod_batch* b, int32_t n_iters);

/* xi_est of every sequence, 6 doubles per sequence into host memory. Synchronises. */
pixvod_status pixvod_batch_get_poses(pixvod_batch* b, double* xi);

/* OR of every sequence's device flags and the batch's own. Synchronises; ETIMEOUT
 * when PIXVOD_FLAG_TIMEOUT is set, else ENUMERIC when any flag is set. */
pixvod_status pixvod_batch_get_status(pixvod_batch* b, uint32_t* flags);

/* Checkpoint of sequence i, in the pixvod_save_state format. Synchronises. */
pixvod_status pixvod_batch_state_size(pixvod_batch* b, int32_t i, size_t* bytes);
pixvod_status pixvod_batch_save_state(pixvod_batch* b, int32_t i, void* h_buf, size_t bytes);

/* Choose the schedule (and blocks per SM for the persistent one, 1..4, clamped
 * to what the device can hold resident). EINVAL on an unknown schedule, and on
 * the persistent one for quadtree sequences. */
pixvod_status pixvod_batch_set_schedule(pixvod_batch* b, int32_t schedule, int32_t blocks_per_sm);
pixvod_status pixvod_batch_get_schedule(pixvod_batch* b, int32_t* schedule, int32_t* blocks_per_sm);

/* Autotuner: times every schedule (plain, batched, persistent with 2, 3 and 4
 * blocks per SM) on `reps` runs of n_iters sweeps, each sequence tracking its
 * keyframe against itself, keeps the fastest, and restores every sequence's
 * keyframe state. Valid right after the first pixvod_batch_track (frame index 1)
 * while the registered frame buffers still hold the keyframes (ESTATE
 * otherwise). Synchronises. times_ms (optional, 5 entries) receives the mean
 * time per run of each candidate in that order (-1 for a candidate not tried:
 * more blocks per SM than the device holds, or any persistent one for quadtree
 * sequences). */
pixvod_status pixvod_batch_autotune(pixvod_batch* b, int32_t n_iters, int32_t reps, float* times_ms);

/* Kernels the batch has launched since creation. */
pixvod_status pixvod_batch_launch_count(pixvod_batch* b, int64_t* out);

/* Bounded waits of the persistent schedule (diagnostics and tests of the failure
 * path). The grid barrier between sweeps polls an arrival counter; after `polls`
 * polls (each followed by a ~64 ns sleep) a block gives up, sets
 * PIXVOD_FLAG_TIMEOUT and leaves the launch, and the batch's status becomes
 * ETIMEOUT. polls = 0 restores the default of 2^24 (about a second). EINVAL if
 * polls < 0. */
pixvod_status pixvod_batch_set_wait_limit(pixvod_batch* b, int64_t polls);

/* Test hook for the failure path: while `on` is nonzero, every persistent launch
 * starts its grid barrier's arrival counter at 2^24 instead of 0, above any grid
 * size, so no arrival is ever counted as the last one and every block's bounded
 * wait runs out (nothing faults and nothing hangs; the blocks return). The
 * frame's state is then invalid.
 * Plain and batched schedules have no grid barrier and are unaffected. */
pixvod_status pixvod_batch_inject_barrier_fault(pixvod_batch* b, int32_t on);

/* Pose average without any device allocation. The paper has no counterpart: this
 * is a library convenience for callers that cannot allocate device memory, such
 * as code that runs while a CUDA stream is being captured, a real-time loop that
 * forbids allocation after start-up, or a plugin whose host framework owns all
 * device memory and offers it no workspace. It computes the seven means the
 * tracker's own reduction computes (xi_est[0..5] and the mean log-depth), equal to
 * them up to FP64 rounding: here rows are summed in row order, the tracker sums
 * 32 x 4 tiles in tile order, both with double accumulation. The inputs are
 * caller-provided planes; the scratch is a static device array of the library
 * instead of a workspace.
 *   d_mu: 7 float32 planes (xi_0..xi_5, log-depth) of height rows of `pitch`
 *         elements, `plane_stride` elements apart (the checkpoint plane layout);
 *   d_out: 7 doubles of device memory (the means); stream: a cudaStream_t.
 * Limits and behaviour: height at most PIXVOD_STATIC_MAX_ROWS (4096); larger
 * heights return EINVAL without touching the device. The static scratch
 * (4096 x 7 doubles + a counter, about 229 KB) is held by every GPU that loads
 * the library until the process exits. The first call on a device resolves the
 * scratch's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture. Every call on a device shares the
 * same scratch: calls whose kernels overlap on the GPU (different streams, no
 * ordering between them) race and give wrong results. The call clears the part
 * of the scratch that must start at zero (an asynchronous cudaMemsetAsync on the
 * stream) and then launches one kernel; it calls no cudaMalloc or cudaFree.
 * EINVAL on null or misaligned pointers, pitch < width, plane_stride <
 * pitch * height or a height out of range; ECUDA on a CUDA error. */
#define PIXVOD_STATIC_MAX_ROWS 4096
pixvod_status pixvod_pose_mean_static(const float* d_mu, int32_t width, int32_t height, int64_t pitch,
                                      int64_t plane_stride, double* d_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PIXVOD_H */
