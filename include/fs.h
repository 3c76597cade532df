/*
 * fs.h -- C ABI of the GB300 non-rectified variational fisheye stereo library
 * (Roxas & Oishi, "Real-Time Variational Fisheye Stereo without Rectification
 * and Undistortion").
 *
 * The library estimates, for a calibrated fisheye pair, the scalar disparity
 * u along the epipolar curves (Sec. III-A) and the range it implies
 * (Sec. III-D) directly on the distorted images: per pyramid level it builds
 * the trajectory field of epipolar tangents (Sec. III-B, Eq. 6-7), warps the
 * second image along it (Eq. 9), linearises the data term along the field
 * (Eq. 3, 5) and runs primal-dual iterations of a tensor-weighted (Eq. 12)
 * Huber-TV-L1 energy (Eq. 11, 13), inside the warping loop of Algorithm 1
 * and the coarse-to-fine scheme of Sec. IV-B, after the pre-rotation of
 * Sec. IV-A.
 *
 * Conventions shared by every entry point
 *   - Images are float32 in [0, 1], row-major, pitch = width (no padding),
 *     pixel centres on integer coordinates, (0, 0) the top-left pixel.
 *   - Device pointers point to memory of the device that was current when the
 *     handle was created; the caller owns them.  The library owns the per-rig
 *     state it allocates in fs_create and frees it in fs_destroy.
 *   - All GPU work of a handle is issued on the CUDA stream given to
 *     fs_create (NULL = the legacy default stream) and is asynchronous unless
 *     stated; the caller synchronises that stream before reading results.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - Errors are returned as fs_status, never thrown; fs_last_error() gives a
 *     message for the last failing call of the calling thread.
 *   - Outside the FOV mask, disparity is 0 and depth is NaN; where the two
 *     rays are parallel the depth is +inf.
 */
#ifndef FS_H
#define FS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FS_OK = 0,
  FS_EINVAL = -1,    /* bad argument (null pointer, size, level, count)      */
  FS_ENOMEM = -2,    /* device allocation failed                             */
  FS_ECUDA = -3,     /* a CUDA call or kernel launch failed                  */
  FS_ECALIB = -4,    /* calibration rejected (e.g. non-monotone r(theta))    */
  FS_ETIMEOUT = -5,  /* a bounded wait ran out                               */
  FS_ECANCELLED = -6 /* the request was cancelled before it ran (server)     */
} fs_status;

/* Host-side fault injection for tests: while the environment variable
 * FS_FAULT_ALLOC is "all" or names an allocation site -- "arena" (the
 * per-handle state of fs_create), "guard" (guard-band bookkeeping),
 * "stage" (fs_solve_host's staging planes), "sched" (the accelerated
 * schedule's table), "energy" (fs_energy's accumulators), "planes" (a served
 * rig's image and output planes) -- that device allocation fails without
 * reaching the device, and the call returns FS_ENOMEM. */

/* Radially symmetric camera models, pixel = c + f * r(theta) * (X, Y)/|(X, Y)|
 * with theta the angle off the optical axis (Sec. III-B allows any model
 * with a defined projection and cites the unified, enhanced unified and
 * Kannala-Brandt models; Sec. III-D notes the closed-form unprojections of
 * the first two).  With s = sin(theta), c = cos(theta):
 *   unified (xi = k[0]):              r = s / (c + xi)
 *   enhanced unified (alpha = k[0], beta = k[1]):
 *                                     r = s / (alpha sqrt(beta s^2 + c^2) + (1 - alpha) c)
 * i.e. the usual forms m = (X, Y) / (Z + xi |X|) and
 * m = (X, Y) / (alpha sqrt(beta (X^2 + Y^2) + Z^2) + (1 - alpha) Z). */
typedef enum {
  FS_PINHOLE = 0,          /* r = tan(theta)                                  */
  FS_EQUIDISTANT = 1,      /* r = theta                                       */
  FS_KANNALA_BRANDT = 2,   /* r = theta + k1 t^3 + k2 t^5 + k3 t^7 + k4 t^9   */
  FS_UNIFIED = 3,          /* r = s / (c + xi),  xi = k[0] >= 0              */
  FS_ENHANCED_UNIFIED = 4  /* alpha = k[0] in [0, 1), beta = k[1] > 0         */
} fs_model;

typedef struct {
  int model;               /* fs_model                                        */
  double fx, fy;           /* focal lengths, pixels                           */
  double cx, cy;           /* principal point, pixels                         */
  double k[4];             /* model parameters (see fs_model; unused = 0)     */
  double fov_deg;          /* full field of view; the mask keeps theta <= fov/2 */
} fs_calib;

/* Rig pose exp(xi_1) of Sec. III-A: X_cam1 = R X_cam0 + t, R row-major. */
typedef struct {
  double R[9];
  double t[3];
} fs_pose;

/* Solver parameters.  beta, eta: Eq. 12 (paper values 9.0, 0.85, Sec. IV-C);
 * du_max: the per-warp clip of delta-u (0.2 px, Sec. IV-C); lambda (data
 * weight) and huber_eps are not stated by the paper.  theta is the
 * over-relaxation of Eq. 11 (1 = Chambolle-Pock Algorithm 1).  precond = 1
 * uses diagonal preconditioning (Pock-Chambolle 2011, alpha = 1), 0 uses
 * tau = sigma = 1/sqrt(8).  block_iters: primal-dual iterations fused per
 * launch by temporal blocking (1..8; 0 = library default).  use_graph = 1
 * captures a solve into a CUDA graph on first use and replays it.
 * pd_schedule: 0 = automatic (levels up to 128 x 128 run all iterations of
 * a warp in one launch of a thread-block cluster holding the whole level,
 * when the GPU can host that cluster; larger levels use temporal blocking),
 * 1 = temporal blocking on every level, FS_SCHED_PERSISTENT (2) = the
 * persistent schedule: after the pre-rotation and the pyramid, every level
 * and warp of a cold solve -- and, in fs_batch_solve, of every pair of the
 * batch -- runs in one persistent launch over a device work list of
 * (pair, level, tile, step) items, each tile waiting only on its neighbours
 * (footprints and depths from fs_autotune's choices).  It needs the Huber-TV
 * regulariser and accel_gamma = 0; warm starts and continuations of such a
 * handle use temporal blocking.  A solve in this schedule waits for its
 * work to finish and returns FS_ETIMEOUT if a wait of the launch ran out
 * (fs_set_wait_limit).  All three give identical results.
 * storage: 0 = FP32; 1 = FP16, 2 = BF16 storage of the images, the warped
 * gradient and residual (I_u, rho0), the tensor T^1/2 and the dual field p,
 * while the disparity (u, u_omega), the warp vector and every operation stay
 * FP32 (values are rounded to nearest when stored).
 * regularizer: FS_REG_HUBER_TV (0) = lambda |rho| + h_eps(T^1/2 grad u), the
 * first-order member of Eq. 10; FS_REG_TGV (1) = the paper's tensor-guided
 * TGV-L1 energy of Eq. 10, lambda |rho| + alpha1 |T^1/2 grad u - v| +
 * alpha0 |grad v| (alpha0 = 17, alpha1 = 1.2 in Sec. IV-C; huber_eps and
 * pd_schedule do not apply; block_iters is the temporal-blocking depth, 0 =
 * tuned or 4), solved by the primal-dual steps of Eq. 11 with diagonal
 * preconditioning; FP32 storage only.
 * deriv: how I_u, the derivative of the warped I1 along the trajectory, is
 * taken.  FS_DERIV_FORWARD (0) = I1(x + w + g) - I1(x + w), the difference of
 * Eq. 7 (g the unit tangent gamma'); FS_DERIV_CENTRAL (1) = half of
 * I1(x + w + g) - I1(x + w - g), exact on a quadratic image and free of the
 * sample I1(x + w) that Eq. 7 shares with the residual rho0, whose noise
 * otherwise biases every warp's step towards +u.
 * accel_gamma: 0 = constant steps and relaxation theta.  > 0 = the step
 * schedule of Chambolle-Pock's Algorithm 2, which Sec. IV-C's "theta updated
 * every iteration" names: iteration k of a warp uses tau_k, sigma_k and
 * theta_k = 1 / sqrt(1 + 2 accel_gamma tau_k), then tau_{k+1} = theta_k
 * tau_k, sigma_{k+1} = sigma_k / theta_k, from tau_0 = sigma_0 = 1/sqrt(8)
 * at every warp (theta is then unused).  Needs precond = 0, the Huber-TV
 * regulariser and FP32 storage (else FS_EINVAL).  The L1 data term is not
 * uniformly convex, so the schedule carries no rate guarantee here. */
#define FS_REG_HUBER_TV 0
#define FS_REG_TGV 1
#define FS_SCHED_PERSISTENT 2
#define FS_DERIV_FORWARD 0
#define FS_DERIV_CENTRAL 1
typedef struct {
  float lambda;
  float huber_eps;
  float du_max;
  float beta;
  float eta;
  float theta;
  int precond;
  int block_iters;
  int use_graph;
  int pd_schedule;
  int storage;
  int regularizer;         /* FS_REG_HUBER_TV or FS_REG_TGV                   */
  float alpha0, alpha1;    /* TGV weights (regularizer = FS_REG_TGV)          */
  int deriv;               /* FS_DERIV_FORWARD or FS_DERIV_CENTRAL            */
  float accel_gamma;       /* 0, or the gamma of the accelerated schedule      */
} fs_params;

typedef struct fs_handle fs_handle;

/* Fill *out with the defaults (lambda 50, eps 0.01, du_max 0.2, beta 9,
 * eta 0.85, theta 1, precond 1, block_iters 0, use_graph 0, Huber-TV,
 * alpha0 17, alpha1 1.2, deriv FS_DERIV_FORWARD, accel_gamma 0).  du_max,
 * beta, eta, alpha0 and alpha1 are the values of Sec. IV-C; the paper
 * states no lambda and no Huber eps.  FS_EINVAL for a null out. */
fs_status fs_default_params(fs_params* out);

/* Create the per-rig state for W x H pairs and `levels` pyramid levels
 * (scale 2 per level, Sec. IV-B/C; level l is ceil(W/2^l) x ceil(H/2^l)).
 * cam[0], cam[1]: calibrations of the two cameras; pose: camera 1 relative
 * to camera 0; prm: NULL for defaults; cuda_stream: a cudaStream_t or NULL.
 * Builds, on the stream, the FOV masks, the calibration field of Sec. IV-A
 * and the trajectory field of every level (Sec. III-B).  Requires
 * 1 <= levels <= 8, every level at least 4 x 4, fx, fy > 0, fov in (0, 360)
 * (< 180 for pinhole), and a Kannala-Brandt r(theta) increasing on
 * [0, fov/2] (else FS_ECALIB).  On success *out owns device memory. */
fs_status fs_create(const fs_calib cam[2], const fs_pose* pose, int W, int H,
                    int levels, const fs_params* prm, void* cuda_stream,
                    fs_handle** out);

/* (No counterpart in the paper: memory planning, as the server's admission
 * by memory budget uses it.)
 * Device bytes fs_create would allocate for a handle of this size, level
 * count and storage (prm NULL = defaults), without allocating: the pyramid's
 * planes (FP32 state, the 16-bit-capable planes in the storage type, float2
 * fields, mask bytes) and the calibration field.  fs_solve_host adds 5
 * planes of W x H floats on its first call.  FS_EINVAL for sizes or levels
 * fs_create rejects. */
fs_status fs_state_bytes(int W, int H, int levels, const fs_params* prm, size_t* out);

/* Replace the pose (exp(xi_1) of Sec. III-A) for the following solves:
 * recomputes, on the handle's stream, the calibration field of Sec. IV-A
 * and the trajectory field of every level (Sec. III-B).  FS_EINVAL for a
 * null pose or a non-finite entry; the previous pose stays in force when
 * the call fails. */
fs_status fs_set_pose(fs_handle* h, const fs_pose* pose);

/* Size of pyramid level `level` (0 = full resolution; each level halves
 * the one above, rounding up, Sec. IV-B).  W or H may be NULL.  FS_EINVAL
 * for a level outside [0, levels). */
fs_status fs_level_size(const fs_handle* h, int level, int* W, int* H);

/* Copy the trajectory field gamma' of a level (Sec. III-B, Eq. 7) to d_out:
 * two planes of H_l x W_l floats, x components then y components.  Unit
 * vectors inside the mask, 0 outside and at epipoles. */
fs_status fs_trajectory_field(fs_handle* h, int level, float* d_out);

/* Run the method on one pair (Algorithm 1 inside the pyramid of Sec. IV-B,
 * after the pre-rotation of Sec. IV-A).  d_I0, d_I1: W x H device images of
 * camera 0 and camera 1.  d_init: NULL to start from u = 0 at the coarsest
 * level; else a W x H disparity (px) to warm-start from, in which case only
 * the finest level runs.  warps >= 1 warps of iters >= 1 primal-dual
 * iterations per level.  d_disp (W x H, px along the epipolar curve) and
 * d_depth (W x H, metres along the camera-0 ray) may be NULL to skip. */
fs_status fs_solve(fs_handle* h, const float* d_I0, const float* d_I1,
                   const float* d_init, int warps, int iters,
                   float* d_disp, float* d_depth);

/* (The paper runs each frame from scratch; this continuation is a serving
 * extension.)  Warm start of the next frame of a video stream from the
 * handle's own last
 * result, with no disparity round trip: the finest level's u and its 2-D
 * correspondence field w, as the last fs_solve / fs_solve_continue of this
 * handle left them, initialise the finest level (u_w = ubar = u, p = 0) and
 * `warps` x `iters` run there, as for a d_init warm start, but w is taken
 * as it was instead of being rebuilt from the disparity along gamma'.
 * FS_EINVAL if the handle holds no result (no solve yet, or fs_autotune /
 * fs_run_stage has run since).  fs_buffer_write of level 0's U and W (in
 * fs_stages.h) replaces the state it continues from. */
fs_status fs_solve_continue(fs_handle* h, const float* d_I0, const float* d_I1, int warps,
                            int iters, float* d_disp, float* d_depth);

/* (No counterpart in the paper: the end-to-end host entry point.)
 * fs_solve from HOST buffers: copies the inputs to the device, solves,
 * copies the outputs back and synchronises the handle's stream before
 * returning.  Host buffers may be pageable or pinned (pinned is faster). */
fs_status fs_solve_host(fs_handle* h, const float* h_I0, const float* h_I1,
                        const float* h_init, int warps, int iters,
                        float* h_disp, float* h_depth);

/* Free the handle and its device memory (synchronises its stream).  A null
 * handle is a no-op.  (No counterpart in the paper.) */
fs_status fs_destroy(fs_handle* h);

/* Message for the last failing call of this thread ("" if none); owned by
 * the library, valid until this thread's next call.  (No counterpart in the
 * paper.) */
const char* fs_last_error(void);

/* ---- Batches: many independent pairs per call -------------------------
 * (No counterpart in the paper, which solves one pair at a time.)
 * A batch groups n handles (each from fs_create: any sizes, calibrations
 * and poses, all on one device) and solves one pair per handle at once.
 * Handle i's work runs on its own internal stream, forked from the batch
 * stream and joined back to it, so the pairs' kernels overlap on the GPU;
 * the whole fork/join schedule is captured into one CUDA graph the first
 * time a set of buffers is seen and replayed afterwards.  Each pair's result
 * is bit-identical to a lone fs_solve of that pair.  A handle may belong to
 * one batch at a time and must not be used alone while a batch solve that
 * includes it is in flight. */
typedef struct fs_batch fs_batch;

/* handles: n >= 1 distinct handles; cuda_stream: the stream the batch's
 * graph is launched on (NULL = legacy default stream). */
fs_status fs_batch_create(fs_handle* const* handles, int n, void* cuda_stream,
                          fs_batch** out);

/* Arrays of n device pointers, as for fs_solve per pair; d_init may be NULL
 * (all cold starts) or hold NULL entries; d_disp / d_depth entries may be
 * NULL.  warps >= 1, iters >= 1 for every pair.  Asynchronous on the batch
 * stream. */
fs_status fs_batch_solve(fs_batch* b, const float* const* d_I0, const float* const* d_I1,
                         const float* const* d_init, int warps, int iters,
                         float* const* d_disp, float* const* d_depth);

/* Bound how many of the batch's pairs run their finest level at the same
 * time: pair i starts its finest level (tensor, upsample, warps) only after
 * pair i - k has finished its own; coarser levels of all pairs still
 * overlap freely.  The finest level's working set (about 60 B per pixel in
 * FP32 storage) is what decides whether concurrent pairs still fit the L2
 * cache, so k = 1 or 2 keeps a 1024x1024 batch L2-resident while its coarse
 * levels, which are latency-bound, run side by side.  k = 0 (the default)
 * sets no bound.  Results are unchanged (each pair's work and order are the
 * same); only the schedule differs.  Takes effect at the next
 * fs_batch_solve, which captures a new graph.  FS_EINVAL for k < 0. */
fs_status fs_batch_set_finest_limit(fs_batch* b, int k);

/* Tune the batch for throughput.  fs_autotune times a pair alone, so it
 * gives the coarse levels (latency-bound) short dependent chains per launch;
 * many pairs sharing the GPU want few, large footprints with little halo
 * instead.  Every handle keeps its own schedule for its two finest levels;
 * for its coarser levels (level 2 and up) this tries, besides every
 * handle's own choices, one common schedule for all pairs from a fixed set
 * (fs_autotune encoding 32, 69, 8, 45), timing `iters` primal-dual
 * iterations on every coarse level of every pair with all pairs at once
 * on the batch's streams, and keeps the fastest (written into the handles,
 * as fs_set_schedule would).  choice (may be NULL): the common coarse
 * choice kept, or -1 for the handles' own.  Results are unchanged (every
 * schedule gives the same bits).  Overwrites the coarse levels' state and
 * synchronises the batch stream; FS_EINVAL for TGV handles or iters < 1.
 * A batch graph is recaptured after any schedule change of its handles. */
fs_status fs_batch_autotune(fs_batch* b, int iters, int* choice);

/* Free the batch (its streams, events and graph; not the handles). */
fs_status fs_batch_destroy(fs_batch* b);

/* ---- For callers that cannot allocate device memory --------------------
 * (The paper has no counterpart: this is a deployment variant.)  A real-time
 * host thread that must not risk the device-wide synchronisation an
 * allocation can cause, a plug-in living inside a framework that owns the
 * whole device memory pool, or a process with a fixed memory cap cannot
 * call cudaMalloc, and fs_create allocates.  fs_pd_iterate_noalloc runs the
 * primal-dual iterations of one warp (the same kernels fs_solve uses:
 * tensor and step sizes, then `iters` iterations of Eq. 11/13) directly on
 * the caller's buffers and allocates nothing: its intermediate planes live
 * in one fixed array compiled into the library, sized for
 * FS_NOALLOC_MAX_PIXELS pixels (53 bytes each, about 13.9 MB), which every
 * GPU that loads the library holds until the process exits.
 *
 *   d_I0    W x H image (the tensor T^1/2 of Eq. 12 is built from it)
 *   d_mask  W x H bytes, nonzero inside the FOV
 *   d_Iu, d_rho0, d_uw  W x H linearisation I_u, rho0 and u_w (Eq. 3, 5)
 *   d_u     W x H disparity, read as the start value and overwritten
 *   d_p     2 x W x H dual variable (x then y plane), read and overwritten
 *   prm     NULL for the defaults; lambda, huber_eps, beta, eta, theta,
 *           precond and block_iters are used; accel_gamma must be 0,
 *           regularizer FS_REG_HUBER_TV and storage 0 (FS_EINVAL
 *           otherwise); deriv plays no part (I_u is given)
 *   cuda_stream  stream for the work (NULL = legacy default stream)
 * All pointers are device pointers, dense row-major (pitch W), owned by
 * the caller.  W, H >= 2, iters >= 1; W * H > FS_NOALLOC_MAX_PIXELS
 * returns FS_EINVAL.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  Every call on a device uses
 * the same array: calls whose work overlaps on the GPU (different streams,
 * or different host threads) race and corrupt each other's results;
 * serialise them.  The array keeps the last call's contents, which no call
 * reads: every plane is written in full before it is used. */
#define FS_NOALLOC_MAX_PIXELS (512 * 512)
fs_status fs_pd_iterate_noalloc(const float* d_I0, const unsigned char* d_mask,
                                const float* d_Iu, const float* d_rho0,
                                const float* d_uw, float* d_u, float* d_p,
                                int W, int H, int iters, const fs_params* prm,
                                void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FS_H */
