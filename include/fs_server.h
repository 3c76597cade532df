/* fs_server.h -- a continuous-batching request server over many stereo rigs.
 *
 * The paper solves one pair at a time on one camera rig (Algorithm 1 in a
 * pyramid, Sec. III-IV) for real-time mapping, and its conclusion (Sec. VI)
 * names initialisation from another estimate as the remedy for large
 * displacements.  This server is a deployment form of the same solver,
 * with no counterpart in the paper: requests (one stereo pair each) arrive
 * from many rigs of different sizes and calibrations, and
 *
 *   - each rig keeps its state resident on the device between requests: the
 *     fs_handle (pyramid planes, FOV masks, calibration and trajectory
 *     fields, Sec. IV-A/IV-B, III-B), its input / output planes and the last
 *     disparity, from which its next frame warm-starts (finest level only,
 *     the disparity's correspondence rebuilt along the trajectory field);
 *   - a rig's first frame, and its first frame after an eviction, is a cold
 *     solve over the whole pyramid;
 *   - requests of one rig run in arrival order, one at a time (they share
 *     that rig's planes); requests of different rigs run concurrently, each
 *     rig on its own CUDA stream, so their kernels overlap on the GPU;
 *   - a request is admitted when (a) fewer than max_inflight requests are on
 *     the GPU, (b) its rig has nothing in flight and no earlier request of
 *     its rig is waiting, and (c) the rig's state is resident or fits the
 *     device-memory budget once idle rigs are evicted, least recently used
 *     first.  A request that cannot be admitted waits; later requests of
 *     other rigs may go ahead of it (no head-of-line blocking across rigs).
 *
 * Each result depends only on its rig's calibration, pose and parameters,
 * its input pair and, for a warm start, the rig's previous disparity; the
 * kernels are deterministic, so a result is bit-identical whether the
 * request ran alone or among others.
 *
 * Latency is measured on the host from fs_server_submit to the moment the
 * result has reached the caller's host buffers (a host callback on the rig's
 * stream after the device-to-host copies).
 *
 * Thread-safety: every fs_server_* call may be made from any thread; one
 * internal dispatcher thread issues all device work.  fs_last_error() holds
 * the message of the calling thread's last failing call; for a request
 * that failed on the dispatcher thread, fs_server_wait returns its status
 * and sets the waiting thread's fs_last_error() to its message.
 */
#ifndef FS_SERVER_H
#define FS_SERVER_H

#include <stddef.h>

#include "fs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fs_server fs_server;

typedef struct {
  size_t hbm_budget;     /* device bytes the rigs' resident state may hold in
                            total (fs_state_bytes of each handle plus 4 planes
                            of W x H floats per rig); 0 = 40 GiB; lowered at
                            creation to the device's free memory less 1 GiB */
  int max_inflight;      /* requests on the GPU at once, >= 1 (default 2: the
                            requests on the GPU share its SMs, so each admitted
                            request stretches the others; at 600 requests/s of
                            the 16-rig load, 2 gave a p99 of 5.0 ms against
                            8.1 ms for 8, at the same saturated rate) */
  int warps, iters;      /* warm-started request: warps x iterations on the
                            finest level */
  int cold_warps, cold_iters;   /* cold request: per pyramid level */
  int warm_mode;         /* how a warm request starts from the rig's last
                            result: 1 = its finest-level u and w as they are
                            (fs_solve_continue); 0 = its disparity, w rebuilt
                            along gamma' (fs_solve with d_init) */
  int autotune;          /* 1: fs_autotune each rig's schedule (for `iters`)
                            when its state is made resident */
  int reserved[2];       /* zero */
} fs_server_config;

typedef struct {
  long long submitted;   /* requests accepted by fs_server_submit */
  long long completed;   /* requests whose result has reached the host */
  long long failed;      /* of those, requests that failed */
  long long cold;        /* requests solved cold (first frame or after eviction) */
  long long evictions;   /* rig states freed to admit another rig */
  long long cancelled;   /* requests cancelled before they ran */
  double p50_ms, p99_ms, max_ms, mean_ms;  /* latency of completed requests */
  double frames_per_s;   /* completed / (last completion - first submission) */
  size_t resident_bytes; /* device bytes of the resident rig states now */
  size_t peak_resident_bytes;
} fs_server_stats;

/* Defaults: 40 GiB budget, 2 in flight, 3 x 50 warm, 10 x 100 cold,
 * warm_mode 1, autotune 1.  FS_EINVAL for a null out. */
fs_status fs_server_default_config(fs_server_config* out);

/* Create a server on the calling thread's current CUDA device.  cfg NULL =
 * defaults.  FS_EINVAL for max_inflight < 1, warps / iters < 1 or a
 * warm_mode other than 0 / 1;
 * FS_ECUDA if no device is usable. */
fs_status fs_server_create(const fs_server_config* cfg, fs_server** out);

/* Register a rig: the arguments of fs_create (prm NULL = defaults; the
 * server forces use_graph = 1 and uses its own stream per rig).  Nothing is
 * allocated until the rig's first request is admitted.  *rig_id receives the
 * rig's index (0, 1, ... in registration order).  FS_ENOMEM if the rig's
 * state alone exceeds the budget; the validation errors of fs_create. */
fs_status fs_server_add_rig(fs_server* s, const fs_calib cam[2], const fs_pose* pose, int W,
                            int H, int levels, const fs_params* prm, int* rig_id);

/* Queue one pair for a rig.  h_I0, h_I1: W x H row-major floats (host
 * memory; pinned memory lets the copies run asynchronously), read when the
 * request is dispatched.  h_disp, h_depth: W x H host outputs, either may be
 * NULL.  All four must stay valid until fs_server_wait for this request has
 * returned.  Never blocks on the device.  *req_id receives the request id. */
fs_status fs_server_submit(fs_server* s, int rig, const float* h_I0, const float* h_I1,
                           float* h_disp, float* h_depth, long long* req_id);

/* Wait up to timeout_s seconds (< 0: no limit) for a request.  On
 * completion returns the request's own status (FS_OK or the error it met),
 * forgets the request, and sets *latency_ms (may be NULL).  FS_ETIMEOUT if
 * it is still pending (it stays known); FS_EINVAL for an unknown id, or
 * while another thread is already waiting for the same request (threads
 * may wait for different requests at once). */
fs_status fs_server_wait(fs_server* s, long long req_id, double timeout_s, double* latency_ms);

/* Cancel a request that is still queued: it will not run, and
 * fs_server_wait returns FS_ECANCELLED for it.  FS_EINVAL for an unknown id
 * or a request already on the GPU or done (it then completes normally).
 * A cancelled warm request of a rig leaves that rig's state as it was, so
 * the rig's next request continues from its last completed frame. */
fs_status fs_server_cancel(fs_server* s, long long req_id);

/* Wait until every submitted request has completed (timeout_s < 0: no
 * limit).  FS_ETIMEOUT if some are still pending. */
fs_status fs_server_drain(fs_server* s, double timeout_s);

/* Counters and latency percentiles since creation or the last reset. */
fs_status fs_server_stats_read(fs_server* s, fs_server_stats* out, int reset);

/* Free every rig's state; the rig stays registered and its next request is
 * solved cold.  Waits for in-flight work. */
fs_status fs_server_evict_all(fs_server* s);

/* Stop the dispatcher, wait for in-flight work, free everything.  Requests
 * still queued are dropped.  No other thread may be inside any fs_server_*
 * call on s (fs_server_wait and fs_server_drain included) when it is called,
 * or call one afterwards: a dropped request never completes, and s is freed.
 * Wait for or drain what you submitted first. */
fs_status fs_server_destroy(fs_server* s);

#ifdef __cplusplus
}
#endif

#endif /* FS_SERVER_H */
