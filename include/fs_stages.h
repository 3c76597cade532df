/*
 * fs_stages.h -- step-by-step access to the per-level state of an fs_handle.
 *
 * fs_solve runs these stages in the order of Algorithm 1; exposing them one
 * at a time lets a caller (a test, a profiler, a custom schedule) set a
 * level's buffers, run a single stage and read the result.  Same
 * conventions as fs.h: dense row-major device buffers (pitch = width of the
 * level), caller-owned, work on the handle's stream.
 *
 * Each stage cites the passage it computes.  The calls after the stages --
 * kernel timing, the autotuner and fs_set_schedule, the energy reduction,
 * the guard-band check, the wait limits -- have no counterpart in the
 * paper: they measure, tune and test the implementation.
 */
#ifndef FS_STAGES_H
#define FS_STAGES_H

#include "fs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Per-level buffers.  "planes" is the number of H_l x W_l float planes a
 * read or write moves (2 = x then y components, 3 = a, b, c). */
typedef enum {
  FS_BUF_I0 = 0,      /* 1: camera-0 image of the level                       */
  FS_BUF_I1 = 1,      /* 1: pre-rotated camera-1 image (Sec. IV-A)            */
  FS_BUF_MASK = 2,    /* 1: FOV mask as 0.0 / 1.0 (read only)                 */
  FS_BUF_GAMMA = 3,   /* 2: trajectory field gamma' (Sec. III-B)              */
  FS_BUF_TENSOR = 4,  /* 3: T^1/2 = [[a, b], [b, c]] (Eq. 12)                 */
  FS_BUF_STEPS = 5,   /* 2: tau, sigma (diagonal preconditioning)             */
  FS_BUF_U = 6,       /* 1: disparity u (px along the curve)                  */
  FS_BUF_UBAR = 7,    /* 1: over-relaxed u (Eq. 11)                           */
  FS_BUF_UW = 8,      /* 1: linearisation point u_omega (Eq. 3)               */
  FS_BUF_P = 9,       /* 2: dual variable p (Eq. 11)                          */
  FS_BUF_W = 10,      /* 2: warp vector w (Eq. 9)                             */
  FS_BUF_IU = 11,     /* 1: I_u, variation of I1 along gamma' (Eq. 5)         */
  FS_BUF_RHO0 = 12,   /* 1: I1(x + w) - I0(x)                                 */
  FS_BUF_G = 13,      /* 2: gamma' at x + w, renormalised (bicubic)           */
  FS_BUF_V = 14,      /* 2: TGV auxiliary field v (Eq. 10; TGV handles only)  */
  FS_BUF_VBAR = 15,   /* 2: over-relaxed v (Eq. 11; TGV handles only)         */
  FS_BUF_Q = 16       /* 4: TGV dual q, rows dv1 (x, y) then dv2 (x, y)       */
} fs_buffer;

typedef enum {
  FS_STAGE_DOWNSAMPLE = 0, /* I0, I1 of `level` -> level + 1 (Sec. IV-B)      */
  FS_STAGE_TENSOR = 1,     /* I0 -> T^1/2 (Eq. 12) and tau, sigma             */
  FS_STAGE_UPSAMPLE = 2,   /* u, w of level + 1 -> level (x2), p <- 0        */
  FS_STAGE_WARP = 3,       /* I0, I1, w, gamma' -> I_u, rho0, g; ubar, u_w <- u (Eq. 3, 5, 9) */
  FS_STAGE_PD = 4,         /* `count` primal-dual iterations (Eq. 11, 13)     */
  FS_STAGE_CLIP = 5,       /* clip delta-u, u_w + du -> u, w += du g (Alg. 1) */
  FS_STAGE_TRAJECTORY = 6, /* rebuild gamma' of the level (Sec. III-B)        */
  FS_STAGE_WARM = 7,       /* warm start from u: w <- walk of u along gamma',
                              ceil(|u|/du_max) equal steps; ubar, u_w <- u, p <- 0 */
  FS_STAGE_CLIP_WARP = 8   /* FS_STAGE_CLIP then FS_STAGE_WARP in one launch (what
                              fs_solve runs between two warps; same results) */
} fs_stage;

/* Copy a level buffer to / from dense device memory of planes x H_l x W_l
 * floats.  FS_BUF_MASK is read-only. */
fs_status fs_buffer_read(fs_handle* h, int level, int buffer, float* d_out);
fs_status fs_buffer_write(fs_handle* h, int level, int buffer, const float* d_in);

/* Run one stage on a level's buffers; `count` is the iteration count of
 * FS_STAGE_PD and ignored by the others. */
fs_status fs_run_stage(fs_handle* h, int level, int stage, int count);

/* Pre-rotate a full-resolution camera-1 image by the calibration field
 * (Sec. IV-A) into the level-0 FS_BUF_I1 buffer. */
fs_status fs_stage_prerotate(fs_handle* h, const float* d_I1);

/* Triangulate level 0 (Sec. III-D): d_disp <- u, d_depth <- range; either
 * may be NULL. */
fs_status fs_stage_depth(fs_handle* h, float* d_disp, float* d_depth);

/* The linearised energy of the current state of `level` (Eq. 10 with the
 * data term of Eq. 3, 5, the handle's regulariser), reduced on the GPU
 * (warp shuffles, FP64 accumulation): out[0] = total, out[1] = data term
 * lam sum_M |rho0 + I_u (u - u_w)|, out[2] = regulariser (Huber-TV:
 * sum h_eps(T^1/2 grad u); TGV: alpha1 sum_M |T^1/2 grad u - v| + alpha0
 * sum |grad v|), out[3] = the L1 residual sum_M |rho0 + I_u (u - u_w)|.
 * Host output; synchronises the handle's stream. */
fs_status fs_energy(fs_handle* h, int level, double out[4]);

/* Kernel timing with CUDA events on the handle's stream.  While enabled,
 * every fs_solve records an event pair around the primal-dual launches of
 * each (level, warp); fs_timing_read synchronises the stream, folds the
 * recorded pairs into per-level totals and returns, for each level l < 8,
 * ms[l] = accumulated primal-dual time, launches[l] = primal-dual kernel
 * launches and pixel_iters[l] = pixel-iterations they processed, since the
 * last reset.  Call it after each solve (a solve reuses the events).
 * reset = 1 clears the totals after reading.  Any output may be NULL. */
fs_status fs_timing_enable(fs_handle* h, int enable);
fs_status fs_timing_read(fs_handle* h, double* ms, long long* launches,
                         double* pixel_iters, int reset);

/* Autotuner of the primal-dual schedule.  For every level, times `iters`
 * iterations (best of 3 after a warm-up, CUDA events on the handle's
 * stream) of each candidate -- the whole-level cluster schedule where the
 * level fits one cluster, and temporal blocking with 1..8 iterations per
 * launch on each of six footprints -- and keeps the fastest for later
 * solves when block_iters = 0 and pd_schedule = 0.  choice (may be NULL) receives per
 * level 0 = cluster, or 8 v + d = depth d (1..8) on footprint v:
 * v = 0: 64 x 64 pixels, 512 threads of 8 rows (choices 1..8);
 * v = 1: 32 x 32, 256 threads of 4 rows (9..16);
 * v = 2: 64 x 32, 256 threads of 8 rows (17..24);
 * v = 3: 64 x 64, 1024 threads of 4 rows (25..32);
 * v = 4: 32 x 32, 1024 threads of 1 row (33..40);
 * v = 5: 32 x 32, 512 threads of 2 rows (41..48);
 * 49..55 = depth 9..15 on 32 x 32 footprints of 1024 threads; and 56..63 =
 * depth 1..8 on 64 x 64 footprints of 1024 threads laid out 48 columns
 * apart, whose inputs the tensor memory accelerator copies into shared
 * memory while the CTA iterates on the previous footprint (one resident
 * CTA per SM walks the footprints; offered where the driver encodes the
 * level's tensor maps); and 64..71 = depth 1..8 on 64 x 48 footprints of
 * 768 threads of 4 rows.  On TGV handles the
 * candidates are 0 = a dual and a primal launch per iteration and 8 v + d =
 * temporal-blocking depth d on a 32 x 32 footprint of 256 (v = 0, choices
 * 1..8), 1024 (v = 1, 9..16) or 512 threads (v = 2, 17..24), or a 64 x 32
 * footprint of 512 (v = 3, 25..32) or 1024 threads (v = 4, 33..40).  Overwrites the levels' state; synchronises the
 * stream.  All candidates give identical results. */
fs_status fs_autotune(fs_handle* h, int iters, int* choice);

/* Set the per-level schedule directly, in fs_autotune's encoding (one entry
 * per level; -1 = the library default for that level), e.g. to reuse a
 * tuning measured earlier.  FS_EINVAL for a value out of range or a cluster
 * choice (0) on a level that does not fit one cluster. */
fs_status fs_set_schedule(fs_handle* h, const int* choice);

/* Guard-band debug mode, the out-of-bounds check in place of a memory
 * sanitizer.  A handle created while the environment variable
 * FS_GUARD_BANDS is a positive integer puts a band of 0xFF bytes before every
 * device plane of its state and after the last one.  A band is two rows of
 * the widest level-0 element (float2), rounded up to 256 bytes.  A stray
 * store into a band is detected; a stray load reads NaN (all-ones float, half
 * and bfloat16), or all mask bits, and shows in the results.  Every fs_solve
 * and fs_solve_continue then ends with this check, which synchronises the
 * handle's stream.  It returns FS_OK when every band is intact, FS_ECUDA
 * naming the plane after the first overwritten band, and FS_EINVAL for a
 * handle made without guard bands.  Results are the same bits as without
 * the bands; only the plane addresses move. */
fs_status fs_guard_check(fs_handle* h);

/* Testing aid for the check above: set byte `offset` of guard band `band`
 * (0 = the band before level 0's mask plane, bands in allocation order) to
 * 0, a store that fs_guard_check must then report; out = the number of
 * bands (may be NULL).  band = -1 only counts.  Writes inside the handle's
 * own allocation.  FS_EINVAL without guard bands or for an index out of
 * range. */
fs_status fs_guard_clobber(fs_handle* h, int band, size_t offset, int* out);

/* The persistent schedule (pd_schedule = FS_SCHED_PERSISTENT) and the
 * TMA-staged footprints (below): every wait of a work item on its
 * neighbours or on the coarser level, or of a CTA on its copies, gives up
 * after `seconds` of GPU global time.  In the persistent schedule the
 * launch then sets its status to FS_ETIMEOUT, every CTA of it returns at
 * its next claim or wait, and the solve returns FS_ETIMEOUT (the level
 * state is then unspecified; the next solve starts afresh); for the TMA
 * footprints see fs_check_waits.  Default 2 s; seconds must be in
 * (0, 3600].  A persistent batch uses the smallest limit among its
 * handles. */
fs_status fs_set_wait_limit(fs_handle* h, double seconds);

/* Testing aid for the bound above: stall = 1 makes the first work items of
 * the finest level of this handle's persistent solves wait for a counter
 * that nothing advances, so that wait runs out, and makes the first launch
 * of every level that runs the TMA-staged footprints (choices 56..63) wait
 * for 16 bytes that no copy delivers; stall = 0 restores the schedule.  A
 * batch stalls when any of its handles does.  Both this call and
 * fs_set_wait_limit drop the handle's captured graph (the bound and the
 * stall are launch arguments); a batch's graph keeps the values it was
 * captured with. */
fs_status fs_persist_stall(fs_handle* h, int stall);

/* The TMA-staged primal-dual footprints (fs_autotune choices 56..63): each
 * launch's CTAs wait on a shared-memory barrier for the copies of every
 * footprint, bounded like the persistent schedule (fs_set_wait_limit).  A
 * wait that runs out makes its CTA return and records FS_ETIMEOUT in the
 * handle.  fs_check_waits synchronises the handle's stream and returns
 * FS_ETIMEOUT (the state of the levels involved is then unspecified) when a
 * wait ran out since the last check, clearing the record, else FS_OK.
 * fs_solve_host checks by itself when the handle's schedule uses these
 * footprints; fs_solve, fs_solve_continue and fs_batch_solve enqueue work
 * and leave the check to the caller. */
fs_status fs_check_waits(fs_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* FS_STAGES_H */
