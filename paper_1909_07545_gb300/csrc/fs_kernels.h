// fs_kernels.h -- kernel declarations shared by the library's translation units.
#pragma once

#include <cuda.h>

#include "cam_df.cuh"
#include "fs_device.cuh"

namespace fs {

// k_pd footprints: 64 x 64 (512 threads), 32 x 32 and 64 x 32 (256 threads)
enum PDVariant {
  PD_TILE_64 = 0,         // 64 x 64 footprint, 64 x 8 threads of 8 rows
  PD_TILE_32 = 1,         // 32 x 32, 32 x 8 threads of 4 rows
  PD_TILE_64x32 = 2,      // 64 x 32, 64 x 4 threads of 8 rows
  PD_TILE_64_T1024 = 3,   // 64 x 64, 64 x 16 threads of 4 rows
  PD_TILE_32_T1024 = 4,   // 32 x 32, 32 x 32 threads of 1 row
  PD_TILE_32_T512 = 5,    // 32 x 32, 32 x 16 threads of 2 rows
  PD_TILE_COUNT = 6
};
// The TMA-staged footprints of k_pd_tma.cu (64 x 64, 1024 threads of 4 rows,
// 48 interior columns, depth <= 8): not a PDVariant of launch_pd.
constexpr int PD_TILE_64_TMA = PD_TILE_COUNT;
// 64 x 48, 64 x 12 threads of 4 rows (768 threads, up to 80 registers):
// a launch_pd variant numbered after the TMA footprints.  A 512 x 512 level
// at depth 6 has 150 of them, one per SM, where 64 x 64 footprints leave
// 31 SMs idle.
constexpr int PD_TILE_64x48_T768 = PD_TILE_COUNT + 1;
enum PDClusterVariant { PD_CLUSTER_16 = 0, PD_CLUSTER_32 = 1 };

__global__ void k_trajectory(DevCamDF cam, df tx, df ty, df tz, LevelView L);
__global__ void k_calib_field(DevCamDF c0, DevCamDF c1, RotDF R, const uint8_t* __restrict__ mask,
                              float4* __restrict__ field, int W, int H, int P);
__global__ void k_copy_in(const float* __restrict__ src, float* __restrict__ dst, int W, int H,
                          int P);
__global__ void k_clip(LevelView L, float du_max);
__global__ void k_depth(LevelView L, DevCam cam, float Cx, float Cy, float Cz,
                        float* __restrict__ disp, float* __restrict__ depth);
__global__ void k_pack(const float* __restrict__ src, int stride, float* __restrict__ dst, int W,
                       int H, int P);
__global__ void k_unpack(const float* __restrict__ src, float* __restrict__ dst, int stride,
                         int W, int H, int P);
__global__ void k_mask_to_float(const uint8_t* __restrict__ m, float* __restrict__ dst, int W,
                                int H, int P);

// Storage-typed kernels, launched through these (the level's storage picks
// the instantiation).
cudaError_t launch_prerotate(const float* I1, const float4* field, const LevelView& L0,
                             cudaStream_t st);
// A dense FP32 image into level L's I0 (which = 0) or I1 (1), with the low
// part of its rounding to the level's storage (the pyramid's carry).
cudaError_t launch_copy_in_image(const float* src, const LevelView& L, int which,
                                 cudaStream_t st);
cudaError_t launch_downsample(const LevelView& F, const LevelView& C, cudaStream_t st);
cudaError_t launch_upsample(const LevelView& C, const LevelView& F, cudaStream_t st);
cudaError_t launch_zero_state(const LevelView& L, cudaStream_t st);
cudaError_t launch_warm_start(const LevelView& L, float du_max, cudaStream_t st);
cudaError_t launch_continue(const LevelView& L, cudaStream_t st);

// TGV-L1 (k_tgv.cu): n iterations, with B = 0 as a dual and a primal launch
// each, else temporally blocked with at most B (1..8) per launch on 32 x 32
// footprints of 256 (variant 0), 1024 (1) or 512 (2) threads, or 64 x 32
// footprints of 512 (3) or 1024 (4) threads (identical results); v, vbar,
// q <- 0; vbar <- v at a warp's start.
constexpr int kTgvVariants = 5;
struct TgvParams;
cudaError_t launch_tgv_iterations(const LevelView& L, const TgvParams& tp, int B, int variant,
                                  int n, cudaStream_t st);
cudaError_t launch_tgv_reset(const LevelView& L, cudaStream_t st);
// Energy terms of a level summed into acc[0..2] (data, regulariser, L1
// residual); acc must be zeroed first (k_energy.cu).
cudaError_t launch_energy(const LevelView& L, float lam, float eps, int tgv, float alpha0,
                          float alpha1, double* acc, cudaStream_t st);
cudaError_t launch_tgv_warp_start(const LevelView& L, cudaStream_t st);
cudaError_t launch_tensor(const LevelView& L, float beta, float eta, int precond,
                          cudaStream_t st);
// consts = 1: also the per-warp constants of the primal-dual iterations
// (the values launch_pd_consts computes), from the I_u, rho0 and u_w the
// kernel writes.
cudaError_t launch_warp(const LevelView& L, int central, float lam, float eps, int consts,
                        cudaStream_t st);
// k_clip of one warp fused with k_warp of the next (same results).
cudaError_t launch_clip_warp(const LevelView& L, float du_max, int central, float lam, float eps,
                             int consts, cudaStream_t st);
cudaError_t launch_tensor_abc(const LevelView& L, float* dst, cudaStream_t st);
cudaError_t launch_pack_s(const SPlane& src, int storage, float* dst, int W, int H, int P,
                          cudaStream_t st);
cudaError_t launch_unpack_s(const float* src, const SPlane& dst, int storage, int W, int H,
                            int P, cudaStream_t st);

// The per-warp constants of the primal-dual iterations (L.dinv, L.sd,
// L.step, L.c0) from the level's sigma, tau, I_u, rho0 and u_w; launch_pd
// and launch_pd_tma read them.  The kernels that start a warp (launch_warp,
// launch_clip_warp) write the same values; this one is for state that
// reached the planes another way (buffer writes, the stage interface).
cudaError_t launch_pd_consts(const LevelView& L, float lam, float eps, cudaStream_t st);

// Primal-dual iterations: n <= B iterations with halo B, tile variant
// `variant`, state read from `in` and written to `out` (distinct buffers).
// chained = true when the launch directly follows another k_pd launch on
// the stream: it is then a programmatic dependent launch that loads its
// per-warp constants while the preceding launch drains, and waits for it
// before reading the state.
cudaError_t launch_pd(int variant, const LevelView& L, const PDState& in, const PDState& out,
                      const PDParams& pp, int B, int n, cudaStream_t st, bool chained = false);

// The tensor maps k_pd_tma copies a footprint through: T^1/2, tau, the
// per-warp constants (launch_pd_consts) and the mask of a level, and the
// state planes of the buffer set the launch reads (each a 2-D tensor of the
// level's W x H pixels, pitch P; boxes of 64 x 64 elements, the mask's
// 80 x 64).
struct PdTmaMaps {
  CUtensorMap sx, sy, tau, dinv, sd, step, c0, mask;
  CUtensorMap u, ubar, p1, p2;
};

// n (<= B <= 8) primal-dual iterations on the TMA-staged footprints (one
// resident CTA per SM walking the footprints), the state read through
// `maps` and written to `out`; chained as in launch_pd.  A copy wait that
// runs out after wait_ns of global time sets *status to FS_ETIMEOUT;
// stall = 1 makes the first wait run out (testing aid).  Same results as
// launch_pd.
cudaError_t launch_pd_tma(const LevelView& L, const PDState& out, const PDParams& pp, int B,
                          int n, bool chained, const PdTmaMaps& maps, int* status,
                          unsigned long long wait_ns, int stall, cudaStream_t st);
// Dynamic shared memory of one k_pd_tma CTA for a storage type.
size_t pd_tma_smem_bytes(int storage);

// Whole-level primal-dual in one thread-block cluster: the tile variant for a
// W x H level (-1 if none), whether its cluster can be resident on this GPU,
// and the launch of n iterations in place.
int pd_cluster_variant(int W, int H);
bool pd_cluster_fits(int variant, int W, int H);
cudaError_t launch_pd_cluster(int variant, const LevelView& L, const PDParams& pp, int n,
                              cudaStream_t st);

// ---------------------------------------------------------------- persistent schedule
// A whole solve (or a batch of them) as one launch over a work list
// (k_persist.cu).  A job is one pyramid level of one pair; its interior tiles
// are the units of work.  Every tile of a job runs the same chain of items:
//   PRE            tensor and step sizes, zero state (coarsest level) or
//                  upsampling from the coarser level, warp + linearisation
//   PD(w, k)       primal-dual block k of warp w (pd_tile, halo B)
//   CLIP(w)        clip + update, and the next warp's linearisation
// Item s of a tile's chain starts once every tile its footprint reaches --
// the tile and its neighbours within `radius` tiles (the eight around it
// when the halo B is at most the interior width) -- has finished item s - 1
// (their counters in `done`), and a PRE once the coarser level of the same
// pair has finished (its counter in level_done).
// Items are claimed in an order in which every item's dependencies come
// earlier, so a claimed item only ever waits on items that running CTAs
// hold.
enum PersistKind { PERSIST_PRE = 0, PERSIST_PD = 1, PERSIST_CLIP = 2 };

struct PersistJob {
  LevelView L;               // the level
  LevelView C;               // the coarser level (upsampling source); unused at the top
  PDParams pp;
  int top;                   // the pair's coarsest level: zero state instead of upsampling
  int variant;               // PD_TILE_64_T1024 or PD_TILE_32_T1024
  int B;                     // halo depth of the primal-dual blocks
  int IW, IH;                // interior tile size
  int radius;                // tiles a footprint reaches on each side: ceil(B / IW), 1 or 2
  int tiles_x, tiles_y;
  int done_base;             // this job's first counter in `done`
  int level_slot;            // this job's counter in level_done
  int coarse_slot;           // the coarser level's counter (-1 at the top)
  int coarse_tiles;          // tiles of the coarser level (its finished count)
  float beta, eta, du_max;
  int precond, central;
  int stall;                 // testing aid: the PRE items wait on a counter nothing sets
};

struct PersistPhase {        // one item kind for every tile of one job
  int first;                 // index of its first item
  int job;
  int kind;                  // PersistKind
  int seq;                   // position in the tile chain (0 = PRE)
  int block;                 // PD: block index within the warp (ping-pong parity)
  int n_iter;                // PD: iterations of the block
  int next_warp;             // CLIP: 1 if another warp follows (fused linearisation)
  int last;                  // CLIP of the last warp: the level is done after it
};

// Device control block of one launch: the claim counter, the abort flag and
// the status (0, or FS_ETIMEOUT when a wait gave up).
struct PersistCtrl {
  unsigned next;
  unsigned abort;
  int status;
  unsigned pad;
};

// The persistent launch: `grid` CTAs of 1024 threads over n_items items.
// wait_ns bounds every wait (global-timer nanoseconds).
cudaError_t launch_persist(int storage, const PersistJob* jobs, const PersistPhase* phases,
                           const int* item_phase, int n_items, PersistCtrl* ctrl, unsigned* done,
                           unsigned* level_done, unsigned long long wait_ns, int grid,
                           cudaStream_t st);
// CTAs of the persistent kernel that fit on the device at once.
int persist_max_ctas(int storage);

}  // namespace fs
