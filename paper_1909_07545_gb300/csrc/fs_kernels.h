// fs_kernels.h -- kernel declarations shared by the library's translation units.
#pragma once

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
cudaError_t launch_warp(const LevelView& L, int central, cudaStream_t st);
// k_clip of one warp fused with k_warp of the next (same results).
cudaError_t launch_clip_warp(const LevelView& L, float du_max, int central, cudaStream_t st);
cudaError_t launch_tensor_abc(const LevelView& L, float* dst, cudaStream_t st);
cudaError_t launch_pack_s(const SPlane& src, int storage, float* dst, int W, int H, int P,
                          cudaStream_t st);
cudaError_t launch_unpack_s(const float* src, const SPlane& dst, int storage, int W, int H,
                            int P, cudaStream_t st);

// Primal-dual iterations: n <= B iterations with halo B, tile variant
// `variant`, state read from `in` and written to `out` (distinct buffers).
// chained = true when the launch directly follows another k_pd launch on
// the stream: it is then a programmatic dependent launch that loads its
// per-warp constants while the preceding launch drains, and waits for it
// before reading the state.
cudaError_t launch_pd(int variant, const LevelView& L, const PDState& in, const PDState& out,
                      const PDParams& pp, int B, int n, cudaStream_t st, bool chained = false);

// Whole-level primal-dual in one thread-block cluster: the tile variant for a
// W x H level (-1 if none), whether its cluster can be resident on this GPU,
// and the launch of n iterations in place.
int pd_cluster_variant(int W, int H);
bool pd_cluster_fits(int variant, int W, int H);
cudaError_t launch_pd_cluster(int variant, const LevelView& L, const PDParams& pp, int n,
                              cudaStream_t st);

}  // namespace fs
