// fs_kernels.h -- kernel declarations shared by the library's translation units.
#pragma once

#include "fs_device.cuh"

namespace fs {

enum PDVariant { PD_TILE_64 = 0, PD_TILE_32 = 1 };
enum PDClusterVariant { PD_CLUSTER_16 = 0, PD_CLUSTER_32 = 1 };

__global__ void k_trajectory(DevCam cam, float tx, float ty, float tz, LevelView L);
__global__ void k_prerotate(const float* __restrict__ I1, const float2* __restrict__ field,
                            SPlane out, int st, int W, int H, int P);
__global__ void k_copy_in_s(const float* __restrict__ src, SPlane dst, int st, int W, int H,
                            int P);
__global__ void k_pack_s(SPlane src, int st, float* __restrict__ dst, int W, int H, int P);
__global__ void k_unpack_s(const float* __restrict__ src, SPlane dst, int st, int W, int H,
                           int P);
__global__ void k_copy_in(const float* __restrict__ src, float* __restrict__ dst, int W, int H,
                          int P);
__global__ void k_downsample(LevelView F, LevelView C);
__global__ void k_upsample(LevelView C, LevelView F);
__global__ void k_zero_state(LevelView L);
__global__ void k_warm_start(LevelView L, float du_max);
__global__ void k_tensor(LevelView L, float beta, float eta, int precond);
__global__ void k_warp(LevelView L);
__global__ void k_clip(LevelView L, float du_max);
__global__ void k_depth(LevelView L, DevCam cam, float Cx, float Cy, float Cz,
                        float* __restrict__ disp, float* __restrict__ depth);
__global__ void k_pack(const float* __restrict__ src, int stride, float* __restrict__ dst, int W,
                       int H, int P);
__global__ void k_unpack(const float* __restrict__ src, float* __restrict__ dst, int stride,
                         int W, int H, int P);
__global__ void k_mask_to_float(const uint8_t* __restrict__ m, float* __restrict__ dst, int W,
                                int H, int P);
__global__ void k_tensor_abc(LevelView L, float* __restrict__ dst);

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
