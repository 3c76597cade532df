// k_energy.cu -- the linearised energy of one warp at a level, reduced on
// the GPU: warp shuffles sum the per-pixel terms, one double-precision atomic
// per warp accumulates them (Eq. 10 and the linearised data term of Eq. 3, 5):
//
//   data         lam sum_{x in M} |rho0 + I_u (u - u_w)|
//   regulariser  Huber-TV: sum_x h_eps(T^1/2 grad u)
//                TGV-L1:   alpha1 sum_{x in M} |T^1/2 grad u - v| + alpha0 sum_x |grad v|
//
// grad: the masked forward differences of the primal-dual steps.  The per-
// pixel terms are FP32; the sums are FP64 from the warp level up.
#include "fs_kernels.h"

namespace fs {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

template <int S>
__global__ void k_energy(LevelView L, float lam, float eps, int tgv, float alpha0,
                         float alpha1, double* __restrict__ acc) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  float data = 0.f, reg = 0.f, resid = 0.f;
  if (x < L.W && y < L.H) {            // no early return: every lane joins the shuffles
    const size_t i = (size_t)y * L.P + x;
    const unsigned m = L.mask[i];
    const float u = L.u[i];
    const float g1 = (m & MASK_GX) ? L.u[i + 1] - u : 0.f;
    const float g2 = (m & MASK_GY) ? L.u[i + L.P] - u : 0.f;
    const float sx = sld<S>(L.sx, i), sy = sld<S>(L.sy, i);
    const float d = sx * g1 + sy * g2;
    const float k1 = g1 - sx * d, k2 = g2 - sy * d;
    if (m & MASK_IN) {
      resid = fabsf(sld<S>(L.rho0, i) + sld<S>(L.Iu, i) * (u - L.uw[i]));
      data = lam * resid;
    }
    if (!tgv) {
      const float n = sqrtf(k1 * k1 + k2 * k2);
      reg = n <= eps ? (eps > 0.f ? n * n / (2.f * eps) : 0.f) : n - 0.5f * eps;
    } else {
      if (m & MASK_IN) reg = alpha1 * sqrtf((k1 - L.v1[i]) * (k1 - L.v1[i]) +
                                            (k2 - L.v2[i]) * (k2 - L.v2[i]));
      const float j11 = (m & MASK_GX) ? L.v1[i + 1] - L.v1[i] : 0.f;
      const float j12 = (m & MASK_GY) ? L.v1[i + L.P] - L.v1[i] : 0.f;
      const float j21 = (m & MASK_GX) ? L.v2[i + 1] - L.v2[i] : 0.f;
      const float j22 = (m & MASK_GY) ? L.v2[i + L.P] - L.v2[i] : 0.f;
      reg += alpha0 * sqrtf(j11 * j11 + j12 * j12 + j21 * j21 + j22 * j22);
    }
  }
  data = warp_sum(data);
  reg = warp_sum(reg);
  resid = warp_sum(resid);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], (double)data);
    atomicAdd(&acc[1], (double)reg);
    atomicAdd(&acc[2], (double)resid);
  }
}

cudaError_t launch_energy(const LevelView& L, float lam, float eps, int tgv, float alpha0,
                          float alpha1, double* acc, cudaStream_t st) {
  const dim3 g((L.W + 31) / 32, (L.H + 7) / 8), b(32, 8);
  switch (L.st) {
    case ST_F16: k_energy<ST_F16><<<g, b, 0, st>>>(L, lam, eps, tgv, alpha0, alpha1, acc); break;
    case ST_BF16: k_energy<ST_BF16><<<g, b, 0, st>>>(L, lam, eps, tgv, alpha0, alpha1, acc); break;
    default: k_energy<ST_F32><<<g, b, 0, st>>>(L, lam, eps, tgv, alpha0, alpha1, acc); break;
  }
  return cudaGetLastError();
}

}  // namespace fs
