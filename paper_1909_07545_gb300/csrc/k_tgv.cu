// k_tgv.cu -- primal-dual iterations of the tensor-guided TGV-L1 energy
// (Sec. III-C, Eq. 10-11):
//
//   E(u, v) = lam |rho_bar(u)| + alpha1 |T^1/2 grad u - v| + alpha0 |grad v|
//
// with v a vector field and grad v its 2 x 2 Jacobian.  One iteration is two
// launches over the level, the dual ascent then the primal descent; every
// pixel reads its own and its right / lower (dual) or left / upper (primal)
// neighbours, so the two launches need no other synchronisation:
//
//   p    <- Pi_alpha1(p + sigma_p (T^1/2 grad ubar - vbar))
//   q    <- Pi_alpha0(q + sigma_q grad vbar)
//   u    <- shrink(u + tau_u div(T^1/2 p))                    (Eq. 13)
//   v    <- v + tau_v (p + div q)
//   ubar <- u' + theta (u' - u),   vbar <- v' + theta (v' - v)
//
// Pi_r projects a pixel's vector onto the ball of radius r (Euclidean for p,
// Frobenius for q): the consistent saddle point of Eq. 10 (Eq. 11 prints the
// weights inside unit-ball projections of the dual steps only).  Steps
// (Pock-Chambolle 2011 diagonal preconditioning on the entrywise bound of
// the block operator (T^1/2 grad u - v, grad v)): tau_u is the Huber-TV
// tau; sigma_p = 1 / (max row sum of |T^1/2| |grad| + 1), which is
// sigma / (1 + sigma) of the stored Huber-TV sigma; sigma_q = 1/2;
// tau_v = 1 / (1 + the active forward differences touching the pixel); all 0
// outside the FOV mask, where u, v, p and q stay put.  precond = 0 uses
// 1/sqrt(12) for all four.
#include "fs_kernels.h"

namespace fs {

namespace {

__device__ __forceinline__ float ball(float n2, float r) {
  // scale that projects a vector of squared norm n2 onto the ball of radius r
  return n2 > r * r ? r * rsqrtf(n2) : 1.f;
}

// T^1/2 p at pixel k with its mask bits (the masked products of px_dual).
__device__ __forceinline__ void t_half_p(const LevelView& L, size_t k, unsigned m, float& t1,
                                         float& t2) {
  const float sx = sld<ST_F32>(L.sx, k), sy = sld<ST_F32>(L.sy, k);
  const float p1 = sld<ST_F32>(L.p1, k), p2 = sld<ST_F32>(L.p2, k);
  const float dp = fmaf(sx, p1, __fmul_rn(sy, p2));
  t1 = (m & MASK_GX) ? fmaf(-sx, dp, p1) : 0.f;
  t2 = (m & MASK_GY) ? fmaf(-sy, dp, p2) : 0.f;
}

constexpr float kScalarStep = 0.28867513459481287f;   // 1 / sqrt(12)

}  // namespace

__global__ void k_tgv_dual(LevelView L, float alpha0, float alpha1, int precond) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  const unsigned m = L.mask[i];
  if (!(m & MASK_IN)) return;
  const bool gx = m & MASK_GX, gy = m & MASK_GY;
  const float sg = L.sig[i];
  const float sp = precond ? (sg > 0.f ? __fdiv_rn(sg, 1.f + sg) : 1.f) : kScalarStep;
  const float sq = precond ? 0.5f : kScalarStep;
  // p: T^1/2 grad ubar - vbar
  const float ub = L.ubar[i];
  const float g1 = gx ? __fsub_rn(L.ubar[i + 1], ub) : 0.f;
  const float g2 = gy ? __fsub_rn(L.ubar[i + L.P], ub) : 0.f;
  const float sx = sld<ST_F32>(L.sx, i), sy = sld<ST_F32>(L.sy, i);
  const float d = fmaf(sx, g1, __fmul_rn(sy, g2));
  const float vb1 = L.vb1[i], vb2 = L.vb2[i];
  float p1 = fmaf(sp, __fsub_rn(fmaf(-sx, d, g1), vb1), sld<ST_F32>(L.p1, i));
  float p2 = fmaf(sp, __fsub_rn(fmaf(-sy, d, g2), vb2), sld<ST_F32>(L.p2, i));
  const float sp_ = ball(fmaf(p1, p1, __fmul_rn(p2, p2)), alpha1);
  sst<ST_F32>(L.p1, i, __fmul_rn(p1, sp_));
  sst<ST_F32>(L.p2, i, __fmul_rn(p2, sp_));
  // q: grad vbar (Jacobian rows dv1, dv2)
  const float j11 = gx ? __fsub_rn(L.vb1[i + 1], vb1) : 0.f;
  const float j12 = gy ? __fsub_rn(L.vb1[i + L.P], vb1) : 0.f;
  const float j21 = gx ? __fsub_rn(L.vb2[i + 1], vb2) : 0.f;
  const float j22 = gy ? __fsub_rn(L.vb2[i + L.P], vb2) : 0.f;
  float q11 = fmaf(sq, j11, L.q11[i]), q12 = fmaf(sq, j12, L.q12[i]);
  float q21 = fmaf(sq, j21, L.q21[i]), q22 = fmaf(sq, j22, L.q22[i]);
  const float n2 = fmaf(q11, q11, fmaf(q12, q12, fmaf(q21, q21, __fmul_rn(q22, q22))));
  const float sc = alpha0 > 0.f ? ball(n2, alpha0) : 0.f;
  L.q11[i] = __fmul_rn(q11, sc);
  L.q12[i] = __fmul_rn(q12, sc);
  L.q21[i] = __fmul_rn(q21, sc);
  L.q22[i] = __fmul_rn(q22, sc);
}

__global__ void k_tgv_primal(LevelView L, float lam, float theta, int precond) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  const unsigned m = L.mask[i];
  if (!(m & MASK_IN)) return;
  const unsigned ml = x > 0 ? L.mask[i - 1] : 0u;
  const unsigned mu = y > 0 ? L.mask[i - L.P] : 0u;
  // u: div(T^1/2 p), then the L1 resolvent (Eq. 13) in its clamp form
  float t1, t2, tl1 = 0.f, tl2, tu1, tu2 = 0.f;
  t_half_p(L, i, m, t1, t2);
  if (x > 0) t_half_p(L, i - 1, ml, tl1, tl2);
  if (y > 0) t_half_p(L, i - L.P, mu, tu1, tu2);
  const float dv = __fadd_rn(__fsub_rn(t1, tl1), __fsub_rn(t2, tu2));
  const float u = L.u[i];
  const float tau = precond ? L.tau[i] : kScalarStep;
  const float uh = fmaf(tau, dv, u);
  const float Iu = sld<ST_F32>(L.Iu, i), rho0 = sld<ST_F32>(L.rho0, i);
  const float step = fabsf(__fmul_rn(__fmul_rn(tau, lam), Iu));
  const float c0 = Iu != 0.f ? __fsub_rn(L.uw[i], __fdiv_rn(rho0, Iu)) : 0.f;
  const float un = __fadd_rn(uh, fminf(fmaxf(__fsub_rn(c0, uh), -step), step));
  L.u[i] = un;
  L.ubar[i] = fmaf(theta, __fsub_rn(un, u), un);
  // v: p + div q
  const bool gx = m & MASK_GX, gy = m & MASK_GY;
  const bool glx = ml & MASK_GX, guy = mu & MASK_GY;
  const float d1 = __fadd_rn(__fsub_rn(gx ? L.q11[i] : 0.f, glx ? L.q11[i - 1] : 0.f),
                             __fsub_rn(gy ? L.q12[i] : 0.f, guy ? L.q12[i - L.P] : 0.f));
  const float d2 = __fadd_rn(__fsub_rn(gx ? L.q21[i] : 0.f, glx ? L.q21[i - 1] : 0.f),
                             __fsub_rn(gy ? L.q22[i] : 0.f, guy ? L.q22[i - L.P] : 0.f));
  const int cnt = (int)gx + (int)glx + (int)gy + (int)guy;
  const float tv = precond ? __fdiv_rn(1.f, (float)(1 + cnt)) : kScalarStep;
  const float v1 = L.v1[i], v2 = L.v2[i];
  const float v1n = fmaf(tv, __fadd_rn(sld<ST_F32>(L.p1, i), d1), v1);
  const float v2n = fmaf(tv, __fadd_rn(sld<ST_F32>(L.p2, i), d2), v2);
  L.v1[i] = v1n;
  L.v2[i] = v2n;
  L.vb1[i] = fmaf(theta, __fsub_rn(v1n, v1), v1n);
  L.vb2[i] = fmaf(theta, __fsub_rn(v2n, v2), v2n);
}

// v, vbar, q <- 0 on a new level (and before a warm start), like p.
__global__ void k_tgv_reset(LevelView L) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  L.v1[i] = L.v2[i] = L.vb1[i] = L.vb2[i] = 0.f;
  L.q11[i] = L.q12[i] = L.q21[i] = L.q22[i] = 0.f;
}

// vbar <- v at the start of a warp (as ubar <- u).
__global__ void k_tgv_warp_start(LevelView L) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  L.vb1[i] = L.v1[i];
  L.vb2[i] = L.v2[i];
}

namespace {
dim3 tgrid(int W, int H) { return dim3((W + 31) / 32, (H + 7) / 8); }
}  // namespace

cudaError_t launch_tgv_iterations(const LevelView& L, const PDParams& pp, float alpha0,
                                  float alpha1, int precond, int n, cudaStream_t st) {
  const dim3 g = tgrid(L.W, L.H), b(32, 8);
  for (int k = 0; k < n; ++k) {
    k_tgv_dual<<<g, b, 0, st>>>(L, alpha0, alpha1, precond);
    k_tgv_primal<<<g, b, 0, st>>>(L, pp.lam, pp.theta, precond);
  }
  return cudaGetLastError();
}

cudaError_t launch_tgv_reset(const LevelView& L, cudaStream_t st) {
  k_tgv_reset<<<tgrid(L.W, L.H), dim3(32, 8), 0, st>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_tgv_warp_start(const LevelView& L, cudaStream_t st) {
  k_tgv_warp_start<<<tgrid(L.W, L.H), dim3(32, 8), 0, st>>>(L);
  return cudaGetLastError();
}

}  // namespace fs
