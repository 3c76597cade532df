// pd_math.cuh -- per-pixel arithmetic of one primal-dual iteration (Eq. 11,
// 13), shared by every primal-dual kernel so that all schedules compute
// bit-identical results.
//
// K = T^1/2 grad with T^1/2 = I - s s^T (s = sqrt(1 - e) n, Eq. 12):
//   dual    p <- P((p + sigma K ubar) / (1 + sigma eps)),  P(q) = q / max(1, |q|)
//           t = masked T^1/2 p (what the divergence of the neighbours reads)
//   primal  uh = u + tau div(T^1/2 p)
//           rb = rho0 + I_u (uh - u_w)
//           u' = uh + tau lam I_u   if rb < -tau lam I_u^2
//                uh - tau lam I_u   if rb >  tau lam I_u^2
//                uh - rb / I_u      otherwise       (Eq. 13, resolvent of the L1 term)
//              = uh + clamp(-rb / I_u, -|tau lam I_u|, |tau lam I_u|)
//           (the three cases are the clamp of the unconstrained step; I_u = 0
//           gives uh).  tau = 0 outside the FOV mask, so u is held there.
#pragma once

#include "fs_device.cuh"

namespace fs {

// Per-pixel constants of one warp.
struct PxConst {
  float sx, sy;      // T^1/2 = I - s s^T
  float dinv, sd;    // 1 / (1 + sigma eps), sigma / (1 + sigma eps)
  float tau, step;   // tau, |tau lam I_u|
  float c0;          // u_w - rho0 / I_u (0 when I_u = 0)
};

// The per-pixel inputs of a warp as stored, fetched with no use in between
// so that a thread's loads for all its rows are in flight together.
struct PxRaw {
  float sx, sy, sig, tau, Iu, rho0, uw;
};

// Fetch from plane index i; v = false (a pixel outside the level) gives the
// inputs of a pixel that never moves (all 0).  i must be a valid index even
// when v is false (callers clamp it), so the loads need no branch.  CG: the
// planes may have been written earlier in the same launch (sld_m).
template <int S, bool CG = false>
__device__ __forceinline__ void px_fetch(const LevelView& L, size_t i, bool v, PxRaw& r) {
  r.sx = sld_m<S, CG>(L.sx, i);
  r.sy = sld_m<S, CG>(L.sy, i);
  r.sig = ldf<CG>(L.sig + i);
  r.tau = ldf<CG>(L.tau + i);
  r.Iu = sld_m<S, CG>(L.Iu, i);
  r.rho0 = sld_m<S, CG>(L.rho0, i);
  r.uw = ldf<CG>(L.uw + i);
  if (!v) r.sx = r.sy = r.sig = r.tau = r.Iu = r.rho0 = r.uw = 0.f;
}

// Per-pixel constants from the fetched inputs (all-zero inputs give the
// constants of px_zero).
__device__ __forceinline__ void px_make(const PxRaw& r, float lam, float eps, PxConst& c) {
  c.sx = r.sx;
  c.sy = r.sy;
  c.dinv = __fdiv_rn(1.f, fmaf(r.sig, eps, 1.f));
  c.sd = __fmul_rn(r.sig, c.dinv);
  c.tau = r.tau;
  c.step = fabsf(__fmul_rn(__fmul_rn(c.tau, lam), r.Iu));
  c.c0 = r.Iu != 0.f ? __fsub_rn(r.uw, __fdiv_rn(r.rho0, r.Iu)) : 0.f;
}

template <int S>
__device__ __forceinline__ void px_load(const LevelView& L, size_t i, float lam, float eps,
                                        PxConst& c) {
  PxRaw r;
  px_fetch<S>(L, i, true, r);
  px_make(r, lam, eps, c);
}

__device__ __forceinline__ void px_zero(PxConst& c) {
  c.sx = c.sy = 0.f;
  c.dinv = 1.f;
  c.sd = c.tau = c.step = c.c0 = 0.f;
}

// Dual ascent at one pixel: ub, right = ubar(x + e1), below = ubar(x + e2).
// Updates p1, p2 and returns the masked products t1, t2 of T^1/2 p.
// MASKED = false is for pixels whose mask bits are all set (in the FOV, both
// forward neighbours too): the masks then select every value as it is, so
// skipping them gives the same bits.
template <bool MASKED = true>
__device__ __forceinline__ void px_dual(unsigned m, float ub, float right, float below,
                                        const PxConst& c, float& p1, float& p2, float& t1,
                                        float& t2) {
  const float g1 = (!MASKED || (m & MASK_GX)) ? __fsub_rn(right, ub) : 0.f;
  const float g2 = (!MASKED || (m & MASK_GY)) ? __fsub_rn(below, ub) : 0.f;
  const float d = fmaf(c.sx, g1, __fmul_rn(c.sy, g2));
  const float k1 = fmaf(-c.sx, d, g1);
  const float k2 = fmaf(-c.sy, d, g2);
  float q1 = fmaf(c.sd, k1, __fmul_rn(p1, c.dinv));
  float q2 = fmaf(c.sd, k2, __fmul_rn(p2, c.dinv));
  // P(q) = q / max(1, |q|): scale by min(1, 1/|q|) (1 for |q| <= 1, also q = 0)
  const float s = fminf(1.f, rsqrtf(fmaf(q1, q1, __fmul_rn(q2, q2))));
  q1 = __fmul_rn(q1, s);
  q2 = __fmul_rn(q2, s);
  p1 = q1;
  p2 = q2;
  const float dp = fmaf(c.sx, q1, __fmul_rn(c.sy, q2));
  t1 = (!MASKED || (m & MASK_GX)) ? fmaf(-c.sx, dp, q1) : 0.f;
  t2 = (!MASKED || (m & MASK_GY)) ? fmaf(-c.sy, dp, q2) : 0.f;
}

// div(T^1/2 p) at a pixel from its own and its left / upper neighbours'
// masked products.
__device__ __forceinline__ float px_div(float t1, float t1_left, float t2, float t2_up) {
  return __fadd_rn(__fsub_rn(t1, t1_left), __fsub_rn(t2, t2_up));
}

// Over-relaxation ubar = u' + theta (u' - u).
__device__ __forceinline__ float px_relax(float un, float u, float theta) {
  return fmaf(theta, __fsub_rn(un, u), un);
}

// Primal descent + shrinkage at one pixel; dv = div(T^1/2 p) at the pixel.
// Returns the new u (unchanged where tau = 0, i.e. outside the mask).
__device__ __forceinline__ float px_primal(float u, float dv, const PxConst& c) {
  const float uh = fmaf(c.tau, dv, u);
  const float du = fminf(fmaxf(__fsub_rn(c.c0, uh), -c.step), c.step);
  return __fadd_rn(uh, du);
}

}  // namespace fs

// ------------------------------------------------------------ two pixels at once
// The same steps on two pixels held as the components of float2 values,
// with the packed FP32 operations of sm_100 and later (__ffma2_rn,
// __fadd2_rn, __fmul2_rn round each component exactly as __fmaf_rn,
// __fadd_rn, __fmul_rn do), so each component gets the bits of the scalar
// functions above; a - b is taken as fma(b, -1, a), the same rounded value.
// Minimum, maximum, the reciprocal square root and the mask selects stay
// per component.  The iteration loop issues about half the FP32
// instructions this way.
namespace fs {

struct PxConst2 {
  float2 sx, sy, dinv, sd, tau, step, c0;
};

__device__ __forceinline__ PxConst2 px_pair(const PxConst& a, const PxConst& b) {
  PxConst2 c;
  c.sx = make_float2(a.sx, b.sx);
  c.sy = make_float2(a.sy, b.sy);
  c.dinv = make_float2(a.dinv, b.dinv);
  c.sd = make_float2(a.sd, b.sd);
  c.tau = make_float2(a.tau, b.tau);
  c.step = make_float2(a.step, b.step);
  c.c0 = make_float2(a.c0, b.c0);
  return c;
}

// b - a, rounded once
__device__ __forceinline__ float2 f2_sub(float2 b, float2 a) {
  return __ffma2_rn(a, make_float2(-1.f, -1.f), b);
}

// px_dual on two pixels; m0, m1: their mask bits.
template <bool MASKED = true>
__device__ __forceinline__ void px_dual2(unsigned m0, unsigned m1, float2 ub, float2 right,
                                         float2 below, const PxConst2& c, float2& p1,
                                         float2& p2, float2& t1, float2& t2) {
  float2 g1 = f2_sub(right, ub);
  float2 g2 = f2_sub(below, ub);
  if constexpr (MASKED) {
    g1.x = (m0 & MASK_GX) ? g1.x : 0.f;
    g1.y = (m1 & MASK_GX) ? g1.y : 0.f;
    g2.x = (m0 & MASK_GY) ? g2.x : 0.f;
    g2.y = (m1 & MASK_GY) ? g2.y : 0.f;
  }
  const float2 d = __ffma2_rn(c.sx, g1, __fmul2_rn(c.sy, g2));
  const float2 nd = make_float2(-d.x, -d.y);
  const float2 k1 = __ffma2_rn(c.sx, nd, g1);
  const float2 k2 = __ffma2_rn(c.sy, nd, g2);
  float2 q1 = __ffma2_rn(c.sd, k1, __fmul2_rn(p1, c.dinv));
  float2 q2 = __ffma2_rn(c.sd, k2, __fmul2_rn(p2, c.dinv));
  const float2 n2 = __ffma2_rn(q1, q1, __fmul2_rn(q2, q2));
  const float2 s = make_float2(fminf(1.f, rsqrtf(n2.x)), fminf(1.f, rsqrtf(n2.y)));
  q1 = __fmul2_rn(q1, s);
  q2 = __fmul2_rn(q2, s);
  p1 = q1;
  p2 = q2;
  const float2 dp = __ffma2_rn(c.sx, q1, __fmul2_rn(c.sy, q2));
  const float2 ndp = make_float2(-dp.x, -dp.y);
  t1 = __ffma2_rn(c.sx, ndp, q1);
  t2 = __ffma2_rn(c.sy, ndp, q2);
  if constexpr (MASKED) {
    t1.x = (m0 & MASK_GX) ? t1.x : 0.f;
    t1.y = (m1 & MASK_GX) ? t1.y : 0.f;
    t2.x = (m0 & MASK_GY) ? t2.x : 0.f;
    t2.y = (m1 & MASK_GY) ? t2.y : 0.f;
  }
}

// px_div, px_primal and px_relax on two pixels.
__device__ __forceinline__ float2 px_div2(float2 t1, float2 t1_left, float2 t2, float2 t2_up) {
  return __fadd2_rn(f2_sub(t1, t1_left), f2_sub(t2, t2_up));
}

__device__ __forceinline__ float2 px_primal2(float2 u, float2 dv, const PxConst2& c) {
  const float2 uh = __ffma2_rn(c.tau, dv, u);
  const float2 r = f2_sub(c.c0, uh);
  const float2 du = make_float2(fminf(fmaxf(r.x, -c.step.x), c.step.x),
                                fminf(fmaxf(r.y, -c.step.y), c.step.y));
  return __fadd2_rn(uh, du);
}

__device__ __forceinline__ float2 px_relax2(float2 un, float2 u, float2 theta) {
  return __ffma2_rn(theta, f2_sub(un, u), un);
}

}  // namespace fs
