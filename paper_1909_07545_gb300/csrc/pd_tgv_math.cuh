// pd_tgv_math.cuh -- per-pixel arithmetic of one TGV-L1 primal-dual
// iteration (Sec. III-C, Eq. 10-11), shared by the launch-per-step kernels
// and the temporally blocked kernel so that both give bit-identical results.
//
//   dual:   p <- Pi_alpha1(p + sigma_p (T^1/2 grad ubar - vbar))
//           q <- Pi_alpha0(q + sigma_q grad vbar)
//   primal: u <- shrink(u + tau_u div(T^1/2 p))            (Eq. 13, clamp form)
//           v <- v + tau_v (p + div q)
//           ubar, vbar <- over-relaxation
//
// The dual also returns what the neighbours' primal steps read: the masked
// products t = T^1/2 p (t1 zero where the x-difference leaves the mask, t2
// where the y-difference does) and q with the same masks (qx = (q11, q21) for
// the x-differences, qy = (q12, q22) for the y-differences).
#pragma once

#include "fs_device.cuh"

namespace fs {

struct TgvParams {
  float lam, theta, alpha0, alpha1;
  int precond;
};

// Per-pixel constants of one warp (all 0 off the FOV mask: nothing moves).
struct TgvConst {
  float sx, sy;        // T^1/2 = I - s s^T
  float sp, sq;        // sigma_p, sigma_q
  float tau, step, c0; // tau_u, |tau_u lam I_u|, u_w - rho0 / I_u
  float tv;            // tau_v
};

constexpr float kTgvScalarStep = 0.28867513459481287f;   // 1 / sqrt(12)

// m: own mask bits; ml, mu: the left and upper neighbours' bits (0 off the
// level); sig, tau: the stored Huber-TV steps; I_u, rho0, u_w: linearisation.
__device__ __forceinline__ void tgv_const(unsigned m, unsigned ml, unsigned mu, float sx,
                                          float sy, float sig, float tau, float Iu, float rho0,
                                          float uw, const TgvParams& tp, TgvConst& c) {
  if (!(m & MASK_IN)) {
    c.sx = c.sy = c.sp = c.sq = c.tau = c.step = c.c0 = c.tv = 0.f;
    return;
  }
  c.sx = sx;
  c.sy = sy;
  if (tp.precond) {
    c.sp = sig > 0.f ? __fdiv_rn(sig, 1.f + sig) : 1.f;   // 1 / (max row sum + 1)
    c.sq = 0.5f;
    c.tau = tau;
    const int cnt = (int)((m & MASK_GX) != 0) + (int)((ml & MASK_GX) != 0) +
                    (int)((m & MASK_GY) != 0) + (int)((mu & MASK_GY) != 0);
    c.tv = __fdiv_rn(1.f, (float)(1 + cnt));
  } else {
    c.sp = c.sq = c.tau = c.tv = kTgvScalarStep;
  }
  c.step = fabsf(__fmul_rn(__fmul_rn(c.tau, tp.lam), Iu));
  c.c0 = Iu != 0.f ? __fsub_rn(uw, __fdiv_rn(rho0, Iu)) : 0.f;
}

__device__ __forceinline__ float tgv_ball(float n2, float r) {
  return n2 > r * r ? r * rsqrtf(n2) : 1.f;
}

// Dual ascent at one pixel from its own and its right (r) / lower (b)
// neighbours' ubar, vbar.  Updates p, q; returns t and the masked q.
__device__ __forceinline__ void tgv_px_dual(unsigned m, float ub, float ub_r, float ub_b,
                                            float vb1, float vb1_r, float vb1_b, float vb2,
                                            float vb2_r, float vb2_b, const TgvConst& c,
                                            const TgvParams& tp, float& p1, float& p2,
                                            float& q11, float& q12, float& q21, float& q22,
                                            float& t1, float& t2, float& qx1, float& qx2,
                                            float& qy1, float& qy2) {
  const bool gx = m & MASK_GX, gy = m & MASK_GY;
  const float g1 = gx ? __fsub_rn(ub_r, ub) : 0.f;
  const float g2 = gy ? __fsub_rn(ub_b, ub) : 0.f;
  const float d = fmaf(c.sx, g1, __fmul_rn(c.sy, g2));
  float a1 = fmaf(c.sp, __fsub_rn(fmaf(-c.sx, d, g1), vb1), p1);
  float a2 = fmaf(c.sp, __fsub_rn(fmaf(-c.sy, d, g2), vb2), p2);
  const float s = tgv_ball(fmaf(a1, a1, __fmul_rn(a2, a2)), tp.alpha1);
  p1 = __fmul_rn(a1, s);
  p2 = __fmul_rn(a2, s);
  const float j11 = gx ? __fsub_rn(vb1_r, vb1) : 0.f;
  const float j12 = gy ? __fsub_rn(vb1_b, vb1) : 0.f;
  const float j21 = gx ? __fsub_rn(vb2_r, vb2) : 0.f;
  const float j22 = gy ? __fsub_rn(vb2_b, vb2) : 0.f;
  const float b11 = fmaf(c.sq, j11, q11), b12 = fmaf(c.sq, j12, q12);
  const float b21 = fmaf(c.sq, j21, q21), b22 = fmaf(c.sq, j22, q22);
  const float n2 = fmaf(b11, b11, fmaf(b12, b12, fmaf(b21, b21, __fmul_rn(b22, b22))));
  const float sc = tp.alpha0 > 0.f ? tgv_ball(n2, tp.alpha0) : 0.f;
  q11 = __fmul_rn(b11, sc);
  q12 = __fmul_rn(b12, sc);
  q21 = __fmul_rn(b21, sc);
  q22 = __fmul_rn(b22, sc);
  const float dp = fmaf(c.sx, p1, __fmul_rn(c.sy, p2));
  t1 = gx ? fmaf(-c.sx, dp, p1) : 0.f;
  t2 = gy ? fmaf(-c.sy, dp, p2) : 0.f;
  qx1 = gx ? q11 : 0.f;
  qx2 = gx ? q21 : 0.f;
  qy1 = gy ? q12 : 0.f;
  qy2 = gy ? q22 : 0.f;
}

// Primal descent at one pixel from its own and its left (l) / upper (u)
// neighbours' masked products.  Updates u, ubar, v, vbar.
__device__ __forceinline__ void tgv_px_primal(float t1, float t1_l, float t2, float t2_u,
                                              float qx1, float qx1_l, float qy1, float qy1_u,
                                              float qx2, float qx2_l, float qy2, float qy2_u,
                                              float p1, float p2, const TgvConst& c,
                                              float theta, float& u, float& ub, float& v1,
                                              float& v2, float& vb1, float& vb2) {
  const float dv = __fadd_rn(__fsub_rn(t1, t1_l), __fsub_rn(t2, t2_u));
  const float uh = fmaf(c.tau, dv, u);
  const float un = __fadd_rn(uh, fminf(fmaxf(__fsub_rn(c.c0, uh), -c.step), c.step));
  ub = fmaf(theta, __fsub_rn(un, u), un);
  u = un;
  const float d1 = __fadd_rn(__fsub_rn(qx1, qx1_l), __fsub_rn(qy1, qy1_u));
  const float d2 = __fadd_rn(__fsub_rn(qx2, qx2_l), __fsub_rn(qy2, qy2_u));
  const float v1n = fmaf(c.tv, __fadd_rn(p1, d1), v1);
  const float v2n = fmaf(c.tv, __fadd_rn(p2, d2), v2);
  vb1 = fmaf(theta, __fsub_rn(v1n, v1), v1n);
  vb2 = fmaf(theta, __fsub_rn(v2n, v2), v2n);
  v1 = v1n;
  v2 = v2n;
}

}  // namespace fs

// ------------------------------------------------------------ two pixels at once
// tgv_px_dual and tgv_px_primal on two pixels held as float2 components,
// with the packed FP32 operations (each component rounded as the scalar
// __fmaf_rn, __fadd_rn, __fmul_rn; a - b as fma(b, -1, a)): the same bits.
// The projections and the mask selects stay per component.
namespace fs {

struct TgvConst2 {
  float2 sx, sy, sp, sq, tau, step, c0, tv;
};

__device__ __forceinline__ TgvConst2 tgv_pair(const TgvConst& a, const TgvConst& b) {
  TgvConst2 c;
  c.sx = make_float2(a.sx, b.sx);
  c.sy = make_float2(a.sy, b.sy);
  c.sp = make_float2(a.sp, b.sp);
  c.sq = make_float2(a.sq, b.sq);
  c.tau = make_float2(a.tau, b.tau);
  c.step = make_float2(a.step, b.step);
  c.c0 = make_float2(a.c0, b.c0);
  c.tv = make_float2(a.tv, b.tv);
  return c;
}

// b - a, rounded once
__device__ __forceinline__ float2 tgv_sub2(float2 b, float2 a) {
  return __ffma2_rn(a, make_float2(-1.f, -1.f), b);
}

__device__ __forceinline__ float2 tgv_sel2(bool kx, bool ky, float2 v) {
  return make_float2(kx ? v.x : 0.f, ky ? v.y : 0.f);
}

// m0, m1: the two pixels' mask bits.
__device__ __forceinline__ void tgv_px_dual2(
    unsigned m0, unsigned m1, float2 ub, float2 ub_r, float2 ub_b, float2 vb1, float2 vb1_r,
    float2 vb1_b, float2 vb2, float2 vb2_r, float2 vb2_b, const TgvConst2& c,
    const TgvParams& tp, float2& p1, float2& p2, float2& q11, float2& q12, float2& q21,
    float2& q22, float2& t1, float2& t2, float2& qx1, float2& qx2, float2& qy1, float2& qy2) {
  const bool gx0 = m0 & MASK_GX, gx1 = m1 & MASK_GX, gy0 = m0 & MASK_GY, gy1 = m1 & MASK_GY;
  const float2 g1 = tgv_sel2(gx0, gx1, tgv_sub2(ub_r, ub));
  const float2 g2 = tgv_sel2(gy0, gy1, tgv_sub2(ub_b, ub));
  const float2 d = __ffma2_rn(c.sx, g1, __fmul2_rn(c.sy, g2));
  const float2 nd = make_float2(-d.x, -d.y);
  const float2 a1 = __ffma2_rn(c.sp, tgv_sub2(__ffma2_rn(c.sx, nd, g1), vb1), p1);
  const float2 a2 = __ffma2_rn(c.sp, tgv_sub2(__ffma2_rn(c.sy, nd, g2), vb2), p2);
  const float2 na = __ffma2_rn(a1, a1, __fmul2_rn(a2, a2));
  const float2 s = make_float2(tgv_ball(na.x, tp.alpha1), tgv_ball(na.y, tp.alpha1));
  p1 = __fmul2_rn(a1, s);
  p2 = __fmul2_rn(a2, s);
  const float2 j11 = tgv_sel2(gx0, gx1, tgv_sub2(vb1_r, vb1));
  const float2 j12 = tgv_sel2(gy0, gy1, tgv_sub2(vb1_b, vb1));
  const float2 j21 = tgv_sel2(gx0, gx1, tgv_sub2(vb2_r, vb2));
  const float2 j22 = tgv_sel2(gy0, gy1, tgv_sub2(vb2_b, vb2));
  const float2 b11 = __ffma2_rn(c.sq, j11, q11), b12 = __ffma2_rn(c.sq, j12, q12);
  const float2 b21 = __ffma2_rn(c.sq, j21, q21), b22 = __ffma2_rn(c.sq, j22, q22);
  const float2 nb = __ffma2_rn(b11, b11, __ffma2_rn(b12, b12, __ffma2_rn(b21, b21,
                                                                          __fmul2_rn(b22, b22))));
  const float2 sc = tp.alpha0 > 0.f
                        ? make_float2(tgv_ball(nb.x, tp.alpha0), tgv_ball(nb.y, tp.alpha0))
                        : make_float2(0.f, 0.f);
  q11 = __fmul2_rn(b11, sc);
  q12 = __fmul2_rn(b12, sc);
  q21 = __fmul2_rn(b21, sc);
  q22 = __fmul2_rn(b22, sc);
  const float2 dp = __ffma2_rn(c.sx, p1, __fmul2_rn(c.sy, p2));
  const float2 ndp = make_float2(-dp.x, -dp.y);
  t1 = tgv_sel2(gx0, gx1, __ffma2_rn(c.sx, ndp, p1));
  t2 = tgv_sel2(gy0, gy1, __ffma2_rn(c.sy, ndp, p2));
  qx1 = tgv_sel2(gx0, gx1, q11);
  qx2 = tgv_sel2(gx0, gx1, q21);
  qy1 = tgv_sel2(gy0, gy1, q12);
  qy2 = tgv_sel2(gy0, gy1, q22);
}

__device__ __forceinline__ void tgv_px_primal2(
    float2 t1, float2 t1_l, float2 t2, float2 t2_u, float2 qx1, float2 qx1_l, float2 qy1,
    float2 qy1_u, float2 qx2, float2 qx2_l, float2 qy2, float2 qy2_u, float2 p1, float2 p2,
    const TgvConst2& c, float2 theta, float2& u, float2& ub, float2& v1, float2& v2,
    float2& vb1, float2& vb2) {
  const float2 dv = __fadd2_rn(tgv_sub2(t1, t1_l), tgv_sub2(t2, t2_u));
  const float2 uh = __ffma2_rn(c.tau, dv, u);
  const float2 r = tgv_sub2(c.c0, uh);
  const float2 un = __fadd2_rn(uh, make_float2(fminf(fmaxf(r.x, -c.step.x), c.step.x),
                                               fminf(fmaxf(r.y, -c.step.y), c.step.y)));
  ub = __ffma2_rn(theta, tgv_sub2(un, u), un);
  u = un;
  const float2 d1 = __fadd2_rn(tgv_sub2(qx1, qx1_l), tgv_sub2(qy1, qy1_u));
  const float2 d2 = __fadd2_rn(tgv_sub2(qx2, qx2_l), tgv_sub2(qy2, qy2_u));
  const float2 v1n = __ffma2_rn(c.tv, __fadd2_rn(p1, d1), v1);
  const float2 v2n = __ffma2_rn(c.tv, __fadd2_rn(p2, d2), v2);
  vb1 = __ffma2_rn(theta, tgv_sub2(v1n, v1), v1n);
  vb2 = __ffma2_rn(theta, tgv_sub2(v2n, v2), v2n);
  v1 = v1n;
  v2 = v2n;
}

}  // namespace fs
