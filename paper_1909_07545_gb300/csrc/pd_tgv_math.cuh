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
