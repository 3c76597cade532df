// level_px.cuh -- the per-pixel work of the level stages other than the
// primal-dual iteration: zero state, upsampling, tensor and step sizes,
// warp + linearisation, clip + update.  The launch-per-stage kernels
// (k_level.cu) and the persistent schedule (k_persist.cu) call the same
// functions, so both compute the same bits.  Template parameter CG: the
// planes read may have been written by another CTA of the same launch
// (loads through L2 only, fs_device.cuh).
#pragma once

#include "fs_device.cuh"

namespace fs {

// ------------------------------------------------------------ zero state
// Algorithm 1's start at the coarsest level: u = ubar = u_w = 0, p = 0, w = 0.
template <int S>
__device__ __forceinline__ void zero_px(const LevelView& L, size_t o) {
  L.u[o] = 0.f; L.ubar[o] = 0.f; L.uw[o] = 0.f;
  sst<S>(L.p1, o, 0.f); sst<S>(L.p2, o, 0.f);
  L.w[o] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------ upsampling
// u, w of level C (coarse) -> pixel (x, y) of level F (fine): bilinear over
// the coarse in-mask samples with renormalised weights, values x2, 0 outside
// the fine mask (Sec. IV-B).  Also ubar = u_w = u and p = 0 on the fine
// level.  Returns w in w_out (the next stage's warp vector).
template <int S, bool CG>
__device__ __forceinline__ float upsample_px(const LevelView& C, const LevelView& F, int x, int y,
                                             float2& w_out) {
  size_t o = (size_t)y * F.P + x;
  float u = 0.f, wx = 0.f, wy = 0.f;
  if (F.mask[o] & MASK_IN) {
    float X = fminf(fmaxf(((float)x + 0.5f) * 0.5f - 0.5f, 0.f), (float)(C.W - 1));
    float Y = fminf(fmaxf(((float)y + 0.5f) * 0.5f - 0.5f, 0.f), (float)(C.H - 1));
    int x0 = min((int)floorf(X), max(C.W - 2, 0));
    int y0 = min((int)floorf(Y), max(C.H - 2, 0));
    int x1 = min(x0 + 1, C.W - 1), y1 = min(y0 + 1, C.H - 1);
    float ax = X - (float)x0, ay = Y - (float)y0;
    int xs[4] = {x0, x1, x0, x1}, ys[4] = {y0, y0, y1, y1};
    float ws[4] = {(1.f - ax) * (1.f - ay), ax * (1.f - ay), (1.f - ax) * ay, ax * ay};
    float den = 0.f, nu = 0.f, nx = 0.f, ny = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      size_t ci = (size_t)ys[k] * C.P + xs[k];
      if (C.mask[ci] & MASK_IN) {
        float2 cw = ldf2<CG>(C.w + ci);
        den += ws[k];
        nu += ws[k] * ldf<CG>(C.u + ci);
        nx += ws[k] * cw.x;
        ny += ws[k] * cw.y;
      }
    }
    if (den > 0.f) {
      float s = 2.f / den;
      u = nu * s; wx = nx * s; wy = ny * s;
    }
  }
  F.u[o] = u; F.ubar[o] = u; F.uw[o] = u;
  w_out = make_float2(wx, wy);
  F.w[o] = w_out;
  sst<S>(F.p1, o, 0.f); sst<S>(F.p2, o, 0.f);
  return u;
}

// ------------------------------------------------------------ tensor + steps
struct TensorAt {
  float sx, sy;            // T^1/2 = I - s s^T
  float aa, bb, cc;        // |a|, |b|, |c|
};

// T^1/2 = e n n^T + n_perp n_perp^T = I - (1 - e) n n^T  (Eq. 12) with
// e = exp(-beta |grad I0|^eta), grad I0 by central differences on the mask
// (one-sided at its edge, 0 where both neighbours leave it).
template <int S>
__device__ __forceinline__ TensorAt tensor_at(const LevelView& L, int x, int y, float beta,
                                              float eta) {
  TensorAt t;
  size_t i = (size_t)y * L.P + x;
  if (!(L.mask[i] & MASK_IN)) { t.sx = t.sy = 0.f; t.aa = 1.f; t.bb = 0.f; t.cc = 1.f; return t; }
  auto I0 = [&](size_t k) { return sld<S>(L.I0, k); };
  float c = I0(i);
  bool r = x + 1 < L.W && (L.mask[i + 1] & MASK_IN);
  bool l = x > 0 && (L.mask[i - 1] & MASK_IN);
  bool d = y + 1 < L.H && (L.mask[i + L.P] & MASK_IN);
  bool u = y > 0 && (L.mask[i - L.P] & MASK_IN);
  float gx = 0.f, gy = 0.f;
  if (r && l) gx = 0.5f * (I0(i + 1) - I0(i - 1));
  else if (r) gx = I0(i + 1) - c;
  else if (l) gx = c - I0(i - 1);
  if (d && u) gy = 0.5f * (I0(i + L.P) - I0(i - L.P));
  else if (d) gy = I0(i + L.P) - c;
  else if (u) gy = c - I0(i - L.P);
  float mag = sqrtf(gx * gx + gy * gy);
  if (mag < 1e-12f) { t.sx = t.sy = 0.f; t.aa = 1.f; t.bb = 0.f; t.cc = 1.f; return t; }
  float nx = gx / mag, ny = gy / mag;
  float one_minus_e = -expm1f(-beta * powf(mag, eta));
  float s = sqrtf(one_minus_e);
  t.sx = s * nx;
  t.sy = s * ny;
  t.aa = fabsf(1.f - one_minus_e * nx * nx);
  t.bb = fabsf(one_minus_e * nx * ny);
  t.cc = fabsf(1.f - one_minus_e * ny * ny);
  return t;
}

// Diagonal preconditioning (Pock-Chambolle 2011, alpha = 1) from the row and
// column sums of the entrywise bound |T^1/2| |grad| of K = T^1/2 grad:
//   sigma(x) = 1 / max(2(|a| m1 + |b| m2), 2(|b| m1 + |c| m2))
//   tau(x)   = 1 / ((|a|+|b|) m1 + (|b|+|c|) m2 at x,
//                   + (|a|+|b|) m1 at x - e1, + (|b|+|c|) m2 at x - e2)
template <int S>
__device__ __forceinline__ void tensor_px(const LevelView& L, int x, int y, float beta, float eta,
                                          int precond) {
  size_t i = (size_t)y * L.P + x;
  uint8_t m = L.mask[i];
  TensorAt t = tensor_at<S>(L, x, y, beta, eta);
  sst<S>(L.sx, i, t.sx);
  sst<S>(L.sy, i, t.sy);
  if (!precond) {
    const float s = 0.35355339059327373f;   // 1/sqrt(8)
    L.tau[i] = (m & MASK_IN) ? s : 0.f;       // tau = 0 holds u outside the mask
    L.sig[i] = s;
    return;
  }
  float m1 = (m & MASK_GX) ? 1.f : 0.f, m2 = (m & MASK_GY) ? 1.f : 0.f;
  float r1 = 2.f * (t.aa * m1 + t.bb * m2);
  float r2 = 2.f * (t.bb * m1 + t.cc * m2);
  float r = fmaxf(r1, r2);
  L.sig[i] = r > 0.f ? 1.f / r : 0.f;
  float col = (t.aa + t.bb) * m1 + (t.bb + t.cc) * m2;
  if (x > 0 && (L.mask[i - 1] & MASK_GX)) {
    TensorAt tl = tensor_at<S>(L, x - 1, y, beta, eta);
    col += tl.aa + tl.bb;
  }
  if (y > 0 && (L.mask[i - L.P] & MASK_GY)) {
    TensorAt tu = tensor_at<S>(L, x, y - 1, beta, eta);
    col += tu.bb + tu.cc;
  }
  L.tau[i] = (col > 0.f && (m & MASK_IN)) ? 1.f / col : 0.f;
}


// ------------------------------------------------------------ warp + linearise
// g = bicubic gamma'(x + w) renormalised (0 if |g| < 1e-6); I1w = I1(x + w);
// rho0 = I1w - I0 (Eq. 3, 9); I_u = I1(x + w + g) - I1w (Eq. 5, 7), or with
// `central` half the difference of the samples at x + w +- g (free of the
// I1w noise that the forward difference shares with rho0).  Starts a warp:
// ubar = u_w = u.
// The linearisation at one FOV pixel for warp vector w (shared by k_warp and
// k_clip_warp, so both give the same bits).
template <int S>
__device__ __forceinline__ void warp_px(const LevelView& L, int x, int y, size_t i, float2 w,
                                        int central, float& Iu, float& rho0, float2& g) {
  g = make_float2(0.f, 0.f);
  float2 gr = sample_bicubic2(L.gamma, L.W, L.H, L.P, x, w.x, y, w.y);
  float n = sqrtf(gr.x * gr.x + gr.y * gr.y);
  if (n >= 1e-6f) g = make_float2(gr.x / n, gr.y / n);
  float I1w = sample_bilinear_s<S>(L.I1, L.W, L.H, L.P, x, w.x, y, w.y);
  float I1g = sample_bilinear_s<S>(L.I1, L.W, L.H, L.P, x, w.x + g.x, y, w.y + g.y);
  if (central) {
    float I1m = sample_bilinear_s<S>(L.I1, L.W, L.H, L.P, x, w.x - g.x, y, w.y - g.y);
    Iu = 0.5f * (I1g - I1m);
  } else {
    Iu = I1g - I1w;
  }
  rho0 = I1w - sld<S>(L.I0, i);
}

// ------------------------------------------------------------ clip + update
// du = clamp(u - u_w, +-du_max); u_{w+1} = u_w + du; w += du g (Algorithm 1,
// Eq. 8-9).  The primal state continues from u_{w+1}.
template <bool CG>
__device__ __forceinline__ float clip_px(const LevelView& L, size_t i, float du_max,
                                         float2& w) {
  float uw = ldf<CG>(L.uw + i);
  float du = fminf(fmaxf(__fsub_rn(ldf<CG>(L.u + i), uw), -du_max), du_max);
  float2 g = ldf2<CG>(L.g + i);
  w = ldf2<CG>(L.w + i);
  w = make_float2(fmaf(du, g.x, w.x), fmaf(du, g.y, w.y));
  return __fadd_rn(uw, du);
}

}  // namespace fs
