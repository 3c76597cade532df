// fs_device.cuh -- FP32 device math shared by the library's kernels:
// camera models, sampling, and the per-level argument blocks.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace fs {

// Mask bits stored per pixel (uint8):
//   MASK_IN  the pixel lies inside the FOV circle (Sec. IV-B)
//   MASK_GX  the forward difference along x stays inside (Neumann, Sec. IV-B)
//   MASK_GY  the forward difference along y stays inside
constexpr uint8_t MASK_IN = 1, MASK_GX = 2, MASK_GY = 4;

// Radially symmetric camera, pixel = c + f * r(theta) * (X, Y)/|(X, Y)|.
struct DevCam {
  int model;            // 0 pinhole, 1 equidistant, 2 Kannala-Brandt, 3 unified
                        // (k1 = xi), 4 enhanced unified (k1 = alpha, k2 = beta)
  float fx, fy, cx, cy;
  float k1, k2, k3, k4;
  float theta_max;      // FOV half-angle (radians)
  float r_max;          // r(theta_max)
};

__host__ __device__ __forceinline__ float cam_r(const DevCam& c, float th) {
  if (c.model == 0) return tanf(th);
  if (c.model == 1) return th;
  if (c.model == 3) return sinf(th) / (cosf(th) + c.k1);
  if (c.model == 4) {
    float s = sinf(th), cs = cosf(th);
    return s / (c.k1 * sqrtf(c.k2 * s * s + cs * cs) + (1.f - c.k1) * cs);
  }
  float t2 = th * th;
  return th * (1.f + t2 * (c.k1 + t2 * (c.k2 + t2 * (c.k3 + t2 * c.k4))));
}

// dr/dtheta
__host__ __device__ __forceinline__ float cam_dr(const DevCam& c, float th) {
  if (c.model == 0) { float cs = cosf(th); return 1.f / (cs * cs); }
  if (c.model == 1) return 1.f;
  if (c.model == 3) {
    float cs = cosf(th), d = cs + c.k1;
    return (1.f + c.k1 * cs) / (d * d);
  }
  if (c.model == 4) {
    float s = sinf(th), cs = cosf(th), q = sqrtf(c.k2 * s * s + cs * cs);
    float D = c.k1 * q + (1.f - c.k1) * cs;
    float dD = c.k1 * s * cs * (c.k2 - 1.f) / q - (1.f - c.k1) * s;
    return (cs * D - s * dD) / (D * D);
  }
  float t2 = th * th;
  return 1.f + t2 * (3.f * c.k1 + t2 * (5.f * c.k2 + t2 * (7.f * c.k3 + t2 * 9.f * c.k4)));
}

// theta with r(theta) = rn on [0, theta_max].  Pinhole and equidistant:
// closed form.  Unified models: closed form (Sec. III-D), clamped to
// theta_max for radii beyond the FOV circle, as the bracketed solve below
// is.  Kannala-Brandt, whose r(theta) can bend strongly near the FOV edge:
// 10 bisection steps first narrow [0, theta_max] to a bracket of width
// theta_max / 1024, then 8 Newton steps converge inside it (a step that
// leaves the bracket is replaced by its midpoint).  r must increase on the
// interval (checked at handle creation).
__device__ __forceinline__ float cam_theta(const DevCam& c, float rn) {
  if (c.model == 1) return rn;
  if (c.model == 0) return atanf(rn);
  if (c.model == 3) {
    // closed form: the ray is (eta m, eta - xi), eta = (xi + sqrt(1 + (1 - xi^2)
    // r^2)) / (1 + r^2)
    float r2 = rn * rn;
    float eta = (c.k1 + sqrtf(fmaxf(1.f + (1.f - c.k1 * c.k1) * r2, 0.f))) / (1.f + r2);
    return fminf(atan2f(eta * rn, eta - c.k1), c.theta_max);
  }
  if (c.model == 4) {
    // closed form: the ray is (m, m_z), m_z = (1 - beta alpha^2 r^2) /
    // (alpha sqrt(1 - (2 alpha - 1) beta r^2) + 1 - alpha)
    float r2 = rn * rn, a = c.k1, b = c.k2;
    float mz = (1.f - b * a * a * r2) /
               (a * sqrtf(fmaxf(1.f - (2.f * a - 1.f) * b * r2, 0.f)) + 1.f - a);
    return fminf(atan2f(rn, mz), c.theta_max);
  }
  float lo = 0.f, hi = c.theta_max;
#pragma unroll 1
  for (int i = 0; i < 10; ++i) {
    float mid = 0.5f * (lo + hi);
    if (cam_r(c, mid) > rn) hi = mid; else lo = mid;
  }
  float th = 0.5f * (lo + hi);
#pragma unroll 1
  for (int i = 0; i < 8; ++i) {
    float f = cam_r(c, th) - rn;
    if (f > 0.f) hi = th; else lo = th;
    float nt = th - f / cam_dr(c, th);
    th = (nt >= lo && nt <= hi) ? nt : 0.5f * (lo + hi);
  }
  return th;
}

struct Ray {
  float x, y, z;        // unit direction
  float ux, uy;         // in-plane unit direction (x, y)/|(x, y)|, (1, 0) on axis
  float theta;
};

__device__ __forceinline__ Ray cam_unproject(const DevCam& c, float px, float py) {
  float mx = (px - c.cx) / c.fx;
  float my = (py - c.cy) / c.fy;
  float rn = sqrtf(mx * mx + my * my);
  Ray r;
  r.theta = cam_theta(c, rn);
  float s, co;
  sincosf(r.theta, &s, &co);
  if (rn > 0.f) { r.ux = mx / rn; r.uy = my / rn; } else { r.ux = 1.f; r.uy = 0.f; }
  r.x = s * r.ux;
  r.y = s * r.uy;
  r.z = co;
  return r;
}

__device__ __forceinline__ float2 cam_project(const DevCam& c, float X, float Y, float Z) {
  float rho = sqrtf(X * X + Y * Y);
  float th = atan2f(rho, Z);
  float r = cam_r(c, th);
  float mx = 0.f, my = 0.f;
  if (rho > 0.f) { mx = r * X / rho; my = r * Y / rho; }
  return make_float2(c.fx * mx + c.cx, c.fy * my + c.cy);
}

// Image-plane velocity d/ds pi(X + s t) at s = 0 for a unit ray X, by the
// chain rule through rho = |(X, Y)| and theta = atan2(rho, Z):
//   dp = f * ( r'(theta) dtheta u + r(theta)/rho (t_xy - u drho) ),
//   drho = u . t_xy, dtheta = Z drho - rho t_z  (|X| = 1),
// with the tangential part written through the 2-D cross product to avoid
// cancellation where t_xy is nearly parallel to u.
__device__ __forceinline__ float2 cam_velocity(const DevCam& c, const Ray& X,
                                               float tx, float ty, float tz) {
  float rho = sqrtf(X.x * X.x + X.y * X.y);
  if (rho < 1e-6f) return make_float2(c.fx * tx / X.z, c.fy * ty / X.z);
  float drho = X.ux * tx + X.uy * ty;
  float dth = X.z * drho - rho * tz;
  float rad = cam_dr(c, X.theta) * dth;
  float tan_scale = cam_r(c, X.theta) / rho;
  // t_xy - u (u . t_xy) = u_perp (u_perp . t_xy), u_perp = (-u_y, u_x)
  float cr = X.ux * ty - X.uy * tx;
  float vx = rad * X.ux - tan_scale * X.uy * cr;
  float vy = rad * X.uy + tan_scale * X.ux * cr;
  return make_float2(c.fx * vx, c.fy * vy);
}

// ---------------------------------------------------------------- sampling

// Sample positions are passed as an integer pixel plus a real offset
// (x + dx, y + dy): splitting off the integer part of the offset keeps the
// fractional position exact to the precision of the offset itself instead of
// rounding x + dx at the magnitude of x (3e-5 px at x ~ 1000 in FP32).
struct Tap {
  int i0, i1;   // the two neighbouring samples
  float a;      // weight of i1
};

// Linear tap pair along one axis of length n for position x + d, the
// position clamped to [0, n - 1].
__device__ __forceinline__ Tap tap_linear(int x, float d, int n) {
  float fl = floorf(d);
  int b = x + (int)fl;
  float f = d - fl;                       // in [0, 1)
  Tap t;
  if (b < 0) { t.i0 = 0; t.a = 0.f; }
  else if (b >= n - 1) { t.i0 = max(n - 2, 0); t.a = n >= 2 ? 1.f : 0.f; }
  else { t.i0 = b; t.a = f; }
  t.i1 = min(t.i0 + 1, n - 1);
  return t;
}

// Bilinear sample at (x + dx, y + dy), position clamped to the image.
__device__ __forceinline__ float sample_bilinear(const float* __restrict__ img, int W, int H,
                                                 int P, int x, float dx, int y, float dy) {
  Tap tx = tap_linear(x, dx, W), ty = tap_linear(y, dy, H);
  const float* r0 = img + (size_t)ty.i0 * P;
  const float* r1 = img + (size_t)ty.i1 * P;
  float v00 = __ldg(r0 + tx.i0), v01 = __ldg(r0 + tx.i1);
  float v10 = __ldg(r1 + tx.i0), v11 = __ldg(r1 + tx.i1);
  float top = fmaf(tx.a, v01 - v00, v00);
  float bot = fmaf(tx.a, v11 - v10, v10);
  return fmaf(ty.a, bot - top, top);
}

// Keys cubic convolution weights (a = -0.5) for the 4 taps at offsets
// -1, 0, 1, 2 around floor(x), s = x - floor(x) in [0, 1).
__device__ __forceinline__ void keys_weights(float s, float w[4]) {
  const float A = -0.5f;
  float s1 = 1.f + s, s2 = 1.f - s, s3 = 2.f - s;
  w[0] = ((A * s1 - 5.f * A) * s1 + 8.f * A) * s1 - 4.f * A;
  w[1] = ((A + 2.f) * s - (A + 3.f)) * s * s + 1.f;
  w[2] = ((A + 2.f) * s2 - (A + 3.f)) * s2 * s2 + 1.f;
  w[3] = ((A * s3 - 5.f * A) * s3 + 8.f * A) * s3 - 4.f * A;
}

// Base index and fraction of x + d clamped to [0, n - 1] for the cubic taps.
__device__ __forceinline__ void cubic_base(int x, float d, int n, int& b, float& s) {
  float fl = floorf(d);
  b = x + (int)fl;
  s = d - fl;
  if (b < 0) { b = 0; s = 0.f; }
  else if (b >= n - 1) { b = n - 1; s = 0.f; }
}

// Bicubic sample of an interleaved float2 field at (x + dx, y + dy),
// position clamped to the image, taps repeating the edge.
__device__ __forceinline__ float2 sample_bicubic2(const float2* __restrict__ f, int W, int H,
                                                  int P, int x, float dx, int y, float dy) {
  int xi, yi;
  float sx_, sy_;
  cubic_base(x, dx, W, xi, sx_);
  cubic_base(y, dy, H, yi, sy_);
  float wx[4], wy[4];
  keys_weights(sx_, wx);
  keys_weights(sy_, wy);
  float sx = 0.f, sy = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int yy = min(max(yi + j - 1, 0), H - 1);
    const float2* row = f + (size_t)yy * P;
    float rx = 0.f, ry = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int xx = min(max(xi + i - 1, 0), W - 1);
      float2 v = __ldg(row + xx);
      rx += wx[i] * v.x;
      ry += wx[i] * v.y;
    }
    sx += wy[j] * rx;
    sy += wy[j] * ry;
  }
  return make_float2(sx, sy);
}

// ---------------------------------------------------------------- storage

// Storage of the images, warped gradients, tensor and dual fields: FP32,
// or FP16 / BF16 with all arithmetic still in FP32 (values are converted on
// load and rounded to nearest on store).
enum Storage { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

// Bytes of one element of a plane in storage st.
__host__ __device__ constexpr size_t storage_size(int st) { return st == ST_F32 ? 4 : 2; }

// A plane of one of those fields; its element type is the level's storage,
// fixed at compile time in every kernel that touches it (sld / sst).
struct SPlane {
  void* p;
};

template <int S>
__device__ __forceinline__ float sld(const SPlane& pl, size_t i) {
  if constexpr (S == ST_F16) return __half2float(__ldg((const __half*)pl.p + i));
  else if constexpr (S == ST_BF16) return __bfloat162float(__ldg((const __nv_bfloat16*)pl.p + i));
  else return __ldg((const float*)pl.p + i);
}

// Loads of planes that another CTA of the same launch may have written (the
// persistent schedule): CG = true reads through L2 only (ld.global.cg), so a
// line an SM's L1 cached earlier in the launch is never served stale.
// CG = false is the plain load the launch-per-stage kernels use.
template <bool CG>
__device__ __forceinline__ float ldf(const float* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <bool CG>
__device__ __forceinline__ float2 ldf2(const float2* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <int S, bool CG>
__device__ __forceinline__ float sld_m(const SPlane& pl, size_t i) {
  if constexpr (!CG) return sld<S>(pl, i);
  else if constexpr (S == ST_F16) return __half2float(__ldcg((const __half*)pl.p + i));
  else if constexpr (S == ST_BF16) return __bfloat162float(__ldcg((const __nv_bfloat16*)pl.p + i));
  else return __ldcg((const float*)pl.p + i);
}

template <int S>
__device__ __forceinline__ void sst(const SPlane& pl, size_t i, float v) {
  if constexpr (S == ST_F16) ((__half*)pl.p)[i] = __float2half_rn(v);
  else if constexpr (S == ST_BF16) ((__nv_bfloat16*)pl.p)[i] = __float2bfloat16_rn(v);
  else ((float*)pl.p)[i] = v;
}

// Bilinear sample of a stored plane at (x + dx, y + dy), clamped.
template <int S>
__device__ __forceinline__ float sample_bilinear_s(const SPlane& img, int W, int H, int P, int x,
                                                   float dx, int y, float dy) {
  Tap tx = tap_linear(x, dx, W), ty = tap_linear(y, dy, H);
  const size_t r0 = (size_t)ty.i0 * P, r1 = (size_t)ty.i1 * P;
  float v00 = sld<S>(img, r0 + tx.i0), v01 = sld<S>(img, r0 + tx.i1);
  float v10 = sld<S>(img, r1 + tx.i0), v11 = sld<S>(img, r1 + tx.i1);
  float top = fmaf(tx.a, v01 - v00, v00);
  float bot = fmaf(tx.a, v11 - v10, v10);
  return fmaf(ty.a, bot - top, top);
}

// ---------------------------------------------------------------- levels

// Device view of one pyramid level (pitch P elements per row).
struct LevelView {
  int W, H, P;
  int st;                // Storage of the SPlane fields
  const uint8_t* mask;
  SPlane I0, I1;
  float2* gamma;
  SPlane sx, sy;         // T^1/2 = I - s s^T, s = sqrt(1 - e) n  (Eq. 12)
  float *tau, *sig;      // primal / dual step sizes
  float *u, *ubar, *uw;
  SPlane p1, p2, Iu, rho0;
  // The per-pixel constants of a warp's primal-dual iterations (PxConst,
  // pd_math.cuh) other than s and tau: 1 / (1 + sigma eps), sigma times
  // that, |tau lam I_u| and u_w - rho0 / I_u; computed once per warp by
  // k_pd_consts from sigma, tau, I_u, rho0 and u_w as stored.
  float *dinv, *sd, *step, *c0;
  float2 *w, *g;
  float *u_alt, *ubar_alt;
  // The low parts of I0 and I1 while the pyramid is built (each image is
  // carried as a float-float value from the pre-rotation down to the
  // coarsest level, so that every stored level is its exact box mean
  // rounded once).  They share the planes of u_alt and ubar_alt, which hold
  // nothing between the primal-dual launches of a warp.
  float *I0lo, *I1lo;
  // TGV-L1 (Eq. 10): v, vbar (2 planes each) and q (4), null otherwise,
  // and an alternate set of the 12 state planes (u, ubar, v1, v2, vb1, vb2,
  // p1, p2, q11, q12, q21, q22) for the temporally blocked kernel
  float *v1, *v2, *vb1, *vb2, *q11, *q12, *q21, *q22;
  float* tgv_alt[12];     // ping-pong copies for k_pd
  SPlane p1_alt, p2_alt;
};

// Primal-dual state planes of one buffer set.
struct PDState {
  float *u, *ubar;
  SPlane p1, p2;
};

struct PDParams {
  float lam, eps, theta;
  // Chambolle-Pock Algorithm 2 steps (scalar steps only), per iteration of
  // a warp: x = tau_k / tau_0, y = 1 / (1 + sigma_k eps), z = sigma_k y,
  // w = theta_k; nullptr for the constant steps.  k0 = the warp's iterations
  // done before this launch.
  const float4* sched = nullptr;
  int k0 = 0;
};

}  // namespace fs
