// cam_df.cuh -- the camera models of fs_device.cuh in float-float arithmetic
// (df.cuh), for the fields that are computed once per pose: the trajectory
// field gamma' (Sec. III-B, Eq. 6-7) and the calibration field of the
// pre-rotation (Sec. IV-A).  Both are stored as floats; computing them to
// about 48 bits first makes each stored value its exact value rounded once.
#pragma once

#include "df.cuh"
#include "fs_device.cuh"

namespace fs {

// A radially symmetric camera, pixel = c + f r(theta) (X, Y)/|(X, Y)|, with
// its constants as float-float words (fs_api.cu builds it from the FP64
// calibration).  model as in DevCam; k1..k4 Kannala-Brandt, k1 = xi
// (unified), k1 = alpha, k2 = beta (enhanced unified).
struct DevCamDF {
  int model;
  df fx, fy, cx, cy;
  df k1, k2, k3, k4;
  df theta_max;          // FOV half-angle
  DevCam f32;            // the same camera in floats (starting points)
};

// A rotation matrix (row-major) as float-float words.
struct RotDF {
  df r[9];
};

// theta limited to the FOV half-angle, as cam_theta limits it.
__device__ __forceinline__ df clamp_fov_df(const DevCamDF& c, df th) {
  return dd_sub(th, c.theta_max).hi > 0.f ? c.theta_max : th;
}

// r(theta) and dr/dtheta given theta and (sin theta, cos theta).
__device__ __forceinline__ void cam_r_df(const DevCamDF& c, df th, df s, df co, df& r,
                                         df& dr) {
  const df one = df_f(1.f);
  switch (c.model) {
    case 0: {                                       // pinhole: tan
      r = dd_div(s, co);
      dr = dd_div(one, dd_mul(co, co));
      return;
    }
    case 1:                                         // equidistant
      r = th;
      dr = one;
      return;
    case 3: {                                       // unified: sin / (cos + xi)
      const df d = dd_add(co, c.k1);
      r = dd_div(s, d);
      dr = dd_div(dd_add(one, dd_mul(c.k1, co)), dd_mul(d, d));
      return;
    }
    case 4: {                                       // enhanced unified
      const df q = dd_sqrt(dd_add(dd_mul(c.k2, dd_mul(s, s)), dd_mul(co, co)));
      const df oma = dd_sub(one, c.k1);
      const df D = dd_add(dd_mul(c.k1, q), dd_mul(oma, co));
      const df dD = dd_sub(dd_div(dd_mul(dd_mul(c.k1, dd_mul(s, co)), dd_sub(c.k2, one)), q),
                           dd_mul(oma, s));
      r = dd_div(s, D);
      dr = dd_div(dd_sub(dd_mul(co, D), dd_mul(s, dD)), dd_mul(D, D));
      return;
    }
    default: {                                      // Kannala-Brandt polynomial
      const df t2 = dd_mul(th, th);
      df p = c.k4;
      p = dd_add(dd_mul(p, t2), c.k3);
      p = dd_add(dd_mul(p, t2), c.k2);
      p = dd_add(dd_mul(p, t2), c.k1);
      r = dd_mul(th, dd_add(one, dd_mul(p, t2)));
      df q = dd_mul_f(c.k4, 9.f);
      q = dd_add(dd_mul(q, t2), dd_mul_f(c.k3, 7.f));
      q = dd_add(dd_mul(q, t2), dd_mul_f(c.k2, 5.f));
      q = dd_add(dd_mul(q, t2), dd_mul_f(c.k1, 3.f));
      dr = dd_add(one, dd_mul(q, t2));
      return;
    }
  }
}

// theta with r(theta) = rn (the FOV half-angle clamp of cam_theta kept for
// radii beyond the FOV circle).
__device__ __forceinline__ df cam_theta_df(const DevCamDF& c, df rn) {
  const df one = df_f(1.f);
  if (c.model == 1) return rn;
  if (c.model == 0) return dd_atan2(rn, one);
  if (c.model == 3) {
    // the ray is (eta m, eta - xi), eta = (xi + sqrt(1 + (1 - xi^2) r^2)) / (1 + r^2)
    const df r2 = dd_mul(rn, rn);
    const df e = dd_div(dd_add(c.k1, dd_sqrt(dd_add(one, dd_mul(dd_sub(one, dd_mul(c.k1, c.k1)),
                                                                 r2)))),
                        dd_add(one, r2));
    return clamp_fov_df(c, dd_atan2(dd_mul(e, rn), dd_sub(e, c.k1)));
  }
  if (c.model == 4) {
    // the ray is (m, m_z), m_z = (1 - beta alpha^2 r^2) /
    // (alpha sqrt(1 - (2 alpha - 1) beta r^2) + 1 - alpha)
    const df r2 = dd_mul(rn, rn);
    const df a = c.k1, b = c.k2;
    const df num = dd_sub(one, dd_mul(dd_mul(b, dd_mul(a, a)), r2));
    const df rad = dd_sub(one, dd_mul(dd_mul(dd_sub(dd_mul_f(a, 2.f), one), b), r2));
    const df den = dd_add(dd_mul(a, dd_sqrt(rad)), dd_sub(one, a));
    return clamp_fov_df(c, dd_atan2(rn, dd_div(num, den)));
  }
  // Kannala-Brandt: the bracketed FP32 solve (relative error ~1e-7), then one
  // Newton step on r(theta) - rn with the residual in float-float, which
  // squares that error
  df th = df_f(cam_theta(c.f32, rn.hi));
  df r, dr;
  cam_r_df(c, th, th, th, r, dr);                   // sin / cos unused by this model
  th = dd_sub(th, dd_div(dd_sub(r, rn), dr));
  return clamp_fov_df(c, th);
}

// The unit ray of pixel (px, py): theta, (sin, cos) of theta and the
// in-plane unit direction u = m / |m| ((1, 0) on the axis).
struct RayDF {
  df th, s, c, ux, uy;
};

__device__ __forceinline__ RayDF cam_unproject_df(const DevCamDF& c, int px, int py) {
  const df mx = dd_div(dd_sub(df_f((float)px), c.cx), c.fx);
  const df my = dd_div(dd_sub(df_f((float)py), c.cy), c.fy);
  const df rn = dd_sqrt(dd_add(dd_mul(mx, mx), dd_mul(my, my)));
  RayDF r;
  r.th = cam_theta_df(c, rn);
  dd_sincos(r.th, r.s, r.c);
  if (rn.hi > 0.f) {
    r.ux = dd_div(mx, rn);
    r.uy = dd_div(my, rn);
  } else {
    r.ux = df_f(1.f);
    r.uy = df_f(0.f);
  }
  return r;
}

// Image-plane velocity d/ds pi(X + s t) at s = 0 for the unit ray X
// (cam_velocity in float-float): with rho = sin theta and z = cos theta,
//   dp = f (r'(theta) dtheta u + r(theta)/rho u_perp (u_perp . t_xy)),
//   dtheta = z (u . t_xy) - rho t_z;
// on the axis dp = f t_xy / z.
__device__ __forceinline__ void cam_velocity_df(const DevCamDF& c, const RayDF& X, df tx,
                                                df ty, df tz, df& vx, df& vy) {
  if (X.s.hi < 1e-6f) {
    vx = dd_div(dd_mul(c.fx, tx), X.c);
    vy = dd_div(dd_mul(c.fy, ty), X.c);
    return;
  }
  df r, dr;
  cam_r_df(c, X.th, X.s, X.c, r, dr);
  const df drho = dd_add(dd_mul(X.ux, tx), dd_mul(X.uy, ty));
  const df dth = dd_sub(dd_mul(X.c, drho), dd_mul(X.s, tz));
  const df rad = dd_mul(dr, dth);
  const df ts = dd_div(r, X.s);
  const df cr = dd_sub(dd_mul(X.ux, ty), dd_mul(X.uy, tx));
  const df tc = dd_mul(ts, cr);
  vx = dd_mul(c.fx, dd_sub(dd_mul(rad, X.ux), dd_mul(tc, X.uy)));
  vy = dd_mul(c.fy, dd_add(dd_mul(rad, X.uy), dd_mul(tc, X.ux)));
}

// Projection of the direction (X, Y, Z) (any length) through the camera.
__device__ __forceinline__ void cam_project_df(const DevCamDF& c, df X, df Y, df Z, df& px,
                                               df& py) {
  const df rho = dd_sqrt(dd_add(dd_mul(X, X), dd_mul(Y, Y)));
  if (!(rho.hi > 0.f)) {
    px = c.cx;
    py = c.cy;
    return;
  }
  const df nrm = dd_sqrt(dd_add(dd_mul(rho, rho), dd_mul(Z, Z)));
  const df s = dd_div(rho, nrm), co = dd_div(Z, nrm);
  const df th = (c.model == 1 || c.model == 2) ? dd_atan2(rho, Z) : df_f(0.f);
  df r, dr;
  cam_r_df(c, th, s, co, r, dr);
  const df k = dd_div(r, rho);
  px = dd_add(dd_mul(c.fx, dd_mul(k, X)), c.cx);
  py = dd_add(dd_mul(c.fy, dd_mul(k, Y)), c.cy);
}

}  // namespace fs
