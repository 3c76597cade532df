// k_level.cu -- per-level kernels of the fisheye stereo path other than the
// primal-dual iteration: trajectory field, calibration field and
// pre-rotation, pyramid down/up-sampling, tensor and step sizes,
// warp + linearisation, clip + update, triangulation.
#include "fs_kernels.h"
#include "level_px.cuh"
#include "pd_math.cuh"

namespace fs {

// ------------------------------------------------------------ float-float stores
// A plane value in storage S (rounded to nearest) and, in lo, the part of
// the float-float value v that the stored value leaves out.
template <int S>
__device__ __forceinline__ float round_storage(float v) {
  if constexpr (S == ST_F16) return __half2float(__float2half_rn(v));
  else if constexpr (S == ST_BF16) return __bfloat162float(__float2bfloat16_rn(v));
  else return v;
}

template <int S>
__device__ __forceinline__ void sst_df(const SPlane& pl, float* __restrict__ lo, size_t i, df v) {
  const float s = round_storage<S>(v.hi);
  sst<S>(pl, i, s);
  lo[i] = __fadd_rn(__fsub_rn(v.hi, s), v.lo);
}

template <int S>
__device__ __forceinline__ df sld_df(const SPlane& pl, const float* __restrict__ lo, size_t i) {
  return df{sld<S>(pl, i), lo[i]};
}

// ------------------------------------------------------------ trajectory field
// gamma'(x) = normalise(d/ds pi(pi^-1(x) + s t')) at s -> 0 (Sec. III-B,
// Eq. 6-7), evaluated as the analytic image-plane velocity of a point on the
// pixel's ray under the (pre-rotated) translation t' (unit vector).  The
// velocity and its normalisation are computed in float-float and rounded
// once.  Zero outside the mask and where the velocity vanishes (epipoles).
__global__ void k_trajectory(DevCamDF cam, df tx, df ty, df tz, LevelView L) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  float2 g = make_float2(0.f, 0.f);
  if (L.mask[i] & MASK_IN) {
    const RayDF r = cam_unproject_df(cam, x, y);
    df vx, vy;
    cam_velocity_df(cam, r, tx, ty, tz, vx, vy);
    const df n = dd_sqrt(dd_add(dd_mul(vx, vx), dd_mul(vy, vy)));
    if (n.hi >= 1e-3f) g = make_float2(dd_div(vx, n).hi, dd_div(vy, n).hi);
  }
  L.gamma[i] = g;
}

// ------------------------------------------------------------ calibration field
// c(x) = pi_1(R X) - x, X = pi_0^-1(x), at the level-0 FOV pixels (Sec. IV-A,
// the pre-rotation: t = 0), 0 elsewhere; in float-float, stored as the float
// pair (hi x, hi y, lo x, lo y).  x stands for pi_0(X), which it equals to
// about 1e-13 px.  (Two identical cameras with R = I have the field exactly
// 0; the host writes that one without this kernel.)
__global__ void k_calib_field(DevCamDF c0, DevCamDF c1, RotDF R, const uint8_t* __restrict__ mask,
                              float4* __restrict__ field, int W, int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  size_t i = (size_t)y * P + x;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (mask[i] & MASK_IN) {
    const RayDF r = cam_unproject_df(c0, x, y);
    const df X[3] = {dd_mul(r.s, r.ux), dd_mul(r.s, r.uy), r.c};
    df Y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      Y[k] = dd_add(dd_add(dd_mul(R.r[3 * k], X[0]), dd_mul(R.r[3 * k + 1], X[1])),
                    dd_mul(R.r[3 * k + 2], X[2]));
    df px, py;
    cam_project_df(c1, Y[0], Y[1], Y[2], px, py);
    const df dx = dd_sub(px, df_f((float)x)), dy = dd_sub(py, df_f((float)y));
    out = make_float4(dx.hi, dy.hi, dx.lo, dy.lo);
  }
  field[i] = out;
}

// ------------------------------------------------------------ pre-rotation
// I1'(x) = I1(x + c(x)), bilinear, position clamped to the image (Sec.
// IV-A); I1 dense FP32 (pitch W), output pitch P in the level's storage.
// The sample position and the interpolation are float-float; the result is
// stored rounded, its low part in lo (the start of the pyramid's carry).
struct TapDF {
  int i0, i1;   // the two neighbouring samples
  df a;         // weight of i1
};

__device__ __forceinline__ TapDF tap_linear_df(int x, df d, int n) {
  float fl;
  df f;
  dd_floor_frac(d, fl, f);
  const int b = x + (int)fl;
  TapDF t;
  if (b < 0) { t.i0 = 0; t.a = df_f(0.f); }
  else if (b >= n - 1) { t.i0 = max(n - 2, 0); t.a = df_f(n >= 2 ? 1.f : 0.f); }
  else { t.i0 = b; t.a = f; }
  t.i1 = min(t.i0 + 1, n - 1);
  return t;
}

template <int S>
__global__ void k_prerotate(const float* __restrict__ I1, const float4* __restrict__ field,
                            SPlane out, float* __restrict__ lo, int W, int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  size_t i = (size_t)y * P + x;
  const float4 c = field[i];
  const TapDF tx = tap_linear_df(x, df{c.x, c.z}, W), ty = tap_linear_df(y, df{c.y, c.w}, H);
  const float* r0 = I1 + (size_t)ty.i0 * W;
  const float* r1 = I1 + (size_t)ty.i1 * W;
  const float v00 = __ldg(r0 + tx.i0), v01 = __ldg(r0 + tx.i1);
  const float v10 = __ldg(r1 + tx.i0), v11 = __ldg(r1 + tx.i1);
  const df top = dd_add(df_f(v00), dd_mul(tx.a, two_sum(v01, -v00)));
  const df bot = dd_add(df_f(v10), dd_mul(tx.a, two_sum(v11, -v10)));
  sst_df<S>(out, lo, i, dd_add(top, dd_mul(ty.a, dd_sub(bot, top))));
}

// Dense FP32 (pitch W) -> pitched plane in the level's storage, with the
// low part of the rounding in lo (0 for FP32 storage): the finest level of
// I0, or a level image written through fs_buffer_write.
template <int S>
__global__ void k_copy_in_s(const float* __restrict__ src, SPlane dst, float* __restrict__ lo,
                            int W, int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  sst_df<S>(dst, lo, (size_t)y * P + x, df_f(src[(size_t)y * W + x]));
}

// Dense (pitch W) -> pitched FP32 copy, used for the warm-start input.
__global__ void k_copy_in(const float* __restrict__ src, float* __restrict__ dst, int W, int H,
                          int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  dst[(size_t)y * P + x] = src[(size_t)y * W + x];
}

// ------------------------------------------------------------ pyramid
// 2x2 box mean over the children inside the finer mask (all existing
// children when none is inside), for I0 and I1 together (Sec. IV-B).  The
// children are float-float (stored value + low part), the mean is formed in
// float-float and stored rounded with its own low part, so each level is
// the exact mean of the exact finer level, rounded once.
template <int S>
__global__ void k_downsample(LevelView F, LevelView C) {
  int X = blockIdx.x * blockDim.x + threadIdx.x;
  int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= C.W || Y >= C.H) return;
  df s0 = df_f(0.f), s1 = df_f(0.f), a0 = df_f(0.f), a1 = df_f(0.f);
  int nin = 0, nall = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int x = 2 * X + i, y = 2 * Y + j;
      if (x < F.W && y < F.H) {
        size_t k = (size_t)y * F.P + x;
        const df v0 = sld_df<S>(F.I0, F.I0lo, k), v1 = sld_df<S>(F.I1, F.I1lo, k);
        a0 = dd_add(a0, v0); a1 = dd_add(a1, v1); ++nall;
        if (F.mask[k] & MASK_IN) { s0 = dd_add(s0, v0); s1 = dd_add(s1, v1); ++nin; }
      }
    }
  }
  size_t o = (size_t)Y * C.P + X;
  if (nin > 0) {
    sst_df<S>(C.I0, C.I0lo, o, dd_div_f(s0, (float)nin));
    sst_df<S>(C.I1, C.I1lo, o, dd_div_f(s1, (float)nin));
  } else {
    sst_df<S>(C.I0, C.I0lo, o, dd_div_f(a0, (float)nall));
    sst_df<S>(C.I1, C.I1lo, o, dd_div_f(a1, (float)nall));
  }
}

// u, w of level C (coarse) -> level F (fine): upsample_px at every pixel.
template <int S>
__global__ void k_upsample(LevelView C, LevelView F) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= F.W || y >= F.H) return;
  float2 w;
  upsample_px<S, false>(C, F, x, y, w);
}

// Warm start at the finest level from a disparity already in L.u: w is
// rebuilt by walking along the trajectory field in n = ceil(|d| / du_max)
// equal steps of d / n, each along the renormalised bicubic gamma' at the
// current point; ubar = u_w = u, p = 0.  Non-finite disparities count as 0
// and n is capped at kMaxWarmSteps.
constexpr int kMaxWarmSteps = 16384;
template <int S>
__global__ void k_warm_start(LevelView L, float du_max) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  float d = L.u[i];
  if (!(L.mask[i] & MASK_IN) || !isfinite(d)) d = 0.f;
  float2 w = make_float2(0.f, 0.f);
  int n = (int)fminf(ceilf(fabsf(d) / du_max), (float)kMaxWarmSteps);
  if (n > 0) {
    float step = d / (float)n;
    for (int k = 0; k < n; ++k) {
      float2 gr = sample_bicubic2(L.gamma, L.W, L.H, L.P, x, w.x, y, w.y);
      float nr = sqrtf(gr.x * gr.x + gr.y * gr.y);
      if (nr >= 1e-6f) {
        w.x = fmaf(step, gr.x / nr, w.x);
        w.y = fmaf(step, gr.y / nr, w.y);
      }
    }
  }
  L.u[i] = d; L.ubar[i] = d; L.uw[i] = d;
  L.w[i] = w;
  sst<S>(L.p1, i, 0.f); sst<S>(L.p2, i, 0.f);
}

// Warm start at the finest level from its own last u and w (a video
// stream's next frame): ubar = u_w = u, p = 0, w kept.  Non-finite
// disparities count as 0 (with w = 0).
template <int S>
__global__ void k_continue(LevelView L) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  float d = L.u[i];
  if (!(L.mask[i] & MASK_IN) || !isfinite(d)) {
    d = 0.f;
    L.w[i] = make_float2(0.f, 0.f);
  }
  L.u[i] = d; L.ubar[i] = d; L.uw[i] = d;
  sst<S>(L.p1, i, 0.f); sst<S>(L.p2, i, 0.f);
}

// Zero state at the coarsest level (Algorithm 1: u_0 = 0, w_0 = 0).
template <int S>
__global__ void k_zero_state(LevelView L) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  zero_px<S>(L, (size_t)y * L.P + x);
}

// ------------------------------------------------------------ tensor + steps
template <int S>
__global__ void k_tensor(LevelView L, float beta, float eta, int precond) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  tensor_px<S>(L, x, y, beta, eta, precond);
}

// ------------------------------------------------------------ warp + linearise
// The per-warp constants of the primal-dual iterations at pixel i
// (launch_pd_consts' values: px_make of the stored sigma, tau, I_u, rho0
// and u_w), written by the kernels that start a warp while they hold
// I_u, rho0 and u_w.
template <int S>
__device__ __forceinline__ void pd_consts_px(const LevelView& L, size_t i, float Iu, float rho0,
                                             float uw, float lam, float eps) {
  PxRaw raw;
  raw.sx = raw.sy = 0.f;                     // not used by px_make's outputs below
  raw.sig = L.sig[i];
  raw.tau = L.tau[i];
  raw.Iu = round_storage<S>(Iu);
  raw.rho0 = round_storage<S>(rho0);
  raw.uw = uw;
  PxConst c;
  px_make(raw, lam, eps, c);
  L.dinv[i] = c.dinv;
  L.sd[i] = c.sd;
  L.step[i] = c.step;
  L.c0[i] = c.c0;
}

// consts: also write the per-warp constants of the primal-dual iterations
// (pd_consts_px; Huber-TV handles).
template <int S>
__global__ void k_warp(LevelView L, int central, float lam, float eps, int consts) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  float Iu = 0.f, rho0 = 0.f;
  float2 g = make_float2(0.f, 0.f);
  if (L.mask[i] & MASK_IN) warp_px<S>(L, x, y, i, L.w[i], central, Iu, rho0, g);
  sst<S>(L.Iu, i, Iu);
  sst<S>(L.rho0, i, rho0);
  L.g[i] = g;
  float u = L.u[i];
  L.ubar[i] = u;
  L.uw[i] = u;
  if (consts) pd_consts_px<S>(L, i, Iu, rho0, u, lam, eps);
}

// ------------------------------------------------------------ clip + update
__global__ void k_clip(LevelView L, float du_max) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  if (!(L.mask[i] & MASK_IN)) return;
  float2 w;
  float un = clip_px<false>(L, i, du_max, w);
  L.u[i] = un;
  L.ubar[i] = un;
  L.uw[i] = un;
  L.w[i] = w;
}

// The end of one warp and the start of the next in one pass: k_clip then
// k_warp at every pixel, with the updated w and u kept in registers (each
// pixel's clip and linearisation read only that pixel's state; the gathers
// read I1 and gamma', which neither writes).
template <int S>
__global__ void k_clip_warp(LevelView L, float du_max, int central, float lam, float eps,
                            int consts) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  float Iu = 0.f, rho0 = 0.f;
  float2 g = make_float2(0.f, 0.f);
  float u;
  if (L.mask[i] & MASK_IN) {
    float2 w;
    u = clip_px<false>(L, i, du_max, w);
    L.w[i] = w;
    L.u[i] = u;
    warp_px<S>(L, x, y, i, w, central, Iu, rho0, g);
  } else {
    u = L.u[i];
  }
  sst<S>(L.Iu, i, Iu);
  sst<S>(L.rho0, i, rho0);
  L.g[i] = g;
  L.ubar[i] = u;
  L.uw[i] = u;
  if (consts) pd_consts_px<S>(L, i, Iu, rho0, u, lam, eps);
}


// ------------------------------------------------------------ triangulation
// Range along the camera-0 ray of x from the rays pi^-1(x) and pi^-1(x + w)
// of the pre-rotated pair (virtual camera-1 centre C = -t'), closest point
// of the two lines: l0 = ((C x r1) . (r0 x r1)) / |r0 x r1|^2 (Sec. III-D).
__global__ void k_depth(LevelView L, DevCam cam, float Cx, float Cy, float Cz,
                        float* __restrict__ disp, float* __restrict__ depth) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x;
  size_t o = (size_t)y * L.W + x;
  bool in = L.mask[i] & MASK_IN;
  if (disp) disp[o] = in ? L.u[i] : 0.f;
  if (!depth) return;
  if (!in) { depth[o] = __int_as_float(0x7fc00000); return; }
  float2 w = L.w[i];
  if (w.x == 0.f && w.y == 0.f) {   // no displacement: the rays coincide, range +inf
    depth[o] = __int_as_float(0x7f800000);
    return;
  }
  Ray r0 = cam_unproject(cam, (float)x, (float)y);
  Ray r1 = cam_unproject(cam, (float)x + w.x, (float)y + w.y);
  float nx = r0.y * r1.z - r0.z * r1.y;
  float ny = r0.z * r1.x - r0.x * r1.z;
  float nz = r0.x * r1.y - r0.y * r1.x;
  float mx = Cy * r1.z - Cz * r1.y;
  float my = Cz * r1.x - Cx * r1.z;
  float mz = Cx * r1.y - Cy * r1.x;
  float den = nx * nx + ny * ny + nz * nz;
  depth[o] = den > 0.f ? (mx * nx + my * ny + mz * nz) / den : __int_as_float(0x7f800000);
}

// ------------------------------------------------------------ buffer access
__global__ void k_pack(const float* __restrict__ src, int stride, float* __restrict__ dst, int W,
                       int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  dst[(size_t)y * W + x] = src[((size_t)y * P + x) * stride];
}

__global__ void k_unpack(const float* __restrict__ src, float* __restrict__ dst, int stride,
                         int W, int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  dst[((size_t)y * P + x) * stride] = src[(size_t)y * W + x];
}

// Stored plane <-> dense FP32 (buffer access to the storage-typed fields).
template <int S>
__global__ void k_pack_s(SPlane src, float* __restrict__ dst, int W, int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  dst[(size_t)y * W + x] = sld<S>(src, (size_t)y * P + x);
}

template <int S>
__global__ void k_unpack_s(const float* __restrict__ src, SPlane dst, int W, int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  sst<S>(dst, (size_t)y * P + x, src[(size_t)y * W + x]);
}

__global__ void k_mask_to_float(const uint8_t* __restrict__ m, float* __restrict__ dst, int W,
                                int H, int P) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  dst[(size_t)y * W + x] = (m[(size_t)y * P + x] & MASK_IN) ? 1.f : 0.f;
}

// T^1/2 entries a, b, c from s: a = 1 - sx^2, b = -sx sy, c = 1 - sy^2.
template <int S>
__global__ void k_tensor_abc(LevelView L, float* __restrict__ dst) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  size_t i = (size_t)y * L.P + x, o = (size_t)y * L.W + x, n = (size_t)L.W * L.H;
  float sx = sld<S>(L.sx, i), sy = sld<S>(L.sy, i);
  dst[o] = 1.f - sx * sx;
  dst[n + o] = -sx * sy;
  dst[2 * n + o] = 1.f - sy * sy;
}

// ---------------------------------------------------------------- launchers
// Host launch of the storage-typed kernels: the level's storage picks the
// compiled instantiation.
namespace {
dim3 grid_of(int W, int H) { return dim3((W + 31) / 32, (H + 7) / 8); }
const dim3 kBlk(32, 8);
}  // namespace

#define FS_STORAGE_SWITCH(st, CALL)                           \
  switch (st) {                                               \
    case ST_F16: { constexpr int S = ST_F16; CALL; } break;   \
    case ST_BF16: { constexpr int S = ST_BF16; CALL; } break; \
    default: { constexpr int S = ST_F32; CALL; } break;       \
  }                                                           \
  return cudaGetLastError();

cudaError_t launch_prerotate(const float* I1, const float4* field, const LevelView& L0,
                             cudaStream_t st) {
  FS_STORAGE_SWITCH(L0.st, (k_prerotate<S><<<grid_of(L0.W, L0.H), kBlk, 0, st>>>(
                               I1, field, L0.I1, L0.I1lo, L0.W, L0.H, L0.P)))
}
cudaError_t launch_copy_in_image(const float* src, const LevelView& L, int which,
                                 cudaStream_t st) {
  const SPlane& dst = which == 0 ? L.I0 : L.I1;
  float* lo = which == 0 ? L.I0lo : L.I1lo;
  FS_STORAGE_SWITCH(L.st, (k_copy_in_s<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(
                              src, dst, lo, L.W, L.H, L.P)))
}
cudaError_t launch_downsample(const LevelView& F, const LevelView& C, cudaStream_t st) {
  FS_STORAGE_SWITCH(F.st, (k_downsample<S><<<grid_of(C.W, C.H), kBlk, 0, st>>>(F, C)))
}
cudaError_t launch_upsample(const LevelView& C, const LevelView& F, cudaStream_t st) {
  FS_STORAGE_SWITCH(F.st, (k_upsample<S><<<grid_of(F.W, F.H), kBlk, 0, st>>>(C, F)))
}
cudaError_t launch_zero_state(const LevelView& L, cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_zero_state<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(L)))
}
cudaError_t launch_warm_start(const LevelView& L, float du_max, cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_warm_start<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(L, du_max)))
}
cudaError_t launch_continue(const LevelView& L, cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_continue<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(L)))
}
cudaError_t launch_tensor(const LevelView& L, float beta, float eta, int precond,
                          cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_tensor<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(L, beta, eta,
                                                                          precond)))
}
cudaError_t launch_warp(const LevelView& L, int central, float lam, float eps, int consts,
                        cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_warp<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(L, central, lam, eps,
                                                                        consts)))
}

cudaError_t launch_clip_warp(const LevelView& L, float du_max, int central, float lam, float eps,
                             int consts, cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_clip_warp<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(
                              L, du_max, central, lam, eps, consts)))
}
cudaError_t launch_tensor_abc(const LevelView& L, float* dst, cudaStream_t st) {
  FS_STORAGE_SWITCH(L.st, (k_tensor_abc<S><<<grid_of(L.W, L.H), kBlk, 0, st>>>(L, dst)))
}
cudaError_t launch_pack_s(const SPlane& src, int storage, float* dst, int W, int H, int P,
                          cudaStream_t st) {
  FS_STORAGE_SWITCH(storage, (k_pack_s<S><<<grid_of(W, H), kBlk, 0, st>>>(src, dst, W, H, P)))
}
cudaError_t launch_unpack_s(const float* src, const SPlane& dst, int storage, int W, int H,
                            int P, cudaStream_t st) {
  FS_STORAGE_SWITCH(storage, (k_unpack_s<S><<<grid_of(W, H), kBlk, 0, st>>>(src, dst, W, H, P)))
}

}  // namespace fs
