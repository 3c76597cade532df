// k_pd.cu -- temporally blocked primal-dual iterations (Eq. 11, 13).
//
// One CTA owns a footprint of FW x (NY * R) pixels: an interior tile plus a
// halo of B pixels on every side.  Thread (tx, ty) keeps the column tx,
// rows ty*R .. ty*R + R - 1 of the footprint in registers (state u, ubar, p
// and the per-warp constants); shared memory only carries what neighbours
// exchange (ubar, and the masked products T^1/2 p).  One iteration makes the
// dependency cone grow by one pixel in every direction, so after n <= B
// iterations the interior is exact and is written back; the halo is
// recomputed by the neighbouring CTAs.  Two CTA barriers per iteration.
// The state is read from one buffer set and written to the other, so no CTA
// can see a neighbour's updated interior while it loads its halo.
//
// Per pixel and iteration, with K = T^1/2 grad and T^1/2 = I - s s^T:
//   p    <- P((p + sigma K ubar) / (1 + sigma eps)),   P(q) = q / max(1, |q|)
//   uh   <- u + tau div(T^1/2 p)
//   u'   <- shrink(uh): rb = rho0 + I_u (uh - u_w)
//           uh + tau lam I_u   if rb < -tau lam I_u^2
//           uh - tau lam I_u   if rb >  tau lam I_u^2
//           uh - rb / I_u      otherwise               (Eq. 13)
//   ubar <- u' + theta (u' - u)
// grad: forward differences masked by MASK_GX / MASK_GY; div: its exact
// negative adjoint; u is only updated inside the FOV mask.
#include "fs_kernels.h"

namespace fs {

template <int FW, int NY, int R>
__global__ void __launch_bounds__(FW * NY, 1)
k_pd(LevelView L, PDState in, PDState out, PDParams pp, int B, int n_iters) {
  constexpr int FH = NY * R;
  __shared__ float s_ub[FH][FW];
  __shared__ float s_t1[FH][FW];
  __shared__ float s_t2[FH][FW];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int IW = FW - 2 * B, IH = FH - 2 * B;
  const int ox = (int)blockIdx.x * IW - B;
  const int oy = (int)blockIdx.y * IH - B;
  const int gx = ox + tx;
  const bool col_in = gx >= 0 && gx < L.W;
  const float lam = pp.lam, eps = pp.eps, theta = pp.theta;

  float u[R], ub[R], p1[R], p2[R], sx[R], sy[R], dinv[R], sd[R], tau[R], step[R], Iu[R],
      rho0[R], uw[R], inv[R];
  unsigned mb = 0;

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int fy = ty * R + r;
    const int gy = oy + fy;
    if (col_in && gy >= 0 && gy < L.H) {
      const size_t i = (size_t)gy * L.P + gx;
      u[r] = in.u[i];
      ub[r] = in.ubar[i];
      p1[r] = in.p1[i];
      p2[r] = in.p2[i];
      sx[r] = L.sx[i];
      sy[r] = L.sy[i];
      const float sg = L.sig[i];
      dinv[r] = 1.f / (1.f + sg * eps);
      sd[r] = sg * dinv[r];
      tau[r] = L.tau[i];
      Iu[r] = L.Iu[i];
      step[r] = (tau[r] * lam) * Iu[r];              // tau lam I_u
      rho0[r] = L.rho0[i];
      uw[r] = L.uw[i];
      inv[r] = Iu[r] != 0.f ? 1.f / Iu[r] : 0.f;
      mb |= (unsigned)L.mask[i] << (3 * r);
    } else {
      u[r] = ub[r] = p1[r] = p2[r] = sx[r] = sy[r] = 0.f;
      dinv[r] = 1.f; sd[r] = 0.f; tau[r] = 0.f; step[r] = 0.f; Iu[r] = 0.f; rho0[r] = 0.f;
      uw[r] = 0.f; inv[r] = 0.f;
    }
    s_ub[fy][tx] = ub[r];
  }
  __syncthreads();

  const int txr = min(tx + 1, FW - 1);
  const int txl = max(tx - 1, 0);

#pragma unroll 1
  for (int it = 0; it < n_iters; ++it) {
    // ---- dual ascent + Huber resolvent + projection
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const unsigned m = mb >> (3 * r);
      const float right = s_ub[fy][txr];
      const float below = (r + 1 < R) ? ub[r + 1] : s_ub[min(fy + 1, FH - 1)][tx];
      const float g1 = (m & MASK_GX) ? right - ub[r] : 0.f;
      const float g2 = (m & MASK_GY) ? below - ub[r] : 0.f;
      const float d = sx[r] * g1 + sy[r] * g2;
      const float k1 = fmaf(-sx[r], d, g1);
      const float k2 = fmaf(-sy[r], d, g2);
      float q1 = fmaf(sd[r], k1, p1[r] * dinv[r]);
      float q2 = fmaf(sd[r], k2, p2[r] * dinv[r]);
      const float nn = q1 * q1 + q2 * q2;
      if (nn > 1.f) {
        const float s = rsqrtf(nn);
        q1 *= s;
        q2 *= s;
      }
      p1[r] = q1;
      p2[r] = q2;
      const float dp = sx[r] * q1 + sy[r] * q2;
      s_t1[fy][tx] = (m & MASK_GX) ? fmaf(-sx[r], dp, q1) : 0.f;
      s_t2[fy][tx] = (m & MASK_GY) ? fmaf(-sy[r], dp, q2) : 0.f;
    }
    __syncthreads();
    // ---- primal descent + pointwise shrinkage + over-relaxation
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const unsigned m = mb >> (3 * r);
      const float dv = s_t1[fy][tx] - s_t1[fy][txl] + s_t2[fy][tx] - s_t2[max(fy - 1, 0)][tx];
      float un = u[r];
      if (m & MASK_IN) {
        const float uh = fmaf(tau[r], dv, u[r]);
        // rho0 + I_u (uh - u_w): the small increment keeps its precision
        // (folding rho0 - I_u u_w first would round at the size of I_u u_w)
        const float rb = fmaf(Iu[r], uh - uw[r], rho0[r]);
        const float thr = step[r] * Iu[r];              // tau lam I_u^2
        un = rb < -thr ? uh + step[r] : (rb > thr ? uh - step[r] : fmaf(-rb, inv[r], uh));
      }
      ub[r] = fmaf(theta, un - u[r], un);
      u[r] = un;
      s_ub[fy][tx] = ub[r];
    }
    __syncthreads();
  }

  if (!col_in || tx < B || tx >= FW - B) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int fy = ty * R + r;
    const int gy = oy + fy;
    if (fy < B || fy >= FH - B || gy < 0 || gy >= L.H) continue;
    const size_t i = (size_t)gy * L.P + gx;
    out.u[i] = u[r];
    out.ubar[i] = ub[r];
    out.p1[i] = p1[r];
    out.p2[i] = p2[r];
  }
}

template <int FW, int NY, int R>
static cudaError_t launch_pd_t(const LevelView& L, const PDState& in, const PDState& out,
                               const PDParams& pp, int B, int n, cudaStream_t st) {
  const int IW = FW - 2 * B, IH = NY * R - 2 * B;
  if (IW <= 0 || IH <= 0 || n < 0 || n > B) return cudaErrorInvalidValue;
  dim3 grid((L.W + IW - 1) / IW, (L.H + IH - 1) / IH);
  k_pd<FW, NY, R><<<grid, dim3(FW, NY), 0, st>>>(L, in, out, pp, B, n);
  return cudaGetLastError();
}

cudaError_t launch_pd(int variant, const LevelView& L, const PDState& in, const PDState& out,
                      const PDParams& pp, int B, int n, cudaStream_t st) {
  switch (variant) {
    case PD_TILE_64: return launch_pd_t<64, 8, 8>(L, in, out, pp, B, n, st);
    case PD_TILE_32: return launch_pd_t<32, 8, 4>(L, in, out, pp, B, n, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fs
