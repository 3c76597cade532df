// pd_tile.cuh -- one CTA's temporally blocked primal-dual footprint (Eq. 11,
// 13): the body of k_pd, shared with the persistent schedule (k_persist.cu)
// so that both compute the same bits.
//
// The CTA owns a footprint of FW x (NY * R) pixels: an interior tile (bx,
// by) of (FW - 2B) x (NY R - 2B) pixels plus a halo of B pixels on every
// side.  Thread (tx, ty) keeps the column tx, rows ty*R .. ty*R + R - 1 of
// the footprint in registers (state u, ubar, p and the per-warp constants);
// shared memory only carries what neighbours exchange (ubar, and the masked
// products T^1/2 p).  One iteration makes the dependency cone grow by one
// pixel in every direction, so after n <= B iterations the interior is exact
// and is written back; the halo is recomputed by the neighbouring tiles.  Two
// CTA barriers per iteration.  The state is read from one buffer set and
// written to the other, so no tile sees a neighbour's updated interior while
// it loads its halo.
#pragma once

#include "pd_math.cuh"

namespace fs {

// The n_iters iterations of pd_tile on a thread's R rows (state in
// registers, neighbours through shared memory); MASKED as in px_dual.
template <int FW, int NY, int R, bool ACC, bool MASKED>
__device__ __forceinline__ void pd_iterate(const PDParams& pp, int n_iters, int tx, int ty,
                                           unsigned mb, const PxConst (&c)[R], float (&u)[R],
                                           float (&ub)[R], float (&p1)[R], float (&p2)[R],
                                           float theta, float (*s_ub)[FW], float (*s_t1)[FW],
                                           float (*s_t2)[FW]) {
  constexpr int FH = NY * R;
  const int txr = min(tx + 1, FW - 1);
  const int txl = max(tx - 1, 0);

  // a thread's own products stay in registers; shared memory carries t1 to
  // the right-hand neighbour and the last row's t2 to the thread below
  // (s_t2 holds one row per thread row: row ty is thread row ty's last)
  float t1r[R], t2r[R];
#pragma unroll 1
  for (int it = 0; it < n_iters; ++it) {
    float4 sk = make_float4(1.f, 0.f, 0.f, 0.f);
    if constexpr (ACC) {
      sk = pp.sched[pp.k0 + it];
      theta = sk.w;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const float right = s_ub[fy][txr];
      const float below = (r + 1 < R) ? ub[r + 1] : s_ub[min(fy + 1, FH - 1)][tx];
      PxConst cr = c[r];
      if constexpr (ACC) {
        cr.dinv = sk.y;
        cr.sd = sk.z;
      }
      px_dual<MASKED>(mb >> (3 * r), ub[r], right, below, cr, p1[r], p2[r], t1r[r], t2r[r]);
      s_t1[fy][tx] = t1r[r];
      if (r == R - 1) s_t2[ty][tx] = t2r[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      // the row above: this thread's previous row, or the last row of the
      // thread above (the top row of the footprint is halo: its own value)
      const float t2_up = r > 0 ? t2r[r - 1] : (ty > 0 ? s_t2[ty - 1][tx] : t2r[0]);
      const float dv = px_div(t1r[r], s_t1[fy][txl], t2r[r], t2_up);
      PxConst cr = c[r];
      if constexpr (ACC) {
        cr.tau = __fmul_rn(c[r].tau, sk.x);
        cr.step = __fmul_rn(c[r].step, sk.x);
      }
      const float un = px_primal(u[r], dv, cr);
      ub[r] = px_relax(un, u[r], theta);
      u[r] = un;
      s_ub[fy][tx] = ub[r];
    }
    __syncthreads();
  }

}

// pd_iterate with the rows paired for the packed FP32 operations (R even):
// pair j holds rows j and j + H (H = R / 2), so the rows below pair j are
// pair j + 1 and the rows above it pair j - 1; only the last pair's lower
// neighbours and the first pair's upper ones come from other threads.  The
// same values in the same order as pd_iterate (px_dual2 and friends), so
// the same bits.
template <int FW, int NY, int R, bool ACC, bool MASKED>
__device__ __forceinline__ void pd_iterate2(const PDParams& pp, int n_iters, int tx, int ty,
                                            unsigned mb, const PxConst (&c)[R], float (&u)[R],
                                            float (&ub)[R], float (&p1)[R], float (&p2)[R],
                                            float theta, float (*s_ub)[FW], float (*s_t1)[FW],
                                            float (*s_t2)[FW]) {
  static_assert(R % 2 == 0, "rows are paired");
  constexpr int FH = NY * R, H = R / 2;
  const int txr = min(tx + 1, FW - 1);
  const int txl = max(tx - 1, 0);
  PxConst2 c2[H];
  float2 u2[H], ub2[H], p12[H], p22[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    c2[j] = px_pair(c[j], c[j + H]);
    u2[j] = make_float2(u[j], u[j + H]);
    ub2[j] = make_float2(ub[j], ub[j + H]);
    p12[j] = make_float2(p1[j], p1[j + H]);
    p22[j] = make_float2(p2[j], p2[j + H]);
  }
  float2 t12[H], t22[H];
  float2 th2 = make_float2(theta, theta);
#pragma unroll 1
  for (int it = 0; it < n_iters; ++it) {
    float4 sk = make_float4(1.f, 0.f, 0.f, 0.f);
    if constexpr (ACC) {
      sk = pp.sched[pp.k0 + it];
      th2 = make_float2(sk.w, sk.w);
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int f0 = ty * R + j, f1 = f0 + H;       // the pair's two footprint rows
      const float2 right = make_float2(s_ub[f0][txr], s_ub[f1][txr]);
      // below: rows j + 1 and j + H + 1 (the next pair), or for the last pair
      // row R - 1... which is H (the first pair's second row) and the next
      // thread's first row
      const float2 below = (j + 1 < H) ? ub2[j + 1]
                                       : make_float2(ub2[0].y, s_ub[min(ty * R + R, FH - 1)][tx]);
      PxConst2 cr = c2[j];
      if constexpr (ACC) {
        cr.dinv = make_float2(sk.y, sk.y);
        cr.sd = make_float2(sk.z, sk.z);
      }
      px_dual2<MASKED>(mb >> (3 * j), mb >> (3 * (j + H)), ub2[j], right, below, cr, p12[j],
                       p22[j], t12[j], t22[j]);
      s_t1[f0][tx] = t12[j].x;
      s_t1[f1][tx] = t12[j].y;
      if (j == H - 1) s_t2[ty][tx] = t22[j].y;       // row R - 1
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const int f0 = ty * R + j, f1 = f0 + H;
      const float2 left = make_float2(s_t1[f0][txl], s_t1[f1][txl]);
      // above: rows j - 1 and j + H - 1 (the previous pair), or for the first
      // pair the thread above's last row (the top row of the footprint is
      // halo: its own value) and row H - 1 (the last pair's first row)
      const float2 up = (j > 0) ? t22[j - 1]
                                : make_float2(ty > 0 ? s_t2[ty - 1][tx] : t22[0].x,
                                              t22[H - 1].x);
      const float2 dv = px_div2(t12[j], left, t22[j], up);
      PxConst2 cr = c2[j];
      if constexpr (ACC) {
        cr.tau = __fmul2_rn(c2[j].tau, make_float2(sk.x, sk.x));
        cr.step = __fmul2_rn(c2[j].step, make_float2(sk.x, sk.x));
      }
      const float2 un = px_primal2(u2[j], dv, cr);
      ub2[j] = px_relax2(un, u2[j], th2);
      u2[j] = un;
      s_ub[f0][tx] = ub2[j].x;
      s_ub[f1][tx] = ub2[j].y;
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < H; ++j) {
    u[j] = u2[j].x;
    u[j + H] = u2[j].y;
    ub[j] = ub2[j].x;
    ub[j + H] = ub2[j].y;
    p1[j] = p12[j].x;
    p1[j + H] = p12[j].y;
    p2[j] = p22[j].x;
    p2[j + H] = p22[j].y;
  }
}

// The iteration loop for R rows per thread: paired (pd_iterate2) when R is
// even, else one row at a time.
template <int FW, int NY, int R, bool ACC, bool MASKED>
__device__ __forceinline__ void pd_iterate_rows(const PDParams& pp, int n_iters, int tx, int ty,
                                                unsigned mb, const PxConst (&c)[R],
                                                float (&u)[R], float (&ub)[R], float (&p1)[R],
                                                float (&p2)[R], float theta, float (*s_ub)[FW],
                                                float (*s_t1)[FW], float (*s_t2)[FW]) {
  if constexpr (R % 2 == 0)
    pd_iterate2<FW, NY, R, ACC, MASKED>(pp, n_iters, tx, ty, mb, c, u, ub, p1, p2, theta, s_ub,
                                        s_t1, s_t2);
  else
    pd_iterate<FW, NY, R, ACC, MASKED>(pp, n_iters, tx, ty, mb, c, u, ub, p1, p2, theta, s_ub,
                                       s_t1, s_t2);
}

// ACC: the accelerated step schedule of pp.sched (FP32 storage, scalar
// steps): iteration it of the block uses entry pp.k0 + it for sigma (all
// pixels), tau and the L1 step (scaled from the stored tau_0 values, 0 off
// the mask) and theta.  CG: the inputs may have been written by other CTAs
// of the same launch (loads through L2 only).  chained: a programmatic
// dependent launch of k_pd (constants loaded before the wait for the
// preceding launch, the state after it).  s_ub, s_t1: shared arrays of
// FH x FW floats, s_t2 of NY x FW.  PRE: the per-warp constants are read
// from L.dinv, L.sd, L.step, L.c0 (launch_pd_consts) instead of being
// derived here from sigma, I_u, rho0 and u_w (the same bits either way).
// Every thread of the CTA (FW x NY) must call it.
template <int FW, int NY, int R, int S, bool ACC, bool CG, bool PRE = false>
__device__ __forceinline__ void pd_tile(const LevelView& L, const PDState& in,
                                        const PDState& out, const PDParams& pp, int B,
                                        int n_iters, int bx, int by, int tx, int ty,
                                        float (*s_ub)[FW], float (*s_t1)[FW],
                                        float (*s_t2)[FW], bool chained) {
  constexpr int FH = NY * R;
  const int IW = FW - 2 * B, IH = FH - 2 * B;
  const int ox = bx * IW - B;
  const int oy = by * IH - B;
  const int gx = ox + tx;
  const bool col_in = gx >= 0 && gx < L.W;
  float theta = pp.theta;

  // Let the next launch of the chain be scheduled as soon as every CTA of
  // this one is resident (it waits for this grid's completion before it
  // reads the state, below).
  if (chained) cudaTriggerProgrammaticLaunchCompletion();

  float u[R], ub[R], p1[R], p2[R];
  PxConst c[R];
  unsigned mb = 0;
  // Addresses clamped into the level and a validity flag per row: every
  // load below is unconditional, so all of a thread's loads are in flight
  // at once instead of one row's after another's.
  const int gxc = min(max(gx, 0), L.W - 1);
  unsigned idx[R];            // < 2^31: levels are at most 32768 x 32768
  bool ok[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gy = oy + ty * R + r;
    ok[r] = col_in && gy >= 0 && gy < L.H;
    idx[r] = (unsigned)(min(max(gy, 0), L.H - 1) * L.P + gxc);
  }
  // per-warp constants first: written by earlier kernels, not by the
  // preceding launch of this chain
  if constexpr (PRE) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const unsigned i = idx[r];
      const float sx = sld_m<S, CG>(L.sx, i), sy = sld_m<S, CG>(L.sy, i);
      const float tau = ldf<CG>(L.tau + i), dinv = ldf<CG>(L.dinv + i);
      const float sd = ldf<CG>(L.sd + i), step = ldf<CG>(L.step + i), c0 = ldf<CG>(L.c0 + i);
      const unsigned m8 = L.mask[i];
      // outside the level: the constants of all-zero inputs (px_make)
      c[r].sx = ok[r] ? sx : 0.f;
      c[r].sy = ok[r] ? sy : 0.f;
      c[r].tau = ok[r] ? tau : 0.f;
      c[r].dinv = ok[r] ? dinv : 1.f;
      c[r].sd = ok[r] ? sd : 0.f;
      c[r].step = ok[r] ? step : 0.f;
      c[r].c0 = ok[r] ? c0 : 0.f;
      mb |= (ok[r] ? m8 : 0u) << (3 * r);
    }
  } else {
    PxRaw raw[R];
    unsigned char m8[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      px_fetch<S, CG>(L, idx[r], ok[r], raw[r]);
      m8[r] = ok[r] ? L.mask[idx[r]] : 0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      px_make(raw[r], pp.lam, pp.eps, c[r]);
      mb |= (unsigned)m8[r] << (3 * r);
    }
  }
  // The state is the preceding launch's output.  It is read through L2:
  // a chained launch starts while up to two launches before it still run
  // (each triggers the next at its start), so an SM's L1 may hold lines of
  // this buffer set that the launch two before cached before it was
  // rewritten.
  if (chained) cudaGridDependencySynchronize();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float a = ldf<true>(in.u + idx[r]), b = ldf<true>(in.ubar + idx[r]);
    const float q1 = sld_m<S, true>(in.p1, idx[r]), q2 = sld_m<S, true>(in.p2, idx[r]);
    u[r] = ok[r] ? a : 0.f;
    ub[r] = ok[r] ? b : 0.f;
    p1[r] = ok[r] ? q1 : 0.f;
    p2[r] = ok[r] ? q2 : 0.f;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) s_ub[ty * R + r][tx] = ub[r];
  __syncthreads();

  // Every footprint pixel inside the level with all three mask bits set
  // (the FOV covers it, with both forward neighbours): the loop without the
  // mask selects computes the same bits with fewer instructions.
  bool full = mb == (R == 1 ? 7u : R == 2 ? 077u : R == 4 ? 07777u : 077777777u);
#pragma unroll
  for (int r = 0; r < R; ++r) full = full && ok[r];
  if (__syncthreads_and(full))
    pd_iterate_rows<FW, NY, R, ACC, false>(pp, n_iters, tx, ty, mb, c, u, ub, p1, p2, theta,
                                           s_ub, s_t1, s_t2);
  else
    pd_iterate_rows<FW, NY, R, ACC, true>(pp, n_iters, tx, ty, mb, c, u, ub, p1, p2, theta,
                                          s_ub, s_t1, s_t2);

  if (!col_in || tx < B || tx >= FW - B) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int fy = ty * R + r;
    const int gy = oy + fy;
    if (fy < B || fy >= FH - B || gy < 0 || gy >= L.H) continue;
    const size_t i = (size_t)gy * L.P + gx;
    out.u[i] = u[r];
    out.ubar[i] = ub[r];
    sst<S>(out.p1, i, p1[r]);
    sst<S>(out.p2, i, p2[r]);
  }
}

}  // namespace fs
