// k_tgv.cu -- primal-dual iterations of the tensor-guided TGV-L1 energy
// (Sec. III-C, Eq. 10-11):
//
//   E(u, v) = lam |rho_bar(u)| + alpha1 |T^1/2 grad u - v| + alpha0 |grad v|
//
// The per-pixel steps are in pd_tgv_math.cuh.  Two schedules compute them
// with identical arithmetic:
//   * launch per step: a dual launch then a primal launch per iteration,
//     state in place (each pixel reads its right / lower neighbours in the
//     dual and its left / upper ones in the primal, so the launch boundary is
//     the only synchronisation needed);
//   * temporal blocking (k_tgv_blocked): a CTA keeps a 32 x 32 footprint's
//     whole state (u, ubar, v, vbar, p, q: 12 values per pixel) in registers
//     for n <= B iterations, exchanging ubar, vbar and the masked products
//     T^1/2 p and q with its neighbours through shared memory; the outer B
//     pixels of the footprint are halo, recomputed by the neighbouring CTAs.
//     State ping-pongs between the level's planes and an alternate set, and
//     a warp runs an even number of launches so that it ends in the level's
//     planes.
// Steps (Pock-Chambolle 2011 diagonal preconditioning of the block operator
// (T^1/2 grad u - v, grad v), in tgv_const): tau_u the Huber-TV tau; sigma_p
// = 1 / (max row sum of |T^1/2| |grad| + 1) from the stored Huber-TV sigma;
// sigma_q = 1/2; tau_v = 1 / (1 + the active differences touching the
// pixel); all 0 off the FOV mask, where nothing moves.
#include <atomic>

#include "fs_kernels.h"
#include "pd_tgv_math.cuh"

namespace fs {

namespace {

__device__ __forceinline__ void load_const(const LevelView& L, size_t i, int x, int y,
                                           const TgvParams& tp, TgvConst& c) {
  const unsigned m = L.mask[i];
  const unsigned ml = x > 0 ? L.mask[i - 1] : 0u;
  const unsigned mu = y > 0 ? L.mask[i - L.P] : 0u;
  tgv_const(m, ml, mu, sld<ST_F32>(L.sx, i), sld<ST_F32>(L.sy, i), L.sig[i], L.tau[i],
            sld<ST_F32>(L.Iu, i), sld<ST_F32>(L.rho0, i), L.uw[i], tp, c);
}

// t = T^1/2 p and the masked q of pixel k (what tgv_px_dual returns).
__device__ __forceinline__ void masked_products(const LevelView& L, size_t k, unsigned m,
                                                float& t1, float& t2, float& qx1, float& qx2,
                                                float& qy1, float& qy2) {
  const float sx = sld<ST_F32>(L.sx, k), sy = sld<ST_F32>(L.sy, k);
  const float p1 = sld<ST_F32>(L.p1, k), p2 = sld<ST_F32>(L.p2, k);
  const float dp = fmaf(sx, p1, __fmul_rn(sy, p2));
  const bool gx = m & MASK_GX, gy = m & MASK_GY;
  t1 = gx ? fmaf(-sx, dp, p1) : 0.f;
  t2 = gy ? fmaf(-sy, dp, p2) : 0.f;
  qx1 = gx ? L.q11[k] : 0.f;
  qx2 = gx ? L.q21[k] : 0.f;
  qy1 = gy ? L.q12[k] : 0.f;
  qy2 = gy ? L.q22[k] : 0.f;
}

}  // namespace

__global__ void k_tgv_dual(LevelView L, TgvParams tp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  const unsigned m = L.mask[i];
  if (!(m & MASK_IN)) return;
  TgvConst c;
  load_const(L, i, x, y, tp, c);
  const bool gx = m & MASK_GX, gy = m & MASK_GY;
  const size_t r = gx ? i + 1 : i, b = gy ? i + L.P : i;   // unread when masked
  float p1 = sld<ST_F32>(L.p1, i), p2 = sld<ST_F32>(L.p2, i);
  float q11 = L.q11[i], q12 = L.q12[i], q21 = L.q21[i], q22 = L.q22[i];
  float t1, t2, qx1, qx2, qy1, qy2;
  tgv_px_dual(m, L.ubar[i], L.ubar[r], L.ubar[b], L.vb1[i], L.vb1[r], L.vb1[b], L.vb2[i],
              L.vb2[r], L.vb2[b], c, tp, p1, p2, q11, q12, q21, q22, t1, t2, qx1, qx2, qy1,
              qy2);
  sst<ST_F32>(L.p1, i, p1);
  sst<ST_F32>(L.p2, i, p2);
  L.q11[i] = q11;
  L.q12[i] = q12;
  L.q21[i] = q21;
  L.q22[i] = q22;
}

__global__ void k_tgv_primal(LevelView L, TgvParams tp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  const unsigned m = L.mask[i];
  if (!(m & MASK_IN)) return;
  TgvConst c;
  load_const(L, i, x, y, tp, c);
  float t1, t2, qx1, qx2, qy1, qy2;
  float t1_l = 0.f, t2_l, qx1_l = 0.f, qx2_l = 0.f, qy1_l, qy2_l;
  float t1_u, t2_u = 0.f, qx1_u, qx2_u, qy1_u = 0.f, qy2_u = 0.f;
  masked_products(L, i, m, t1, t2, qx1, qx2, qy1, qy2);
  if (x > 0) masked_products(L, i - 1, L.mask[i - 1], t1_l, t2_l, qx1_l, qx2_l, qy1_l, qy2_l);
  if (y > 0)
    masked_products(L, i - L.P, L.mask[i - L.P], t1_u, t2_u, qx1_u, qx2_u, qy1_u, qy2_u);
  float u = L.u[i], ub, v1 = L.v1[i], v2 = L.v2[i], vb1, vb2;
  tgv_px_primal(t1, t1_l, t2, t2_u, qx1, qx1_l, qy1, qy1_u, qx2, qx2_l, qy2, qy2_u,
                sld<ST_F32>(L.p1, i), sld<ST_F32>(L.p2, i), c, tp.theta, u, ub, v1, v2, vb1,
                vb2);
  L.u[i] = u;
  L.ubar[i] = ub;
  L.v1[i] = v1;
  L.v2[i] = v2;
  L.vb1[i] = vb1;
  L.vb2[i] = vb2;
}

// One set of the 12 state planes of a TGV level.
struct TgvState {
  float* s[12];   // u, ubar, v1, v2, vb1, vb2, p1, p2, q11, q12, q21, q22
};

template <int FW, int NY, int R>
__global__ void __launch_bounds__(FW * NY, FW * NY >= 512 ? 1 : 2)
k_tgv_blocked(LevelView L, TgvState in, TgvState out, TgvParams tp, int B, int n_iters,
              int chained) {
  constexpr int FH = NY * R;
  // neighbours' values: ubar, vbar (read by the dual from the right / below)
  // and t, masked q (read by the primal from the left / above); nine FH x FW
  // planes of dynamic shared memory (tgv_smem_bytes)
  extern __shared__ float tgv_smem[];
  typedef float Plane[FW];
  Plane* s_ub = reinterpret_cast<Plane*>(tgv_smem + 0 * FH * FW);
  Plane* s_vb1 = reinterpret_cast<Plane*>(tgv_smem + 1 * FH * FW);
  Plane* s_vb2 = reinterpret_cast<Plane*>(tgv_smem + 2 * FH * FW);
  Plane* s_t1 = reinterpret_cast<Plane*>(tgv_smem + 3 * FH * FW);
  Plane* s_t2 = reinterpret_cast<Plane*>(tgv_smem + 4 * FH * FW);
  Plane* s_qx1 = reinterpret_cast<Plane*>(tgv_smem + 5 * FH * FW);
  Plane* s_qx2 = reinterpret_cast<Plane*>(tgv_smem + 6 * FH * FW);
  Plane* s_qy1 = reinterpret_cast<Plane*>(tgv_smem + 7 * FH * FW);
  Plane* s_qy2 = reinterpret_cast<Plane*>(tgv_smem + 8 * FH * FW);

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int IW = FW - 2 * B, IH = FH - 2 * B;
  const int ox = (int)blockIdx.x * IW - B;
  const int oy = (int)blockIdx.y * IH - B;
  const int gx = ox + tx;
  const bool col_in = gx >= 0 && gx < L.W;

  if (chained) cudaTriggerProgrammaticLaunchCompletion();

  // constants (written before the chain; unconditional loads from clamped
  // addresses, rows off the level made inert)
  const int gxc = min(max(gx, 0), L.W - 1);
  unsigned idx[R];
  bool ok[R];
  TgvConst c[R];
  unsigned mb = 0;
  {
    // every load first, from clamped addresses (the left / upper neighbour
    // of column / row 0 is read as the pixel itself and its bits dropped),
    // then the constants: a thread's loads are all in flight together
    float sx[R], sy[R], sg[R], ta[R], iu[R], r0[R], uw[R];
    unsigned m[R], ml[R], mu[R];
    const unsigned dl = gxc > 0 ? 1u : 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gy = oy + ty * R + r;
      ok[r] = col_in && gy >= 0 && gy < L.H;
      const int gyc = min(max(gy, 0), L.H - 1);
      idx[r] = (unsigned)(gyc * L.P + gxc);
      const unsigned du = gyc > 0 ? (unsigned)L.P : 0u;
      sx[r] = sld<ST_F32>(L.sx, idx[r]);
      sy[r] = sld<ST_F32>(L.sy, idx[r]);
      sg[r] = L.sig[idx[r]];
      ta[r] = L.tau[idx[r]];
      iu[r] = sld<ST_F32>(L.Iu, idx[r]);
      r0[r] = sld<ST_F32>(L.rho0, idx[r]);
      uw[r] = L.uw[idx[r]];
      m[r] = L.mask[idx[r]];
      ml[r] = L.mask[idx[r] - dl];
      mu[r] = L.mask[idx[r] - du];
      if (!dl) ml[r] = 0u;
      if (!du) mu[r] = 0u;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const unsigned mm = ok[r] ? m[r] : 0u;
      tgv_const(mm, ml[r], mu[r], sx[r], sy[r], sg[r], ta[r], iu[r], r0[r], uw[r], tp, c[r]);
      mb |= mm << (3 * r);
    }
  }
  // the state is the preceding launch's output, read through L2 (a chained
  // launch may start while the launch two before it still caches lines of
  // this buffer set in L1)
  if (chained) cudaGridDependencySynchronize();
  float u[R], ub[R], v1[R], v2[R], vb1[R], vb2[R], p1[R], p2[R], q11[R], q12[R], q21[R],
      q22[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const unsigned k = idx[r];
    float a[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) a[j] = __ldcg(in.s[j] + k);
    const float z = ok[r] ? 1.f : 0.f;   // off the level: inert zeros
    u[r] = a[0] * z; ub[r] = a[1] * z; v1[r] = a[2] * z; v2[r] = a[3] * z;
    vb1[r] = a[4] * z; vb2[r] = a[5] * z; p1[r] = a[6] * z; p2[r] = a[7] * z;
    q11[r] = a[8] * z; q12[r] = a[9] * z; q21[r] = a[10] * z; q22[r] = a[11] * z;
    const int fy = ty * R + r;
    s_ub[fy][tx] = ub[r];
    s_vb1[fy][tx] = vb1[r];
    s_vb2[fy][tx] = vb2[r];
  }
  __syncthreads();

  const int txr = min(tx + 1, FW - 1), txl = max(tx - 1, 0);
  if constexpr (R % 2 == 0) {
    // rows in pairs (j, j + H) on the packed FP32 operations, as in
    // pd_iterate2: the rows below pair j are pair j + 1, those above it
    // pair j - 1; the same values in the same order, so the same bits
    constexpr int H = R / 2;
    TgvConst2 c2[H];
    float2 u2[H], ub2[H], v12[H], v22[H], vb12[H], vb22[H], p12[H], p22[H];
    float2 q112[H], q122[H], q212[H], q222[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      c2[j] = tgv_pair(c[j], c[j + H]);
      u2[j] = make_float2(u[j], u[j + H]);
      ub2[j] = make_float2(ub[j], ub[j + H]);
      v12[j] = make_float2(v1[j], v1[j + H]);
      v22[j] = make_float2(v2[j], v2[j + H]);
      vb12[j] = make_float2(vb1[j], vb1[j + H]);
      vb22[j] = make_float2(vb2[j], vb2[j + H]);
      p12[j] = make_float2(p1[j], p1[j + H]);
      p22[j] = make_float2(p2[j], p2[j + H]);
      q112[j] = make_float2(q11[j], q11[j + H]);
      q122[j] = make_float2(q12[j], q12[j + H]);
      q212[j] = make_float2(q21[j], q21[j + H]);
      q222[j] = make_float2(q22[j], q22[j + H]);
    }
    const float2 th2 = make_float2(tp.theta, tp.theta);
    float2 t12[H], t22[H], qx12[H], qx22[H], qy12[H], qy22[H];
    const int fnext = min(ty * R + R, FH - 1);     // the thread below's first row
    const int fprev = max(ty * R - 1, 0);          // the thread above's last row
#pragma unroll 1
    for (int it = 0; it < n_iters; ++it) {
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const int f0 = ty * R + j, f1 = f0 + H;
        const bool last = j + 1 == H;
        const float2 ub_b = last ? make_float2(ub2[0].y, s_ub[fnext][tx]) : ub2[j + 1];
        const float2 vb1_b = last ? make_float2(vb12[0].y, s_vb1[fnext][tx]) : vb12[j + 1];
        const float2 vb2_b = last ? make_float2(vb22[0].y, s_vb2[fnext][tx]) : vb22[j + 1];
        tgv_px_dual2(mb >> (3 * j), mb >> (3 * (j + H)), ub2[j],
                     make_float2(s_ub[f0][txr], s_ub[f1][txr]), ub_b, vb12[j],
                     make_float2(s_vb1[f0][txr], s_vb1[f1][txr]), vb1_b, vb22[j],
                     make_float2(s_vb2[f0][txr], s_vb2[f1][txr]), vb2_b, c2[j], tp, p12[j],
                     p22[j], q112[j], q122[j], q212[j], q222[j], t12[j], t22[j], qx12[j],
                     qx22[j], qy12[j], qy22[j]);
        s_t1[f0][tx] = t12[j].x;   s_t1[f1][tx] = t12[j].y;
        s_t2[f0][tx] = t22[j].x;   s_t2[f1][tx] = t22[j].y;
        s_qx1[f0][tx] = qx12[j].x; s_qx1[f1][tx] = qx12[j].y;
        s_qx2[f0][tx] = qx22[j].x; s_qx2[f1][tx] = qx22[j].y;
        s_qy1[f0][tx] = qy12[j].x; s_qy1[f1][tx] = qy12[j].y;
        s_qy2[f0][tx] = qy22[j].x; s_qy2[f1][tx] = qy22[j].y;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const int f0 = ty * R + j, f1 = f0 + H;
        // above: the previous pair, or for the first pair the thread above's
        // last row (the footprint's top row reads itself) and row H - 1
        const float2 t2_u = j > 0 ? t22[j - 1] : make_float2(s_t2[fprev][tx], t22[H - 1].x);
        const float2 qy1_u = j > 0 ? qy12[j - 1] : make_float2(s_qy1[fprev][tx], qy12[H - 1].x);
        const float2 qy2_u = j > 0 ? qy22[j - 1] : make_float2(s_qy2[fprev][tx], qy22[H - 1].x);
        tgv_px_primal2(t12[j], make_float2(s_t1[f0][txl], s_t1[f1][txl]), t22[j], t2_u,
                       qx12[j], make_float2(s_qx1[f0][txl], s_qx1[f1][txl]), qy12[j], qy1_u,
                       qx22[j], make_float2(s_qx2[f0][txl], s_qx2[f1][txl]), qy22[j], qy2_u,
                       p12[j], p22[j], c2[j], th2, u2[j], ub2[j], v12[j], v22[j], vb12[j],
                       vb22[j]);
        s_ub[f0][tx] = ub2[j].x;   s_ub[f1][tx] = ub2[j].y;
        s_vb1[f0][tx] = vb12[j].x; s_vb1[f1][tx] = vb12[j].y;
        s_vb2[f0][tx] = vb22[j].x; s_vb2[f1][tx] = vb22[j].y;
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      u[j] = u2[j].x;     u[j + H] = u2[j].y;
      ub[j] = ub2[j].x;   ub[j + H] = ub2[j].y;
      v1[j] = v12[j].x;   v1[j + H] = v12[j].y;
      v2[j] = v22[j].x;   v2[j + H] = v22[j].y;
      vb1[j] = vb12[j].x; vb1[j + H] = vb12[j].y;
      vb2[j] = vb22[j].x; vb2[j + H] = vb22[j].y;
      p1[j] = p12[j].x;   p1[j + H] = p12[j].y;
      p2[j] = p22[j].x;   p2[j + H] = p22[j].y;
      q11[j] = q112[j].x; q11[j + H] = q112[j].y;
      q12[j] = q122[j].x; q12[j + H] = q122[j].y;
      q21[j] = q212[j].x; q21[j + H] = q212[j].y;
      q22[j] = q222[j].x; q22[j + H] = q222[j].y;
    }
  } else {
  float t1[R], t2[R], qx1[R], qx2[R], qy1[R], qy2[R];
#pragma unroll 1
  for (int it = 0; it < n_iters; ++it) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const int fb = min(fy + 1, FH - 1);
      const float ub_b = (r + 1 < R) ? ub[r + 1] : s_ub[fb][tx];
      const float vb1_b = (r + 1 < R) ? vb1[r + 1] : s_vb1[fb][tx];
      const float vb2_b = (r + 1 < R) ? vb2[r + 1] : s_vb2[fb][tx];
      tgv_px_dual(mb >> (3 * r), ub[r], s_ub[fy][txr], ub_b, vb1[r], s_vb1[fy][txr], vb1_b,
                  vb2[r], s_vb2[fy][txr], vb2_b, c[r], tp, p1[r], p2[r], q11[r], q12[r],
                  q21[r], q22[r], t1[r], t2[r], qx1[r], qx2[r], qy1[r], qy2[r]);
      s_t1[fy][tx] = t1[r];
      s_t2[fy][tx] = t2[r];
      s_qx1[fy][tx] = qx1[r];
      s_qx2[fy][tx] = qx2[r];
      s_qy1[fy][tx] = qy1[r];
      s_qy2[fy][tx] = qy2[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const int fu = max(fy - 1, 0);
      const float t2_u = r > 0 ? t2[r - 1] : s_t2[fu][tx];
      const float qy1_u = r > 0 ? qy1[r - 1] : s_qy1[fu][tx];
      const float qy2_u = r > 0 ? qy2[r - 1] : s_qy2[fu][tx];
      tgv_px_primal(t1[r], s_t1[fy][txl], t2[r], t2_u, qx1[r], s_qx1[fy][txl], qy1[r], qy1_u,
                    qx2[r], s_qx2[fy][txl], qy2[r], qy2_u, p1[r], p2[r], c[r], tp.theta,
                    u[r], ub[r], v1[r], v2[r], vb1[r], vb2[r]);
      s_ub[fy][tx] = ub[r];
      s_vb1[fy][tx] = vb1[r];
      s_vb2[fy][tx] = vb2[r];
    }
    __syncthreads();
  }
  }

  if (!col_in || tx < B || tx >= FW - B) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int fy = ty * R + r;
    if (fy < B || fy >= FH - B || !ok[r]) continue;
    const unsigned k = idx[r];
    const float a[12] = {u[r], ub[r], v1[r], v2[r], vb1[r], vb2[r], p1[r], p2[r],
                         q11[r], q12[r], q21[r], q22[r]};
#pragma unroll
    for (int j = 0; j < 12; ++j) out.s[j][k] = a[j];
  }
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

TgvState primary(const LevelView& L) {
  return TgvState{{L.u, L.ubar, L.v1, L.v2, L.vb1, L.vb2, (float*)L.p1.p, (float*)L.p2.p,
                   L.q11, L.q12, L.q21, L.q22}};
}

TgvState alternate(const LevelView& L) {
  TgvState s;
  for (int j = 0; j < 12; ++j) s.s[j] = L.tgv_alt[j];
  return s;
}

template <int FW, int NY, int R>
cudaError_t launch_blocked_t(const LevelView& L, const TgvState& in, const TgvState& out,
                             const TgvParams& tp, int B, int n, bool chained, cudaStream_t st) {
  const int IW = FW - 2 * B, IH = NY * R - 2 * B;
  if (IW <= 0 || IH <= 0 || n < 0 || n > B) return cudaErrorInvalidValue;
  constexpr size_t smem = 9 * (size_t)FW * NY * R * sizeof(float);
  if constexpr (smem > 48 * 1024) {      // above the default limit: opt in once per device
    static std::atomic<unsigned long long> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(opted.load() & bit)) {
      e = cudaFuncSetAttribute(k_tgv_blocked<FW, NY, R>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      opted.fetch_or(bit);
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((L.W + IW - 1) / IW, (L.H + IH - 1) / IH, 1);
  cfg.blockDim = dim3(FW, NY, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_tgv_blocked<FW, NY, R>, L, in, out, tp, B, n,
                            chained ? 1 : 0);
}

// The 32 x 32 footprint on 256 threads of 4 rows (variant 0), 1024 threads
// of 1 row (1) or 512 threads of 2 rows (2): more threads shorten each
// thread's dependent chain per iteration on the latency-bound levels.  The
// 64 x 32 footprint on 512 threads of 4 rows (3) or 1024 threads of 2 rows
// (4): less halo recomputed per interior pixel on the large levels (72 KB
// of shared memory).
cudaError_t launch_blocked(int variant, const LevelView& L, const TgvState& in,
                           const TgvState& out, const TgvParams& tp, int B, int n, bool chained,
                           cudaStream_t st) {
  switch (variant) {
    case 0: return launch_blocked_t<32, 8, 4>(L, in, out, tp, B, n, chained, st);
    case 1: return launch_blocked_t<32, 32, 1>(L, in, out, tp, B, n, chained, st);
    case 2: return launch_blocked_t<32, 16, 2>(L, in, out, tp, B, n, chained, st);
    case 3: return launch_blocked_t<64, 8, 4>(L, in, out, tp, B, n, chained, st);
    case 4: return launch_blocked_t<64, 16, 2>(L, in, out, tp, B, n, chained, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_tgv_iterations(const LevelView& L, const TgvParams& tp, int B, int variant,
                                  int n, cudaStream_t st) {
  if (B <= 0) {                       // a dual and a primal launch per iteration
    const dim3 g = tgrid(L.W, L.H), b(32, 8);
    for (int k = 0; k < n; ++k) {
      k_tgv_dual<<<g, b, 0, st>>>(L, tp);
      k_tgv_primal<<<g, b, 0, st>>>(L, tp);
    }
    return cudaGetLastError();
  }
  // temporal blocking: at most B iterations per launch, an even number of
  // launches (when n >= 2) so that the state ends in the level's planes
  int nl = (n + B - 1) / B;
  if (nl % 2 == 1 && n >= 2) ++nl;
  const TgvState A = primary(L), Bs = alternate(L);
  for (int k = 0, done = 0; k < nl; ++k) {
    int m = (n - done) / (nl - k);
    if ((n - done) % (nl - k)) ++m;
    cudaError_t e = launch_blocked(variant, L, (k % 2 == 0) ? A : Bs, (k % 2 == 0) ? Bs : A,
                                   tp, B, m, k > 0, st);
    if (e != cudaSuccess) return e;
    done += m;
  }
  if (nl % 2 == 1) {                  // a single launch: copy the state back
    const size_t bytes = (size_t)L.P * L.H * sizeof(float);
    for (int j = 0; j < 12; ++j) {
      cudaError_t e = cudaMemcpyAsync(A.s[j], Bs.s[j], bytes, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
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
