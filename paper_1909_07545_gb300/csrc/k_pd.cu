// k_pd.cu -- primal-dual iterations (Eq. 11, 13) in two schedules.
//
// Per-pixel arithmetic: pd_math.cuh (identical in both schedules).
//
// 1. k_pd -- temporal blocking, for levels too large to stay on chip: one
//    CTA per footprint, the body in pd_tile.cuh (an interior tile plus a halo
//    of B pixels, n <= B iterations per launch).  Six footprints (PDVariant)
//    trade registers per thread (R rows) against resident warps and halo
//    recomputation; the autotuner picks one per level.  ACC instantiations
//    read the accelerated step schedule, one table entry per iteration of
//    the warp.
//
// 2. k_pd_cluster -- the whole level resident in one thread-block cluster
//    (at most 16 CTAs, one tile each, no halo), for the coarse levels.  Each
//    CTA pushes its border values into halo cells of its neighbours' shared
//    memory (remote stores into distributed shared memory), so all reads stay
//    local; two cluster barriers per iteration.  All iterations of a warp run
//    in one launch and the state is updated in place.
//
// grad: forward differences masked by MASK_GX / MASK_GY; div: its exact
// negative adjoint; u is only updated inside the FOV mask.
#include <cooperative_groups.h>

#include "fs_kernels.h"
#include "pd_tile.cuh"

namespace cg = cooperative_groups;

namespace fs {

// The per-warp constants of the iterations (PxConst other than s, tau)
// into L.dinv, L.sd, L.step, L.c0, from the stored sigma, tau, I_u, rho0
// and u_w by the same px_make the other schedules apply (so the same bits).
template <int S>
__global__ void k_pd_consts(LevelView L, float lam, float eps) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= L.W || y >= L.H) return;
  const size_t i = (size_t)y * L.P + x;
  PxRaw raw;
  px_fetch<S>(L, i, true, raw);
  PxConst c;
  px_make(raw, lam, eps, c);
  L.dinv[i] = c.dinv;
  L.sd[i] = c.sd;
  L.step[i] = c.step;
  L.c0[i] = c.c0;
}

cudaError_t launch_pd_consts(const LevelView& L, float lam, float eps, cudaStream_t st) {
  const dim3 blk(32, 8), grd((L.W + 31) / 32, (L.H + 7) / 8);
  switch (L.st) {
    case ST_F16: k_pd_consts<ST_F16><<<grd, blk, 0, st>>>(L, lam, eps); break;
    case ST_BF16: k_pd_consts<ST_BF16><<<grd, blk, 0, st>>>(L, lam, eps); break;
    default: k_pd_consts<ST_F32><<<grd, blk, 0, st>>>(L, lam, eps); break;
  }
  return cudaGetLastError();
}

template <int FW, int NY, int R, int S, bool ACC>
__global__ void __launch_bounds__(FW * NY, FW * NY >= 512 ? 1 : 2)
k_pd(LevelView L, PDState in, PDState out, PDParams pp, int B, int n_iters, int chained) {
  constexpr int FH = NY * R;
  __shared__ float s_ub[FH][FW];
  __shared__ float s_t1[FH][FW];
  __shared__ float s_t2[NY][FW];
  pd_tile<FW, NY, R, S, ACC, false, true>(L, in, out, pp, B, n_iters, (int)blockIdx.x,
                                          (int)blockIdx.y, (int)threadIdx.x, (int)threadIdx.y,
                                          s_ub, s_t1, s_t2, chained != 0);
}

template <int TW, int NY, int R, int S>
__global__ void __launch_bounds__(TW * NY, 1)
k_pd_cluster(LevelView L, PDParams pp, int n_iters) {
  constexpr int TH = NY * R;
  constexpr int SU = TW + 1;          // s_ub: TH+1 rows of TW+1 (right column, bottom row = halo)
  constexpr int S1 = TW + 1;          // s_t1: TH rows of TW+1 (column 0 = left halo)
  __shared__ float s_ub[(TH + 1) * SU];
  __shared__ float s_t1[TH * S1];
  __shared__ float s_t2[(TH + 1) * TW];   // row 0 = top halo

  cg::cluster_group cl = cg::this_cluster();
  const dim3 cb = cl.block_index();
  const dim3 cd = cl.dim_blocks();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ox = (int)cb.x * TW, oy = (int)cb.y * TH;
  const int gx = ox + tx;
  const bool col_in = gx < L.W;
  const float theta = pp.theta;

  // Neighbouring tiles' shared memory: borders are pushed into their halo
  // cells with remote stores, so every read below is a local one.
  const unsigned cw = cd.x;
  float* to_left_ub = cb.x > 0 ? cl.map_shared_rank(s_ub, (cb.x - 1) + cb.y * cw) : nullptr;
  float* to_up_ub = cb.y > 0 ? cl.map_shared_rank(s_ub, cb.x + (cb.y - 1) * cw) : nullptr;
  float* to_right_t1 = cb.x + 1 < cd.x ? cl.map_shared_rank(s_t1, (cb.x + 1) + cb.y * cw) : nullptr;
  float* to_down_t2 = cb.y + 1 < cd.y ? cl.map_shared_rank(s_t2, cb.x + (cb.y + 1) * cw) : nullptr;

  // halo cells with no neighbour stay 0 (the masks zero their terms anyway)
  const int nthr = TW * NY, tid = ty * TW + tx;
  for (int k = tid; k < TH + 1; k += nthr) s_ub[k * SU + TW] = 0.f;
  for (int k = tid; k < TW; k += nthr) { s_ub[TH * SU + k] = 0.f; s_t2[k] = 0.f; }
  for (int k = tid; k < TH; k += nthr) s_t1[k * S1] = 0.f;
  cl.sync();                                   // zeroing before any neighbour pushes

  float u[R], ub[R], p1[R], p2[R];
  PxConst c[R];
  unsigned mb = 0;
  // clamped addresses and unconditional loads, as in k_pd
  const int gxc = min(gx, L.W - 1);
  unsigned idx[R];            // < 2^31: levels are at most 32768 x 32768
  bool ok[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gy = oy + ty * R + r;
    ok[r] = col_in && gy < L.H;
    idx[r] = (unsigned)(min(gy, L.H - 1) * L.P + gxc);
  }
  {
    PxRaw raw[R];
    unsigned char m8[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float a = L.u[idx[r]], b = L.ubar[idx[r]];
      const float q1 = sld<S>(L.p1, idx[r]), q2 = sld<S>(L.p2, idx[r]);
      u[r] = ok[r] ? a : 0.f;
      ub[r] = ok[r] ? b : 0.f;
      p1[r] = ok[r] ? q1 : 0.f;
      p2[r] = ok[r] ? q2 : 0.f;
      px_fetch<S>(L, idx[r], ok[r], raw[r]);
      m8[r] = ok[r] ? L.mask[idx[r]] : 0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      px_make(raw[r], pp.lam, pp.eps, c[r]);
      mb |= (unsigned)m8[r] << (3 * r);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int fy = ty * R + r;
    s_ub[fy * SU + tx] = ub[r];
    if (tx == 0 && to_left_ub) to_left_ub[fy * SU + TW] = ub[r];
    if (fy == 0 && to_up_ub) to_up_ub[TH * SU + tx] = ub[r];
  }
  cl.sync();

#pragma unroll 1
  for (int it = 0; it < n_iters; ++it) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const float right = s_ub[fy * SU + tx + 1];
      const float below = (r + 1 < R) ? ub[r + 1] : s_ub[(fy + 1) * SU + tx];
      float t1, t2;
      px_dual(mb >> (3 * r), ub[r], right, below, c[r], p1[r], p2[r], t1, t2);
      s_t1[fy * S1 + tx + 1] = t1;
      s_t2[(fy + 1) * TW + tx] = t2;
      if (tx == TW - 1 && to_right_t1) to_right_t1[fy * S1] = t1;
      if (fy == TH - 1 && to_down_t2) to_down_t2[tx] = t2;
    }
    cl.sync();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int fy = ty * R + r;
      const float dv = px_div(s_t1[fy * S1 + tx + 1], s_t1[fy * S1 + tx],
                              s_t2[(fy + 1) * TW + tx], s_t2[fy * TW + tx]);
      const float un = px_primal(u[r], dv, c[r]);
      ub[r] = px_relax(un, u[r], theta);
      u[r] = un;
      s_ub[fy * SU + tx] = ub[r];
      if (tx == 0 && to_left_ub) to_left_ub[fy * SU + TW] = ub[r];
      if (fy == 0 && to_up_ub) to_up_ub[TH * SU + tx] = ub[r];
    }
    cl.sync();
  }

  if (!col_in) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gy = oy + ty * R + r;
    if (gy >= L.H) continue;
    const size_t i = (size_t)gy * L.P + gx;
    L.u[i] = u[r];
    L.ubar[i] = ub[r];
    sst<S>(L.p1, i, p1[r]);
    sst<S>(L.p2, i, p2[r]);
  }
}

template <int FW, int NY, int R, int S, bool ACC = false>
static cudaError_t launch_pd_t(const LevelView& L, const PDState& in, const PDState& out,
                               const PDParams& pp, int B, int n, bool chained,
                               cudaStream_t st) {
  const int IW = FW - 2 * B, IH = NY * R - 2 * B;
  if (IW <= 0 || IH <= 0 || n < 0 || n > B) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((L.W + IW - 1) / IW, (L.H + IH - 1) / IH, 1);
  cfg.blockDim = dim3(FW, NY, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_pd<FW, NY, R, S, ACC>, L, in, out, pp, B, n, chained ? 1 : 0);
}

template <int S>
static cudaError_t launch_pd_s(int variant, const LevelView& L, const PDState& in,
                               const PDState& out, const PDParams& pp, int B, int n,
                               cudaStream_t st, bool chained) {
  switch (variant) {
    case PD_TILE_64: return launch_pd_t<64, 8, 8, S>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_32: return launch_pd_t<32, 8, 4, S>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_64x32: return launch_pd_t<64, 4, 8, S>(L, in, out, pp, B, n, chained, st);
    // the 64 x 64 footprint with 1024 threads of 4 rows (64 registers):
    // twice the resident warps of 512 threads of 8 rows
    case PD_TILE_64_T1024: return launch_pd_t<64, 16, 4, S>(L, in, out, pp, B, n, chained, st);
    // small levels: the 32 x 32 footprint spread over more threads, which
    // shortens each thread's dependent chain per iteration (the small levels
    // are latency-bound, not issue-bound)
    case PD_TILE_32_T1024: return launch_pd_t<32, 32, 1, S>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_32_T512: return launch_pd_t<32, 16, 2, S>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_64x48_T768: return launch_pd_t<64, 12, 4, S>(L, in, out, pp, B, n, chained, st);
    default: return cudaErrorInvalidValue;
  }
}

// The accelerated schedule (FP32 storage only) on each footprint.
static cudaError_t launch_pd_acc(int variant, const LevelView& L, const PDState& in,
                                 const PDState& out, const PDParams& pp, int B, int n,
                                 cudaStream_t st, bool chained) {
  if (L.st != ST_F32) return cudaErrorInvalidValue;
  switch (variant) {
    case PD_TILE_64: return launch_pd_t<64, 8, 8, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_32: return launch_pd_t<32, 8, 4, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_64x32: return launch_pd_t<64, 4, 8, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_64_T1024: return launch_pd_t<64, 16, 4, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_32_T1024: return launch_pd_t<32, 32, 1, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_32_T512: return launch_pd_t<32, 16, 2, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    case PD_TILE_64x48_T768: return launch_pd_t<64, 12, 4, ST_F32, true>(L, in, out, pp, B, n, chained, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pd(int variant, const LevelView& L, const PDState& in, const PDState& out,
                      const PDParams& pp, int B, int n, cudaStream_t st, bool chained) {
  if (pp.sched) return launch_pd_acc(variant, L, in, out, pp, B, n, st, chained);
  switch (L.st) {
    case ST_F16: return launch_pd_s<ST_F16>(variant, L, in, out, pp, B, n, st, chained);
    case ST_BF16: return launch_pd_s<ST_BF16>(variant, L, in, out, pp, B, n, st, chained);
    default: return launch_pd_s<ST_F32>(variant, L, in, out, pp, B, n, st, chained);
  }
}

// ---------------------------------------------------------------- clusters

template <int TW, int NY, int R>
static bool cluster_dims(int W, int H, unsigned& cx, unsigned& cy) {
  constexpr int TH = NY * R;
  cx = (unsigned)((W + TW - 1) / TW);
  cy = (unsigned)((H + TH - 1) / TH);
  return cx * cy <= 16;
}

template <int TW, int NY, int R>
static cudaLaunchConfig_t cluster_config(unsigned cx, unsigned cy, cudaStream_t st,
                                         cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cx, cy, 1);
  cfg.blockDim = dim3(TW, NY, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cx;
  attr[0].val.clusterDim.y = cy;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// True when a cluster of the tiles covering W x H can be resident (cluster
// sizes above 8 need the non-portable opt-in; the occupancy query says
// whether a GPC has room for it).
template <int TW, int NY, int R, int S>
static bool cluster_fits_s(int W, int H) {
  unsigned cx, cy;
  if (!cluster_dims<TW, NY, R>(W, H, cx, cy)) return false;
  if (cudaFuncSetAttribute(k_pd_cluster<TW, NY, R, S>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<TW, NY, R>(cx, cy, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_pd_cluster<TW, NY, R, S>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

// every storage instantiation must fit (a handle picks one at creation)
template <int TW, int NY, int R>
static bool cluster_fits_t(int W, int H) {
  return cluster_fits_s<TW, NY, R, ST_F32>(W, H) && cluster_fits_s<TW, NY, R, ST_F16>(W, H) &&
         cluster_fits_s<TW, NY, R, ST_BF16>(W, H);
}

template <int TW, int NY, int R, int S>
static cudaError_t launch_cluster_s(const LevelView& L, const PDParams& pp, int n,
                                    cudaStream_t st) {
  unsigned cx, cy;
  if (!cluster_dims<TW, NY, R>(L.W, L.H, cx, cy) || n < 1) return cudaErrorInvalidValue;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config<TW, NY, R>(cx, cy, st, attr);
  return cudaLaunchKernelEx(&cfg, k_pd_cluster<TW, NY, R, S>, L, pp, n);
}

template <int TW, int NY, int R>
static cudaError_t launch_cluster_t(const LevelView& L, const PDParams& pp, int n,
                                    cudaStream_t st) {
  switch (L.st) {
    case ST_F16: return launch_cluster_s<TW, NY, R, ST_F16>(L, pp, n, st);
    case ST_BF16: return launch_cluster_s<TW, NY, R, ST_BF16>(L, pp, n, st);
    default: return launch_cluster_s<TW, NY, R, ST_F32>(L, pp, n, st);
  }
}

int pd_cluster_variant(int W, int H) {
  if (W <= 64 && H <= 64) return PD_CLUSTER_16;
  if (W <= 128 && H <= 128) return PD_CLUSTER_32;
  return -1;
}

bool pd_cluster_fits(int variant, int W, int H) {
  switch (variant) {
    case PD_CLUSTER_16: return cluster_fits_t<16, 4, 4>(W, H);
    case PD_CLUSTER_32: return cluster_fits_t<32, 8, 4>(W, H);
    default: return false;
  }
}

cudaError_t launch_pd_cluster(int variant, const LevelView& L, const PDParams& pp, int n,
                              cudaStream_t st) {
  switch (variant) {
    case PD_CLUSTER_16: return launch_cluster_t<16, 4, 4>(L, pp, n, st);
    case PD_CLUSTER_32: return launch_cluster_t<32, 8, 4>(L, pp, n, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fs
