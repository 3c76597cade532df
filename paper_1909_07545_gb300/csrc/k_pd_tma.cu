// k_pd_tma.cu -- primal-dual iterations (Eq. 11, 13) on the large levels
// with every footprint's inputs staged in shared memory by the tensor memory
// accelerator (TMA).  The per-pixel arithmetic and the iteration loop are
// those of k_pd (pd_math.cuh, pd_tile.cuh), so the results are the same bits.
//
// Why: a 64 x 64 footprint of 1024 threads holds all 64K registers of an
// SM, so in k_pd nothing covers the start of a footprint, when every thread
// waits for its 44 loads (11 planes x 4 rows).  Here each CTA stays resident
// and takes footprints blockIdx.x, + gridDim.x, ... in turn; while it
// iterates on one, the TMA copies the next one's planes into shared memory,
// so only the first footprint of a CTA waits on L2.
//
// Geometry.  Footprints of 64 x 64 pixels, 1024 threads of 4 rows (as
// PD_TILE_64_T1024).  A tiled TMA copy must start on a 16-byte boundary, so
// footprints start at column 48 bx - 8 (a multiple of 8 elements: 16 bytes
// of a 2-byte plane, 32 of a 4-byte one) and own the 48 interior columns
// 48 bx .. 48 bx + 47; the 8-column margins allow up to 8 iterations per
// launch.  Rows have no alignment rule and keep the margin B of the blocking
// depth (origin by (64 - 2B) - B).  After n <= B iterations the interior is
// exact (its dependency cone stays inside the footprint), so every footprint
// geometry computes the same values.  The mask (1 byte per pixel, 16-element
// rule) comes as an 80-column box from 48 bx - 16.  Copies that reach
// outside the level are filled with zeros, which are the inputs k_pd gives
// such pixels (no mask bit, all constants and state 0).
//
// Synchronisation.  One mbarrier: the leader thread arms it with the bytes
// of a footprint (arrive.expect_tx) and issues the twelve copies; every
// thread waits on its phase (try_wait.parity) before reading the planes.
// The planes of the next footprint are requested only after a CTA barrier
// that follows every thread's reads of the current one.  Every wait is
// bounded by wait_ns of global time; a wait that runs out sets *status to
// FS_ETIMEOUT and the CTA returns.
#include <algorithm>

#include "fs.h"
#include "fs_kernels.h"
#include "pd_tile.cuh"

namespace fs {

namespace {

constexpr int kFW = 64, kNY = 16, kR = 4, kFH = kNY * kR;   // 64 x 64, 1024 threads
constexpr int kIW = 48, kXM = 8;                             // interior columns, column margin
constexpr int kMaskW = 80, kMaskOff = 16;                    // mask box: 80 columns from 48 bx - 16

// Offsets (bytes) of the staged planes, the exchange planes of pd_iterate
// and the mbarrier in dynamic shared memory; all multiples of 128.
template <int S>
struct TmaLayout {
  static constexpr size_t f32 = (size_t)kFW * kFH * 4;                   // an FP32 plane
  static constexpr size_t sp = (size_t)kFW * kFH * storage_size(S);      // a storage plane
  // FP32: tau and the per-warp constants dinv, sd, step, c0, then u, ubar;
  // storage type: s_x, s_y, p1, p2
  static constexpr size_t tau = 0, dinv = f32, sd = 2 * f32, step = 3 * f32, c0 = 4 * f32;
  static constexpr size_t u = 5 * f32, ub = 6 * f32;
  static constexpr size_t sx = 7 * f32, sy = sx + sp, p1 = sy + sp, p2 = p1 + sp;
  static constexpr size_t mask = p2 + sp;                                // kMaskW x kFH bytes
  static constexpr size_t x_ub = mask + (size_t)kMaskW * kFH;            // kFH x kFW floats
  static constexpr size_t x_t1 = x_ub + f32;                             // kFH x kFW floats
  static constexpr size_t x_t2 = x_t1 + f32;                             // kNY x kFW floats
  static constexpr size_t bar = x_t2 + (size_t)kNY * kFW * 4;
  static constexpr size_t bytes = bar + 128;
  // bytes one footprint's copies deliver (boxes count whole, zero fill included)
  static constexpr unsigned tx = (unsigned)(7 * f32 + 4 * sp + (size_t)kMaskW * kFH);
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  // make the initialised barrier visible to the TMA unit (the async proxy)
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// One 2-D tiled copy of the box at column x, row y of the tensor `map` into
// shared memory at dst, completing on the mbarrier bar.
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// The leader's requests for footprint `tile`: the per-warp constants (and
// the mask), then, when `state`, the primal-dual state of the input set.
template <int S>
__device__ __forceinline__ void request(const PdTmaMaps& m, unsigned char* smem, uint32_t bar,
                                        int tile, int tiles_x, int IH, int B, bool consts,
                                        bool state) {
  using Lay = TmaLayout<S>;
  const int bx = tile % tiles_x, by = tile / tiles_x;
  const int x = bx * kIW - kXM, y = by * IH - B;
  if (consts) {
    tma_load(smem_addr(smem + Lay::tau), &m.tau, x, y, bar);
    tma_load(smem_addr(smem + Lay::dinv), &m.dinv, x, y, bar);
    tma_load(smem_addr(smem + Lay::sd), &m.sd, x, y, bar);
    tma_load(smem_addr(smem + Lay::step), &m.step, x, y, bar);
    tma_load(smem_addr(smem + Lay::c0), &m.c0, x, y, bar);
    tma_load(smem_addr(smem + Lay::sx), &m.sx, x, y, bar);
    tma_load(smem_addr(smem + Lay::sy), &m.sy, x, y, bar);
    tma_load(smem_addr(smem + Lay::mask), &m.mask, bx * kIW - kMaskOff, y, bar);
  }
  if (state) {
    tma_load(smem_addr(smem + Lay::u), &m.u, x, y, bar);
    tma_load(smem_addr(smem + Lay::ub), &m.ubar, x, y, bar);
    tma_load(smem_addr(smem + Lay::p1), &m.p1, x, y, bar);
    tma_load(smem_addr(smem + Lay::p2), &m.p2, x, y, bar);
  }
}

// A staged storage-typed value (FP16 / BF16 converted to float).
template <int S>
__device__ __forceinline__ float sval(const unsigned char* plane, int k) {
  if constexpr (S == ST_F16) return __half2float(reinterpret_cast<const __half*>(plane)[k]);
  else if constexpr (S == ST_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(plane)[k]);
  else return reinterpret_cast<const float*>(plane)[k];
}

}  // namespace

// n_iters (<= B <= 8) iterations on every footprint of the level; the state
// is read (through the copies in `maps`) from one buffer set and written to
// `out`.  chained: a programmatic dependent launch (the first footprint's
// constants are requested before the wait for the preceding launch, its
// state after).  stall: testing aid, the first wait never completes.
template <int S, bool ACC>
__global__ void __launch_bounds__(kFW * kNY, 1)
k_pd_tma(LevelView L, PDState out, PDParams pp, int B, int n_iters, int chained,
         const __grid_constant__ PdTmaMaps maps, int* status, unsigned long long wait_ns,
         int stall) {
  using Lay = TmaLayout<S>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool leader = tx == 0 && ty == 0;
  const int IH = kFH - 2 * B;
  const int tiles_x = (L.W + kIW - 1) / kIW;
  const int ntiles = tiles_x * ((L.H + IH - 1) / IH);
  float(*s_ub)[kFW] = reinterpret_cast<float(*)[kFW]>(smem + Lay::x_ub);
  float(*s_t1)[kFW] = reinterpret_cast<float(*)[kFW]>(smem + Lay::x_t1);
  float(*s_t2)[kFW] = reinterpret_cast<float(*)[kFW]>(smem + Lay::x_t2);
  const uint32_t bar = smem_addr(smem + Lay::bar);

  // the next launch of the chain may be scheduled once every CTA of this one
  // is resident (it waits for this grid's completion before its state)
  if (chained) cudaTriggerProgrammaticLaunchCompletion();
  int tile = blockIdx.x;
  if (leader) {
    mbar_init(bar, 1);
    if (tile < ntiles) {
      mbar_expect_tx(bar, Lay::tx + (stall ? 16u : 0u));
      request<S>(maps, smem, bar, tile, tiles_x, IH, B, true, false);
    }
  }
  if (chained) cudaGridDependencySynchronize();
  if (leader && tile < ntiles) request<S>(maps, smem, bar, tile, tiles_x, IH, B, false, true);
  __syncthreads();

  unsigned parity = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    bool late = false;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
      if (global_ns() - t0 > wait_ns) {
        late = true;
        break;
      }
    }
    if (__syncthreads_or(late)) {
      if (leader) atomicCAS(status, 0, (int)FS_ETIMEOUT);
      return;
    }
    parity ^= 1u;

    // this thread's 4 rows of column tx from the staged planes
    float u[kR], ub[kR], p1[kR], p2[kR];
    PxConst c[kR];
    unsigned mb = 0;
    {
      // (outside the level the copies read zeros: the constants of k_pd's
      // all-zero inputs, except dinv = 0 instead of 1, which only scales a
      // dual that is 0 there and stays 0)
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int k = (ty * kR + r) * kFW + tx;
        auto f32 = [&](size_t plane) { return reinterpret_cast<const float*>(smem + plane)[k]; };
        c[r].tau = f32(Lay::tau);
        c[r].dinv = f32(Lay::dinv);
        c[r].sd = f32(Lay::sd);
        c[r].step = f32(Lay::step);
        c[r].c0 = f32(Lay::c0);
        c[r].sx = sval<S>(smem + Lay::sx, k);
        c[r].sy = sval<S>(smem + Lay::sy, k);
        u[r] = f32(Lay::u);
        ub[r] = f32(Lay::ub);
        p1[r] = sval<S>(smem + Lay::p1, k);
        p2[r] = sval<S>(smem + Lay::p2, k);
        mb |= (unsigned)smem[Lay::mask + (ty * kR + r) * kMaskW + tx + (kMaskOff - kXM)]
              << (3 * r);
      }
      __syncthreads();            // every thread has read the staged planes
      const int next = tile + (int)gridDim.x;
      if (leader && next < ntiles) {
        // order the reads above before the copies that overwrite the planes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, Lay::tx);
        request<S>(maps, smem, bar, next, tiles_x, IH, B, true, true);
      }
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) s_ub[ty * kR + r][tx] = ub[r];
    __syncthreads();

    // every pixel of the footprint in the level with all three mask bits
    // set (pixels outside the level were filled with mask 0)
    float theta = pp.theta;
    if (__syncthreads_and(mb == 07777u))
      pd_iterate_rows<kFW, kNY, kR, ACC, false>(pp, n_iters, tx, ty, mb, c, u, ub, p1, p2,
                                                theta, s_ub, s_t1, s_t2);
    else
      pd_iterate_rows<kFW, kNY, kR, ACC, true>(pp, n_iters, tx, ty, mb, c, u, ub, p1, p2,
                                               theta, s_ub, s_t1, s_t2);

    // the interior back to global memory
    const int bx = tile % tiles_x, by = tile / tiles_x;
    const int gx = bx * kIW - kXM + tx;
    if (tx < kXM || tx >= kXM + kIW || gx >= L.W) continue;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const int fy = ty * kR + r;
      const int gy = by * IH - B + fy;
      if (fy < B || fy >= kFH - B || gy >= L.H) continue;
      const size_t i = (size_t)gy * L.P + gx;
      out.u[i] = u[r];
      out.ubar[i] = ub[r];
      sst<S>(out.p1, i, p1[r]);
      sst<S>(out.p2, i, p2[r]);
    }
  }
}

namespace {

template <int S, bool ACC>
cudaError_t launch_tma_t(const LevelView& L, const PDState& out, const PDParams& pp, int B,
                         int n, bool chained, const PdTmaMaps& maps, int* status,
                         unsigned long long wait_ns, int stall, cudaStream_t st) {
  using Lay = TmaLayout<S>;
  static bool configured = false;
  static int sms = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_pd_tma<S, ACC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Lay::bytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    configured = true;
  }
  const int IH = kFH - 2 * B;
  const int ntiles = ((L.W + kIW - 1) / kIW) * ((L.H + IH - 1) / IH);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::min(ntiles, sms), 1, 1);
  cfg.blockDim = dim3(kFW, kNY, 1);
  cfg.dynamicSmemBytes = Lay::bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_pd_tma<S, ACC>, L, out, pp, B, n, chained ? 1 : 0, maps,
                            status, wait_ns, stall);
}

}  // namespace

size_t pd_tma_smem_bytes(int storage) {
  switch (storage) {
    case ST_F16: return TmaLayout<ST_F16>::bytes;
    case ST_BF16: return TmaLayout<ST_BF16>::bytes;
    default: return TmaLayout<ST_F32>::bytes;
  }
}

cudaError_t launch_pd_tma(const LevelView& L, const PDState& out, const PDParams& pp, int B,
                          int n, bool chained, const PdTmaMaps& maps, int* status,
                          unsigned long long wait_ns, int stall, cudaStream_t st) {
  if (B < 1 || B > kXM || n < 0 || n > B || L.W < 1 || L.H < 1) return cudaErrorInvalidValue;
  if (pp.sched) {
    if (L.st != ST_F32) return cudaErrorInvalidValue;
    return launch_tma_t<ST_F32, true>(L, out, pp, B, n, chained, maps, status, wait_ns, stall, st);
  }
  switch (L.st) {
    case ST_F16:
      return launch_tma_t<ST_F16, false>(L, out, pp, B, n, chained, maps, status, wait_ns, stall,
                                         st);
    case ST_BF16:
      return launch_tma_t<ST_BF16, false>(L, out, pp, B, n, chained, maps, status, wait_ns,
                                          stall, st);
    default:
      return launch_tma_t<ST_F32, false>(L, out, pp, B, n, chained, maps, status, wait_ns, stall,
                                         st);
  }
}

}  // namespace fs
