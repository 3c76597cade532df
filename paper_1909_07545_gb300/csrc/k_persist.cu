// k_persist.cu -- the persistent schedule: all levels and warps of a solve,
// or of a batch of solves of uneven sizes, in one launch over a work list
// (the structures and the dependency rule are in fs_kernels.h).
//
// Each CTA (1024 threads, one per SM) claims the next item with an atomic
// counter, waits until the item's dependencies are met, does the item's
// work with the same per-pixel functions the launch-per-stage kernels use
// (level_px.cuh, pd_tile.cuh), and publishes its completion:
//
//   producer: stores -> CTA barrier -> thread 0: fence, st.release done[t]
//   consumer: warp 0: ld.acquire done[n] >= s -> CTA barrier -> loads
//
// Planes written during the launch are read through L2 only (the CG loads
// of fs_device.cuh), so an SM never reads a line its L1 cached earlier.
// Items are claimed in dependency order, so every item an item waits on is
// held by a CTA that is already running: the launch cannot deadlock, also
// when other work shares the GPU.  Every wait is still bounded by wait_ns
// of global time; a wait that runs out sets the status to FS_ETIMEOUT and
// the abort flag, and every CTA returns at its next claim or wait.
#include "fs.h"
#include "fs_kernels.h"
#include "level_px.cuh"
#include "pd_tile.cuh"

namespace fs {

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Warp 0: wait until the item's dependencies are met, one counter per lane,
// all polled at once: lanes 0 .. (2r+1)^2 - 1 the tiles within r = radius
// of the tile, itself included (item s needs their counters >= s; r <= 2,
// so at most 25 lanes), or, for a PRE, lane 0 the coarser level's
// finished-tile count and lane 1 the testing stall.  False when the launch
// was aborted or the wait ran out (lane 0 then sets the status to
// FS_ETIMEOUT and the abort flag).
__device__ bool wait_deps(const PersistJob& J, const PersistPhase& ph, int bx, int by,
                          const unsigned* done, const unsigned* level_done, PersistCtrl* ctrl,
                          unsigned long long wait_ns) {
  const int lane = threadIdx.x & 31;
  const unsigned* c = nullptr;
  unsigned need = 0;
  if (ph.kind == PERSIST_PRE) {
    if (lane == 0 && J.coarse_slot >= 0) {
      c = level_done + J.coarse_slot;
      need = (unsigned)J.coarse_tiles;
    } else if (lane == 1 && J.stall) {
      c = level_done + J.level_slot;        // a count nothing reaches
      need = ~0u;
    }
  } else if (lane < (2 * J.radius + 1) * (2 * J.radius + 1)) {
    const int side = 2 * J.radius + 1;
    const int x = bx + lane % side - J.radius, y = by + lane / side - J.radius;
    if (x >= 0 && x < J.tiles_x && y >= 0 && y < J.tiles_y) {
      c = done + J.done_base + y * J.tiles_x + x;
      need = (unsigned)ph.seq;
    }
  }
  const unsigned long long t0 = global_ns();
  for (;;) {
    const bool ok = c == nullptr || ld_acquire(c) >= need;
    if (__all_sync(0xffffffffu, ok)) return true;
    int stop = 0;
    if (lane == 0) {
      if (ld_acquire(&ctrl->abort)) {
        stop = 1;
      } else if (global_ns() - t0 > wait_ns) {
        atomicCAS(&ctrl->status, 0, (int)FS_ETIMEOUT);
        atomicExch(&ctrl->abort, 1u);
        stop = 1;
      }
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    __nanosleep(32);
  }
}

// The interior pixels of tile (bx, by), visited by all threads.
template <typename F>
__device__ __forceinline__ void for_tile_pixels(const PersistJob& J, int bx, int by, F f) {
  const int x0 = bx * J.IW, y0 = by * J.IH;
  const int w = min(J.IW, J.L.W - x0), h = min(J.IH, J.L.H - y0);
  for (int k = threadIdx.x; k < w * h; k += blockDim.x) f(x0 + k % w, y0 + k / w);
}

// PRE: what the stage kernels TENSOR, zero state or UPSAMPLE, then WARP do at
// these pixels (k_tensor, k_zero_state / k_upsample, k_warp).
template <int S>
__device__ __noinline__ void pre_item(const PersistJob& J, int bx, int by) {
  const LevelView& L = J.L;
  for_tile_pixels(J, bx, by, [&](int x, int y) {
    const size_t i = (size_t)y * L.P + x;
    tensor_px<S>(L, x, y, J.beta, J.eta, J.precond);
    float2 w = make_float2(0.f, 0.f);
    float u = 0.f;
    if (J.top) zero_px<S>(L, i);
    else u = upsample_px<S, true>(J.C, L, x, y, w);
    float Iu = 0.f, rho0 = 0.f;
    float2 g = make_float2(0.f, 0.f);
    if (L.mask[i] & MASK_IN) warp_px<S>(L, x, y, i, w, J.central, Iu, rho0, g);
    sst<S>(L.Iu, i, Iu);
    sst<S>(L.rho0, i, rho0);
    L.g[i] = g;
    L.ubar[i] = u;
    L.uw[i] = u;
  });
}

// CLIP: k_clip, or k_clip_warp when another warp follows.
template <int S>
__device__ __noinline__ void clip_item(const PersistJob& J, const PersistPhase& ph, int bx,
                                       int by) {
  const LevelView& L = J.L;
  for_tile_pixels(J, bx, by, [&](int x, int y) {
    const size_t i = (size_t)y * L.P + x;
    const bool in = L.mask[i] & MASK_IN;
    if (!ph.next_warp) {
      if (!in) return;
      float2 w;
      const float un = clip_px<true>(L, i, J.du_max, w);
      L.u[i] = un;
      L.ubar[i] = un;
      L.uw[i] = un;
      L.w[i] = w;
      return;
    }
    float Iu = 0.f, rho0 = 0.f;
    float2 g = make_float2(0.f, 0.f);
    float u;
    if (in) {
      float2 w;
      u = clip_px<true>(L, i, J.du_max, w);
      L.w[i] = w;
      L.u[i] = u;
      warp_px<S>(L, x, y, i, w, J.central, Iu, rho0, g);
    } else {
      u = ldf<true>(L.u + i);
    }
    sst<S>(L.Iu, i, Iu);
    sst<S>(L.rho0, i, rho0);
    L.g[i] = g;
    L.ubar[i] = u;
    L.uw[i] = u;
  });
}

// PD(w, k): one temporally blocked footprint, state from the buffer set of
// the block's parity to the other (even blocks read the primary set).
template <int S>
__device__ __noinline__ void pd_item(const PersistJob& J, const PersistPhase& ph, int bx, int by,
                                     float* smem) {
  const LevelView& L = J.L;
  const PDState A{L.u, L.ubar, L.p1, L.p2};
  const PDState Bs{L.u_alt, L.ubar_alt, L.p1_alt, L.p2_alt};
  const PDState& in = (ph.block % 2 == 0) ? A : Bs;
  const PDState& out = (ph.block % 2 == 0) ? Bs : A;
  const int t = threadIdx.x;
  if (J.variant == PD_TILE_64_T1024) {
    float(*s)[64] = reinterpret_cast<float(*)[64]>(smem);
    pd_tile<64, 16, 4, S, false, true>(L, in, out, J.pp, J.B, ph.n_iter, bx, by, t % 64, t / 64,
                                       s, s + 64, s + 128, false);
  } else {
    float(*s)[32] = reinterpret_cast<float(*)[32]>(smem);
    pd_tile<32, 32, 1, S, false, true>(L, in, out, J.pp, J.B, ph.n_iter, bx, by, t % 32, t / 32,
                                       s, s + 32, s + 64, false);
  }
}

}  // namespace

template <int S>
__global__ void __launch_bounds__(1024, 1)
k_persist(const PersistJob* __restrict__ jobs, const PersistPhase* __restrict__ phases,
          const int* __restrict__ item_phase, int n_items, PersistCtrl* ctrl,
          unsigned* done, unsigned* level_done, unsigned long long wait_ns) {
  extern __shared__ float smem[];               // three planes of the largest footprint
  __shared__ int s_item, s_ok;
  __shared__ PersistPhase s_ph;
  // The next item is claimed while the current one is worked on, and thread
  // 0 decodes it while the CTA drains (the claim's and the decode's
  // latencies hide behind the work).  A CTA then holds two items, the second
  // not started; the smallest unfinished item is always being worked on, so
  // the launch still makes progress.
  if (threadIdx.x == 0) {
    const int i = (int)atomicAdd(&ctrl->next, 1u);
    s_item = i < n_items ? i : -1;
    if (i < n_items) s_ph = phases[item_phase[i]];
  }
  __syncthreads();
  for (;;) {
    const int i = s_item;
    if (i < 0) return;
    const PersistPhase ph = s_ph;
    const PersistJob& J = jobs[ph.job];
    const int t = i - ph.first;
    const int bx = t % J.tiles_x, by = t / J.tiles_x;
    int nxt = -1;
    if (threadIdx.x == 0) nxt = (int)atomicAdd(&ctrl->next, 1u);
    if (threadIdx.x < 32) {
      const bool ok = wait_deps(J, ph, bx, by, done, level_done, ctrl, wait_ns);
      if (threadIdx.x == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    if (ph.kind == PERSIST_PRE) pre_item<S>(J, bx, by);
    else if (ph.kind == PERSIST_PD) pd_item<S>(J, ph, bx, by, smem);
    else clip_item<S>(J, ph, bx, by);
    // Publish: the barrier joins every thread's stores, thread 0's fence
    // orders them (cumulatively, through the barrier) before the release.
    __syncthreads();
    if (threadIdx.x == 0) {
      const bool more = nxt < n_items;
      PersistPhase nph{};
      if (more) nph = phases[item_phase[nxt]];
      __threadfence();
      st_release(done + J.done_base + t, (unsigned)ph.seq + 1u);
      if (ph.last) atomicAdd(level_done + J.level_slot, 1u);
      s_item = (more && !ld_acquire(&ctrl->abort)) ? nxt : -1;
      s_ph = nph;
    }
    __syncthreads();
  }
}

namespace {

constexpr size_t kPersistSmem = 3 * 64 * 64 * sizeof(float);   // 48 KB, dynamic

// The kernel of a storage type, with its dynamic shared memory allowed.
template <int S>
cudaError_t persist_kernel(void (**k)(const PersistJob*, const PersistPhase*, const int*, int,
                                      PersistCtrl*, unsigned*, unsigned*, unsigned long long)) {
  *k = k_persist<S>;
  return cudaFuncSetAttribute(k_persist<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kPersistSmem);
}

cudaError_t persist_kernel_of(int storage,
                              void (**k)(const PersistJob*, const PersistPhase*, const int*, int,
                                         PersistCtrl*, unsigned*, unsigned*,
                                         unsigned long long)) {
  switch (storage) {
    case ST_F16: return persist_kernel<ST_F16>(k);
    case ST_BF16: return persist_kernel<ST_BF16>(k);
    default: return persist_kernel<ST_F32>(k);
  }
}

}  // namespace

cudaError_t launch_persist(int storage, const PersistJob* jobs, const PersistPhase* phases,
                           const int* item_phase, int n_items, PersistCtrl* ctrl, unsigned* done,
                           unsigned* level_done, unsigned long long wait_ns, int grid,
                           cudaStream_t st) {
  if (n_items <= 0 || grid <= 0) return cudaErrorInvalidValue;
  void (*k)(const PersistJob*, const PersistPhase*, const int*, int, PersistCtrl*, unsigned*,
            unsigned*, unsigned long long) = nullptr;
  cudaError_t e = persist_kernel_of(storage, &k);
  if (e != cudaSuccess) return e;
  k<<<dim3((unsigned)grid), dim3(1024), kPersistSmem, st>>>(jobs, phases, item_phase, n_items,
                                                            ctrl, done, level_done, wait_ns);
  return cudaGetLastError();
}

int persist_max_ctas(int storage) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  void (*k)(const PersistJob*, const PersistPhase*, const int*, int, PersistCtrl*, unsigned*,
            unsigned*, unsigned long long) = nullptr;
  cudaError_t e = persist_kernel_of(storage, &k);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 1024, kPersistSmem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per;
}

}  // namespace fs
