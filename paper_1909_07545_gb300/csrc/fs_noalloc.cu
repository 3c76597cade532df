// fs_noalloc.cu -- fs_pd_iterate_noalloc: the primal-dual iterations of one
// warp on caller buffers, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host thread with a hard real-time
// budget (an allocation can synchronise the device and stall it), a plug-in
// running inside a host framework that owns the whole device memory pool, or
// a process started with a fixed memory cap.  For them this entry point runs
// the same kernels as the fs_handle path but keeps every intermediate plane
// in one file-scope __device__ array of fixed size, so the call itself
// allocates nothing.  That array is part of the library image: every GPU
// that loads libfs.so holds kNoAllocBytes of it until the process exits.
#include <cstdio>
#include <mutex>

#include "fs.h"
#include "fs_kernels.h"

using namespace fs;

namespace {

constexpr size_t kMaxPixels = FS_NOALLOC_MAX_PIXELS;
// planes: ubar, sx, sy, tau, sig, u_alt, ubar_alt, p1_alt, p2_alt and the
// per-warp constants dinv, sd, step, c0 (float) followed by the mask bits
// (one byte per pixel)
constexpr size_t kFloatPlanes = 13;
constexpr size_t kNoAllocBytes = kMaxPixels * (kFloatPlanes * sizeof(float) + 1);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device addresses of g_noalloc_scratch, one per device, looked up once.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

fs_status scratch_for_current_device(unsigned char** out, char* msg, size_t len) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(msg, len, "cudaGetDevice failed or device id out of range: %s",
             cudaGetErrorString(e));
    return FS_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      snprintf(msg, len, "cudaGetSymbolAddress of the scratch array failed: %s",
               cudaGetErrorString(e));
      return FS_ECUDA;
    }
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return FS_OK;
}

// Mask bits from a caller mask (nonzero = inside the FOV): MASK_IN, and the
// forward-difference bits MASK_GX / MASK_GY where the neighbour is inside too.
__global__ void k_mask_bits(const unsigned char* __restrict__ m, uint8_t* __restrict__ bits,
                            int W, int H) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  size_t i = (size_t)y * W + x;
  uint8_t b = 0;
  if (m[i]) {
    b = MASK_IN;
    if (x + 1 < W && m[i + 1]) b |= MASK_GX;
    if (y + 1 < H && m[i + W]) b |= MASK_GY;
  }
  bits[i] = b;
}

}  // namespace

// Sets the thread's fs_last_error message (fs_api.cu); not exported.
fs_status fs_internal_set_error(fs_status s, const char* msg);

extern "C" fs_status fs_pd_iterate_noalloc(const float* d_I0, const unsigned char* d_mask,
                                           const float* d_Iu, const float* d_rho0,
                                           const float* d_uw, float* d_u, float* d_p, int W,
                                           int H, int iters, const fs_params* prm,
                                           void* cuda_stream) {
  char msg[256];
  if (!d_I0 || !d_mask || !d_Iu || !d_rho0 || !d_uw || !d_u || !d_p)
    return fs_internal_set_error(FS_EINVAL, "fs_pd_iterate_noalloc: null buffer");
  if (W < 2 || H < 2 || iters < 1)
    return fs_internal_set_error(FS_EINVAL, "fs_pd_iterate_noalloc: need W, H >= 2, iters >= 1");
  if ((size_t)W * (size_t)H > kMaxPixels) {
    snprintf(msg, sizeof(msg),
             "fs_pd_iterate_noalloc: %d x %d = %zu pixels exceeds the fixed scratch of %zu "
             "pixels (FS_NOALLOC_MAX_PIXELS); use fs_create/fs_run_stage instead",
             W, H, (size_t)W * H, kMaxPixels);
    return fs_internal_set_error(FS_EINVAL, msg);
  }
  fs_params p;
  if (prm) {
    p = *prm;
  } else {
    fs_default_params(&p);
  }
  if (!(p.lambda > 0) || !(p.huber_eps >= 0) || !(p.theta >= 0 && p.theta <= 1) ||
      p.block_iters < 0 || p.block_iters > 8)
    return fs_internal_set_error(FS_EINVAL, "fs_pd_iterate_noalloc: parameter out of range");
  if (p.accel_gamma != 0.f)      // the schedule table lives on a handle
    return fs_internal_set_error(FS_EINVAL,
                                 "fs_pd_iterate_noalloc: accel_gamma is not supported here");
  // what this entry point computes: Huber-TV iterations on FP32 buffers
  // (p.deriv has no role here: I_u is an input)
  if (p.regularizer != FS_REG_HUBER_TV)
    return fs_internal_set_error(FS_EINVAL,
                                 "fs_pd_iterate_noalloc: only the Huber-TV regulariser is "
                                 "supported here (regularizer must be FS_REG_HUBER_TV)");
  if (p.storage != 0)
    return fs_internal_set_error(FS_EINVAL,
                                 "fs_pd_iterate_noalloc: buffers are FP32 (storage must be 0)");
  unsigned char* base = nullptr;
  fs_status s = scratch_for_current_device(&base, msg, sizeof(msg));
  if (s != FS_OK) return fs_internal_set_error(s, msg);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)W * H;
  float* f = (float*)base;
  LevelView L{};
  L.W = W; L.H = H; L.P = W;
  L.st = ST_F32;
  L.I0.p = const_cast<float*>(d_I0);
  L.Iu.p = const_cast<float*>(d_Iu);
  L.rho0.p = const_cast<float*>(d_rho0);
  L.uw = const_cast<float*>(d_uw);
  L.u = d_u;
  L.p1.p = d_p;
  L.p2.p = d_p + n;
  L.ubar = f + 0 * n;
  L.sx.p = f + 1 * n;
  L.sy.p = f + 2 * n;
  L.tau = f + 3 * n;
  L.sig = f + 4 * n;
  L.u_alt = f + 5 * n;
  L.ubar_alt = f + 6 * n;
  L.p1_alt.p = f + 7 * n;
  L.p2_alt.p = f + 8 * n;
  L.dinv = f + 9 * n;
  L.sd = f + 10 * n;
  L.step = f + 11 * n;
  L.c0 = f + 12 * n;
  uint8_t* bits = (uint8_t*)(f + kFloatPlanes * n);
  L.mask = bits;

  // every scratch plane is written in full below before it is read, so the
  // contents left by an earlier call never reach this one
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  k_mask_bits<<<grd, blk, 0, st>>>(d_mask, bits, W, H);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_tensor(L, p.beta, p.eta, p.precond, st);
  if (e == cudaSuccess) e = launch_pd_consts(L, p.lambda, p.huber_eps, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L.ubar, d_u, n * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "fs_pd_iterate_noalloc: %s", cudaGetErrorString(e));
    return fs_internal_set_error(FS_ECUDA, msg);
  }

  // same launch schedule as the handle path: at most B iterations per
  // launch, an even number of launches so the state ends in the caller's
  // buffers
  int B = p.block_iters <= 0 ? 4 : p.block_iters;
  int nl = (iters + B - 1) / B;
  if (nl % 2 == 1 && iters >= 2) ++nl;
  int variant = (W >= 128 && H >= 128) ? PD_TILE_64 : PD_TILE_32;
  PDParams pp{p.lambda, p.huber_eps, p.theta};
  PDState A{L.u, L.ubar, L.p1, L.p2};
  PDState Bs{L.u_alt, L.ubar_alt, L.p1_alt, L.p2_alt};
  for (int k = 0, done = 0; k < nl; ++k) {
    int m = (iters - done) / (nl - k);
    if ((iters - done) % (nl - k)) ++m;
    e = launch_pd(variant, L, (k % 2 == 0) ? A : Bs, (k % 2 == 0) ? Bs : A, pp, B, m, st);
    if (e != cudaSuccess) break;
    done += m;
  }
  if (e == cudaSuccess && nl % 2 == 1) {
    const size_t bytes = n * sizeof(float);
    e = cudaMemcpyAsync(A.u, Bs.u, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(A.p1.p, Bs.p1.p, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(A.p2.p, Bs.p2.p, bytes, cudaMemcpyDeviceToDevice, st);
  }
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "fs_pd_iterate_noalloc: %s", cudaGetErrorString(e));
    return fs_internal_set_error(FS_ECUDA, msg);
  }
  return FS_OK;
}
