// fs_api.cu -- the C ABI (include/fs.h, include/fs_stages.h): handle
// lifecycle, FP64 host geometry, and the Algorithm 1 schedule of kernels on
// the handle's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "fs.h"
#include "pd_tgv_math.cuh"
#include "fs_stages.h"
#include "fs_kernels.h"

using namespace fs;

namespace {

thread_local std::string g_err;

fs_status fail(fs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define FS_CUDA(expr)                                                             \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(FS_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));      \
  } while (0)

#define FS_LAUNCH(name, call)                                                     \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(FS_ECUDA, "launch of %s failed: %s", name, cudaGetErrorString(e_)); \
  } while (0)

#define FS_LAUNCHED(name)                                                         \
  do {                                                                            \
    cudaError_t e_ = cudaGetLastError();                                          \
    if (e_ != cudaSuccess)                                                        \
      return fail(FS_ECUDA, "launch of %s failed: %s", name, cudaGetErrorString(e_)); \
  } while (0)

constexpr int kMaxLevels = 8;

struct HostLevel {
  int W = 0, H = 0, P = 0;
  double fx = 0, fy = 0, cx = 0, cy = 0;   // level calibration (camera 0)
  int cluster = -1;                         // whole-level cluster variant, -1 if none
  int tuned = -1;                           // autotuned choice: 0 cluster, 1..8 depth, -1 none
  int tuned_variant = -1;                   // autotuned tile variant, -1: by size
  LevelView v{};
  // tensor maps of the TMA-staged primal-dual footprints, reading buffer
  // set 0 (primary) and set 1 (alternate); tma_ok = false if the driver
  // could not encode them (the TMA choices are then refused)
  PdTmaMaps tma[2];
  bool tma_ok = false;
  // the per-warp constants of the primal-dual iterations may not match the
  // level's sigma, tau, I_u, rho0 and u_w (cleared by the warp-start
  // kernels, which write both; run_pd recomputes them when set)
  bool consts_stale = true;
};

// Denominator of the enhanced unified model, alpha sqrt(beta s^2 + c^2) +
// (1 - alpha) c (the unified model is alpha = xi / (1 + xi), beta = 1 up
// to the scale 1 + xi; both are written out).
double eucm_den(const fs_calib& c, double s, double cs) {
  return c.k[0] * std::sqrt(c.k[1] * s * s + cs * cs) + (1.0 - c.k[0]) * cs;
}

double radial(const fs_calib& c, double th) {
  if (c.model == FS_PINHOLE) return std::tan(th);
  if (c.model == FS_EQUIDISTANT) return th;
  if (c.model == FS_UNIFIED) return std::sin(th) / (std::cos(th) + c.k[0]);
  if (c.model == FS_ENHANCED_UNIFIED) return std::sin(th) / eucm_den(c, std::sin(th), std::cos(th));
  double t2 = th * th;
  return th * (1.0 + t2 * (c.k[0] + t2 * (c.k[1] + t2 * (c.k[2] + t2 * c.k[3]))));
}

DevCam dev_cam(const fs_calib& c, double fx, double fy, double cx, double cy) {
  DevCam d;
  d.model = c.model;
  d.fx = (float)fx; d.fy = (float)fy; d.cx = (float)cx; d.cy = (float)cy;
  d.k1 = (float)c.k[0]; d.k2 = (float)c.k[1]; d.k3 = (float)c.k[2]; d.k4 = (float)c.k[3];
  double tm = c.fov_deg * M_PI / 360.0;
  d.theta_max = (float)tm;
  d.r_max = (float)radial(c, tm);
  return d;
}

// The camera of a level (focal lengths and centre of the level, the lens
// of c) in float-float words for the once-per-pose kernels.
DevCamDF dev_cam_df(const fs_calib& c, double fx, double fy, double cx, double cy) {
  DevCamDF d;
  d.model = c.model;
  d.fx = df_from_double(fx); d.fy = df_from_double(fy);
  d.cx = df_from_double(cx); d.cy = df_from_double(cy);
  d.k1 = df_from_double(c.k[0]); d.k2 = df_from_double(c.k[1]);
  d.k3 = df_from_double(c.k[2]); d.k4 = df_from_double(c.k[3]);
  d.theta_max = df_from_double(c.fov_deg * M_PI / 360.0);
  d.f32 = dev_cam(c, fx, fy, cx, cy);
  return d;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (the library
// links the runtime only); null if the driver does not provide it.  The
// lookup is a function-local static's initialiser, which C++ runs once even
// when several threads create handles at the same time.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// A 2-D tensor map of a W x H plane of es-byte elements with a row pitch of
// P elements, copied in boxes of bw x bh elements; out-of-range elements
// of a box read as zero.
bool encode_plane(CUtensorMap* m, const void* base, int es, int W, int H, int P, int bw,
                  int bh) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const CUtensorMapDataType t = es == 4   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                : es == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                          : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const cuuint64_t dim[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t stride[1] = {(cuuint64_t)P * (cuuint64_t)es};
  const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
  const cuuint32_t step[2] = {1, 1};
  return enc(m, t, 2, const_cast<void*>(base), dim, stride, box, step,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The maps of k_pd_tma for level L (64 x 64 boxes; the mask's 80 x 64).
bool build_tma_maps(HostLevel& L) {
  const LevelView& v = L.v;
  const int es = (int)storage_size(v.st);
  bool ok = true;
  for (int set = 0; set < 2 && ok; ++set) {
    PdTmaMaps& m = L.tma[set];
    auto f32 = [&](CUtensorMap* t, const void* p) { return encode_plane(t, p, 4, v.W, v.H, v.P, 64, 64); };
    auto spl = [&](CUtensorMap* t, const SPlane& p) { return encode_plane(t, p.p, es, v.W, v.H, v.P, 64, 64); };
    ok = spl(&m.sx, v.sx) && spl(&m.sy, v.sy) && f32(&m.tau, v.tau) && f32(&m.dinv, v.dinv) &&
         f32(&m.sd, v.sd) && f32(&m.step, v.step) && f32(&m.c0, v.c0) &&
         encode_plane(&m.mask, v.mask, 1, v.W, v.H, v.P, 80, 64) &&
         f32(&m.u, set == 0 ? v.u : v.u_alt) && f32(&m.ubar, set == 0 ? v.ubar : v.ubar_alt) &&
         spl(&m.p1, set == 0 ? v.p1 : v.p1_alt) && spl(&m.p2, set == 0 ? v.p2 : v.p2_alt);
  }
  L.tma_ok = ok;
  return ok;
}

fs_status check_calib(const fs_calib& c, int which) {
  if (c.model < FS_PINHOLE || c.model > FS_ENHANCED_UNIFIED)
    return fail(FS_EINVAL, "camera %d: unknown model %d", which, c.model);
  if (c.model == FS_UNIFIED && !(c.k[0] >= 0 && std::isfinite(c.k[0])))
    return fail(FS_ECALIB, "camera %d: unified model needs xi >= 0", which);
  if (c.model == FS_ENHANCED_UNIFIED && !(c.k[0] >= 0 && c.k[0] < 1 && c.k[1] > 0 &&
                                          std::isfinite(c.k[1])))
    return fail(FS_ECALIB, "camera %d: enhanced unified model needs 0 <= alpha < 1, beta > 0",
                which);
  if (!(c.fx > 0) || !(c.fy > 0) || !std::isfinite(c.cx) || !std::isfinite(c.cy))
    return fail(FS_ECALIB, "camera %d: focal lengths must be > 0, centre finite", which);
  if (!(c.fov_deg > 0 && c.fov_deg < 360))
    return fail(FS_ECALIB, "camera %d: fov_deg must be in (0, 360)", which);
  if (c.model == FS_PINHOLE && !(c.fov_deg < 180))
    return fail(FS_ECALIB, "camera %d: a pinhole fov must be < 180 degrees", which);
  if (c.model >= FS_KANNALA_BRANDT) {
    // r(theta) must be finite and increase on [0, fov/2] (10^4 samples);
    // for the unified models this also keeps the denominator positive
    double tm = c.fov_deg * M_PI / 360.0, prev = 0.0;
    for (int i = 1; i < 10000; ++i) {
      double r = radial(c, tm * i / 9999.0);
      if (!(r > prev) || !std::isfinite(r))
        return fail(FS_ECALIB, "camera %d: r(theta) not increasing", which);
      prev = r;
    }
  }
  return FS_OK;
}

inline dim3 grid2(int W, int H) { return dim3((W + 31) / 32, (H + 7) / 8); }
const dim3 kBlock2(32, 8);

}  // namespace

// Host-side NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Sets the thread's fs_last_error message for the other translation units.
fs_status fs_internal_set_error(fs_status s, const char* msg) {
  g_err = msg;
  return s;
}

// Every device allocation of the library goes through here.  Host-side fault
// injection for tests: while the environment variable FS_FAULT_ALLOC names
// this allocation's site ("arena", "planes", "stage", "sched", "energy",
// "guard") or is "all", the allocation fails with cudaErrorMemoryAllocation
// without reaching the device.
cudaError_t fs_internal_malloc(void** p, size_t bytes, const char* site) {
  const char* f = std::getenv("FS_FAULT_ALLOC");
  if (f && (std::strcmp(f, "all") == 0 || std::strcmp(f, site) == 0)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

namespace {
struct PersistPlan;   // the persistent schedule's work list (below)
}  // namespace

struct fs_handle {
  fs_calib cam[2];
  fs_pose pose;
  fs_params prm;
  int W = 0, H = 0, L = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  HostLevel lv[kMaxLevels];
  float4* cfield = nullptr;               // calibration field c(x), float-float (x, y hi; x, y lo)
  double tp[3] = {0, 0, 0};
  void* arena = nullptr;
  // staging for fs_solve_host
  float* stage = nullptr;
  // CUDA graph cache of one solve
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[7] = {};
  int gwarps = 0, giters = 0;
  // primal-dual timing: one event pair per (level, warp) of the last solve
  int timing = 0;
  std::vector<cudaEvent_t> ev;          // 2 per (level, warp)
  int ev_warps = 0;                      // warps recorded by the last solve
  int ev_iters = 0;
  int ev_levels = 0;                     // levels it ran (1 for a warm start)
  bool ev_pending = false;
  double t_ms[kMaxLevels] = {};
  long long t_launch[kMaxLevels] = {};
  double t_pxit[kMaxLevels] = {};
  // the finest level's u and w hold the result of the last solve
  bool has_state = false;
  double* eacc = nullptr;                // fs_energy's 3 device accumulators
  // guard-band mode (FS_GUARD_BANDS=1 at creation): a band of 0xFF bytes
  // before every plane and after the last; band offsets (bytes into the
  // arena) on the device, the plane that follows each band on the host
  size_t guard = 0;
  std::vector<unsigned long long> gband;
  std::vector<std::string> gname;
  unsigned long long* gband_dev = nullptr;
  int* gflag = nullptr;
  // the accelerated step schedule (accel_gamma > 0): one float4 per
  // iteration of a warp, for the last iteration count it was built for
  float4* sched = nullptr;
  int sched_cap = 0, sched_iters = 0;
  // the persistent schedule (pd_schedule = FS_SCHED_PERSISTENT): the work
  // list of this handle's cold solves, the bound of every wait in it, and
  // the testing aid that makes one wait run out
  PersistPlan* plan = nullptr;
  unsigned long long wait_ns = 2000000000ull;
  int persist_stall = 0;
  // bumped whenever a launch argument a captured graph holds changes (the
  // schedule, the wait bound, the stall aid): batches key their graphs on it
  unsigned sched_gen = 0;
  // set to FS_ETIMEOUT by a TMA-staged primal-dual launch whose copy wait
  // ran out (in the arena; read and cleared by fs_check_waits)
  int* pd_status = nullptr;
};

namespace fs {

// One block per guard band: the lowest band index whose bytes are not all
// 0xFF goes to *first_bad (left at INT_MAX when every band is intact).
__global__ void k_guard_check(const uint32_t* __restrict__ base,
                              const unsigned long long* __restrict__ band, int n_band,
                              size_t words, int* first_bad) {
  const int b = blockIdx.x;
  if (b >= n_band) return;
  const uint32_t* p = base + band[b] / 4;
  bool bad = false;
  for (size_t i = threadIdx.x; i < words; i += blockDim.x) bad |= p[i] != 0xFFFFFFFFu;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicMin(first_bad, b);
}

}  // namespace fs

namespace {

fs_status upload_masks(fs_handle* h, std::vector<uint8_t>& host) {
  const fs_calib& c = h->cam[0];
  double rmax = radial(c, c.fov_deg * M_PI / 360.0);
  for (int l = 0; l < h->L; ++l) {
    HostLevel& L = h->lv[l];
    host.assign((size_t)L.P * L.H, 0);
    auto inside = [&](int x, int y) {
      double mx = (x - L.cx) / L.fx, my = (y - L.cy) / L.fy;
      return std::hypot(mx, my) <= rmax;
    };
    for (int y = 0; y < L.H; ++y)
      for (int x = 0; x < L.W; ++x) {
        bool m = inside(x, y);
        uint8_t b = m ? MASK_IN : 0;
        if (m && x + 1 < L.W && inside(x + 1, y)) b |= MASK_GX;
        if (m && y + 1 < L.H && inside(x, y + 1)) b |= MASK_GY;
        host[(size_t)y * L.P + x] = b;
      }
    FS_CUDA(cudaMemcpy((void*)L.v.mask, host.data(), host.size(), cudaMemcpyHostToDevice));
  }
  return FS_OK;
}

// gamma' of level l (k_trajectory) with the level's camera and the unit
// direction of t' as float-float words.
fs_status launch_trajectory(fs_handle* h, int l, cudaStream_t st) {
  HostLevel& L = h->lv[l];
  double n = std::sqrt(h->tp[0] * h->tp[0] + h->tp[1] * h->tp[1] + h->tp[2] * h->tp[2]);
  k_trajectory<<<grid2(L.W, L.H), kBlock2, 0, st>>>(
      dev_cam_df(h->cam[0], L.fx, L.fy, L.cx, L.cy), df_from_double(h->tp[0] / n),
      df_from_double(h->tp[1] / n), df_from_double(h->tp[2] / n), L.v);
  FS_LAUNCHED("k_trajectory");
  return FS_OK;
}

// The per-pose fields on the handle's stream: the calibration field of the
// pre-rotation (Sec. IV-A) and every level's trajectory field (Sec. III-B).
// t' = R^T t and its direction are FP64 on the host; both kernels compute in
// float-float and store floats.
fs_status build_fields(fs_handle* h) {
  const double* R = h->pose.R;
  const double* t = h->pose.t;
  for (int i = 0; i < 3; ++i) h->tp[i] = R[0 + i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2];
  double n = std::sqrt(h->tp[0] * h->tp[0] + h->tp[1] * h->tp[1] + h->tp[2] * h->tp[2]);
  if (!(n > 0) || !std::isfinite(n))
    return fail(FS_EINVAL, "pose: translation must be non-zero and finite");
  HostLevel& L0 = h->lv[0];
  bool identity = memcmp(&h->cam[0], &h->cam[1], sizeof(fs_calib)) == 0;
  for (int i = 0; i < 9 && identity; ++i) identity = R[i] == ((i % 4 == 0) ? 1.0 : 0.0);
  if (identity) {       // the same lens, no rotation: c(x) = pi_0(pi_0^-1(x)) - x = 0
    FS_CUDA(cudaMemsetAsync(h->cfield, 0, (size_t)L0.P * L0.H * sizeof(float4), h->stream));
  } else {
    RotDF Rd;
    for (int i = 0; i < 9; ++i) Rd.r[i] = df_from_double(R[i]);
    k_calib_field<<<grid2(L0.W, L0.H), kBlock2, 0, h->stream>>>(
        dev_cam_df(h->cam[0], L0.fx, L0.fy, L0.cx, L0.cy),
        dev_cam_df(h->cam[1], h->cam[1].fx, h->cam[1].fy, h->cam[1].cx, h->cam[1].cy), Rd,
        L0.v.mask, h->cfield, L0.W, L0.H, L0.P);
    FS_LAUNCHED("k_calib_field");
  }
  for (int l = 0; l < h->L; ++l) {
    fs_status s = launch_trajectory(h, l, h->stream);
    if (s != FS_OK) return s;
  }
  return FS_OK;
}

// Iterations fused per k_pd launch (temporal-blocking depth).  0 picks by
// level size: 6 for levels wider than 512 px, where the halo recomputation
// starts to cost more than the saved launches, 8 below (launch-latency
// bound); measured on GB300 with the 1024 x 1024 workload.
int pd_block(const fs_handle* h, int l) {
  int b = h->prm.block_iters;
  if (b <= 0 && h->lv[l].tuned >= 1) return h->lv[l].tuned;
  if (b <= 0) return (h->lv[l].W > 512 || h->lv[l].H > 512) ? 6 : 8;
  return b > 8 ? 8 : b;
}

// A schedule choice of fs_autotune / fs_set_schedule: 0 = cluster (Huber-TV)
// or a launch per step (TGV); 8 v + 1 .. 8 v + 8 = blocking depth 1..8 on
// footprint variant v (PDVariant: 64 x 64 of 512 threads, 32 x 32 of 256,
// 64 x 32, 64 x 64 of 1024, 32 x 32 of 1024, 32 x 32 of 512), so 1..48;
// 49..55 = depth 9..15 on 32 x 32 footprints of 1024 threads (deeper
// blocking for the small levels, whose launches cost more than the extra
// halo: they leave most SMs idle); 56..63 = depth 1..8 on the TMA-staged
// 64 x 64 footprints of 1024 threads (k_pd_tma); 64..71 = depth 1..8 on
// 64 x 48 footprints of 768 threads; TGV: 8 v + 1 .. 8 v + 8 = depth on the
// TGV footprint v, 0..4, so 1..40; -1 = none.
constexpr int kDeepChoices = 7;
constexpr int kFirstTmaChoice = 8 * PD_TILE_COUNT + kDeepChoices + 1;
constexpr int kFirst768Choice = kFirstTmaChoice + 8;
constexpr int kMaxChoice = kFirst768Choice + 7;
constexpr int kMaxTgvChoice = 8 * kTgvVariants;
bool is_tma_choice(int c, bool tgv) { return !tgv && c >= kFirstTmaChoice && c < kFirst768Choice; }
void decode_choice(int c, bool tgv, int& depth, int& variant) {
  if (c <= 0) { depth = c; variant = -1; return; }
  if (!tgv && c >= kFirst768Choice) {
    depth = 1 + c - kFirst768Choice;
    variant = PD_TILE_64x48_T768;
    return;
  }
  if (is_tma_choice(c, tgv)) {
    depth = 1 + c - kFirstTmaChoice;
    variant = PD_TILE_64_TMA;
    return;
  }
  if (!tgv && c > 8 * PD_TILE_COUNT) {
    depth = 8 + (c - 8 * PD_TILE_COUNT);
    variant = PD_TILE_32_T1024;
    return;
  }
  depth = 1 + (c - 1) % 8;
  variant = (c - 1) / 8;
}

// Whether level l runs the whole-level cluster schedule.
bool use_cluster(const fs_handle* h, int l) {
  const HostLevel& L = h->lv[l];
  if (L.cluster < 0 || h->prm.pd_schedule != 0 || h->prm.accel_gamma > 0) return false;
  if (h->prm.block_iters <= 0 && L.tuned >= 1) return false;   // tuner chose blocking
  return true;
}

// Whether a solve of h runs the TMA-staged footprints on some level.
bool uses_tma(const fs_handle* h) {
  if (h->prm.regularizer == FS_REG_TGV || h->prm.block_iters > 0) return false;
  for (int l = 0; l < h->L; ++l)
    if (h->lv[l].tuned >= 1 && h->lv[l].tuned_variant == PD_TILE_64_TMA) return true;
  return false;
}

// Number of k_pd launches for `iters` iterations with at most B per launch:
// ceil(iters / B), raised to an even count (when iters >= 2) so that the
// ping-pong state ends in the primary buffers (a launch may then run 0
// iterations, i.e. only copy its interior across).
int pd_launches(int iters, int B) {
  int n = (iters + B - 1) / B;
  if (n % 2 == 1 && iters >= 2) ++n;
  return n;
}

// The accelerated schedule's table for at least `iters` iterations per
// warp, built in FP64 on the host and stored as FP32 (synchronous; called
// outside any graph capture, before the launches that read it).  The table
// for n iterations is a prefix of the one for more, so it only grows; a
// reallocation moves it, and the handle's cached graph is dropped then
// (batches key their graphs on the table's address).
fs_status ensure_schedule(fs_handle* h, int iters) {
  if (!(h->prm.accel_gamma > 0) || h->sched_iters >= iters) return FS_OK;
  if (iters > h->sched_cap) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->sched) cudaFree(h->sched);
    h->sched = nullptr;
    h->sched_cap = 0;
    if (fs_internal_malloc((void**)&h->sched, (size_t)iters * sizeof(float4), "sched") !=
        cudaSuccess) {
      cudaGetLastError();
      h->sched = nullptr;
      return fail(FS_ENOMEM, "accelerated schedule allocation failed");
    }
    h->sched_cap = iters;
  }
  std::vector<float4> tab((size_t)iters);
  const double t0 = 1.0 / std::sqrt(8.0), g = h->prm.accel_gamma, eps = h->prm.huber_eps;
  double t = t0, s = t0;
  for (int k = 0; k < iters; ++k) {
    const double th = 1.0 / std::sqrt(1.0 + 2.0 * g * t);
    const double dinv = 1.0 / (1.0 + s * eps);
    tab[k] = make_float4((float)(t / t0), (float)dinv, (float)(s * dinv), (float)th);
    t *= th;
    s /= th;
  }
  FS_CUDA(cudaStreamSynchronize(h->stream));
  FS_CUDA(cudaMemcpy(h->sched, tab.data(), tab.size() * sizeof(float4), cudaMemcpyHostToDevice));
  h->sched_iters = iters;
  return FS_OK;
}

fs_status run_pd(fs_handle* h, int l, int iters, cudaStream_t st) {
  HostLevel& L = h->lv[l];
  PDParams pp{h->prm.lambda, h->prm.huber_eps, h->prm.theta};
  if (h->prm.accel_gamma > 0) {
    if (!h->sched || h->sched_iters < iters)
      return fail(FS_EINVAL, "accelerated schedule not built for %d iterations", iters);
    pp.sched = h->sched;
  }
  if (h->prm.regularizer == FS_REG_TGV) {
    TgvParams tp{h->prm.lambda, h->prm.theta, h->prm.alpha0, h->prm.alpha1, h->prm.precond};
    // block_iters when set, else the tuned depth, else 4 (0 = launch per
    // step); the tuned footprint, else the 256-thread one
    int B = h->prm.block_iters > 0 ? h->prm.block_iters : (L.tuned >= 0 ? L.tuned : 4);
    int v = (h->prm.block_iters <= 0 && L.tuned_variant >= 0) ? L.tuned_variant : 0;
    FS_LAUNCH("k_tgv", launch_tgv_iterations(L.v, tp, B, v, iters, st));
    return FS_OK;
  }
  if (use_cluster(h, l)) {
    cudaError_t e = launch_pd_cluster(L.cluster, L.v, pp, iters, st);
    if (e != cudaSuccess)
      return fail(FS_ECUDA, "launch of k_pd_cluster failed: %s", cudaGetErrorString(e));
    return FS_OK;
  }
  int B = pd_block(h, l);
  int variant = L.tuned_variant >= 0 && h->prm.block_iters <= 0
                    ? L.tuned_variant
                    : ((L.W >= 128 && L.H >= 128) ? PD_TILE_64 : PD_TILE_32);
  PDState A{L.v.u, L.v.ubar, L.v.p1, L.v.p2};
  PDState Bs{L.v.u_alt, L.v.ubar_alt, L.v.p1_alt, L.v.p2_alt};
  const bool tma = variant == PD_TILE_64_TMA;
  if (tma && !L.tma_ok) return fail(FS_EINVAL, "level %d: no tensor maps for the TMA footprints", l);
  if (L.consts_stale) {
    FS_LAUNCH("k_pd_consts", launch_pd_consts(L.v, h->prm.lambda, h->prm.huber_eps, st));
    L.consts_stale = false;
  }
  int nl = pd_launches(iters, B);
  for (int k = 0, done = 0; k < nl; ++k) {
    int n = (iters - done) / (nl - k);          // spread the iterations evenly
    if ((iters - done) % (nl - k)) ++n;
    const PDState& in = (k % 2 == 0) ? A : Bs;
    const PDState& out = (k % 2 == 0) ? Bs : A;
    pp.k0 = done;
    cudaError_t e = tma ? launch_pd_tma(L.v, out, pp, B, n, k > 0, L.tma[k % 2], h->pd_status,
                                        h->wait_ns, (h->persist_stall && k == 0) ? 1 : 0, st)
                        : launch_pd(variant, L.v, in, out, pp, B, n, st, k > 0);
    if (e != cudaSuccess)
      return fail(FS_ECUDA, "launch of %s failed: %s", tma ? "k_pd_tma" : "k_pd",
                  cudaGetErrorString(e));
    done += n;
  }
  if (nl % 2 == 1) {   // a single launch: bring the state back to the primary set
    size_t bytes = (size_t)L.P * L.H * sizeof(float);
    size_t sbytes = (size_t)L.P * L.H * storage_size(L.v.st);
    FS_CUDA(cudaMemcpyAsync(A.u, Bs.u, bytes, cudaMemcpyDeviceToDevice, st));
    FS_CUDA(cudaMemcpyAsync(A.ubar, Bs.ubar, bytes, cudaMemcpyDeviceToDevice, st));
    FS_CUDA(cudaMemcpyAsync(A.p1.p, Bs.p1.p, sbytes, cudaMemcpyDeviceToDevice, st));
    FS_CUDA(cudaMemcpyAsync(A.p2.p, Bs.p2.p, sbytes, cudaMemcpyDeviceToDevice, st));
  }
  return FS_OK;
}

fs_status run_stage(fs_handle* h, int l, int stage, int count, cudaStream_t st) {
  HostLevel& L = h->lv[l];
  const int consts = h->prm.regularizer == FS_REG_TGV ? 0 : 1;
  // every stage but the iterations and the warp starts can change sigma,
  // tau, I_u, rho0 or u_w
  if (stage != FS_STAGE_PD && stage != FS_STAGE_WARP && stage != FS_STAGE_CLIP_WARP)
    L.consts_stale = true;
  switch (stage) {
    case FS_STAGE_DOWNSAMPLE:
      if (l + 1 >= h->L) return fail(FS_EINVAL, "downsample: level %d has no coarser level", l);
      FS_LAUNCH("k_downsample", launch_downsample(L.v, h->lv[l + 1].v, st));
      return FS_OK;
    case FS_STAGE_TENSOR:
      FS_LAUNCH("k_tensor", launch_tensor(L.v, h->prm.beta, h->prm.eta, h->prm.precond, st));
      return FS_OK;
    case FS_STAGE_UPSAMPLE:
      if (l + 1 >= h->L) return fail(FS_EINVAL, "upsample: level %d has no coarser level", l);
      FS_LAUNCH("k_upsample", launch_upsample(h->lv[l + 1].v, L.v, st));
      if (h->prm.regularizer == FS_REG_TGV) FS_LAUNCH("k_tgv_reset", launch_tgv_reset(L.v, st));
      return FS_OK;
    case FS_STAGE_WARP:
      FS_LAUNCH("k_warp", launch_warp(L.v, h->prm.deriv == FS_DERIV_CENTRAL, h->prm.lambda,
                                      h->prm.huber_eps, consts, st));
      L.consts_stale = !consts;
      if (h->prm.regularizer == FS_REG_TGV)
        FS_LAUNCH("k_tgv_warp_start", launch_tgv_warp_start(L.v, st));
      return FS_OK;
    case FS_STAGE_PD: {
      if (count < 1) return fail(FS_EINVAL, "pd: count must be >= 1");
      fs_status s = ensure_schedule(h, count);
      return s != FS_OK ? s : run_pd(h, l, count, st);
    }
    case FS_STAGE_CLIP:
      k_clip<<<grid2(L.W, L.H), kBlock2, 0, st>>>(L.v, h->prm.du_max);
      FS_LAUNCHED("k_clip");
      return FS_OK;
    case FS_STAGE_CLIP_WARP:
      FS_LAUNCH("k_clip_warp", launch_clip_warp(L.v, h->prm.du_max,
                                                h->prm.deriv == FS_DERIV_CENTRAL, h->prm.lambda,
                                                h->prm.huber_eps, consts, st));
      L.consts_stale = !consts;
      if (h->prm.regularizer == FS_REG_TGV)
        FS_LAUNCH("k_tgv_warp_start", launch_tgv_warp_start(L.v, st));
      return FS_OK;
    case FS_STAGE_WARM:
      FS_LAUNCH("k_warm_start", launch_warm_start(L.v, h->prm.du_max, st));
      if (h->prm.regularizer == FS_REG_TGV) FS_LAUNCH("k_tgv_reset", launch_tgv_reset(L.v, st));
      return FS_OK;
    case FS_STAGE_TRAJECTORY:
      return launch_trajectory(h, l, st);
    default:
      return fail(FS_EINVAL, "unknown stage %d", stage);
  }
}

// The end of a warp (clip + update, Eq. 8-9) and, when another warp
// follows, its start (warp + linearise) in one fused launch.
fs_status clip_then_warp(fs_handle* h, int l, bool next, cudaStream_t st) {
  return run_stage(h, l, next ? FS_STAGE_CLIP_WARP : FS_STAGE_CLIP, 0, st);
}

fs_status enqueue_depth(fs_handle* h, float* disp, float* depth, cudaStream_t st) {
  HostLevel& L0 = h->lv[0];
  DevCam c = dev_cam(h->cam[0], L0.fx, L0.fy, L0.cx, L0.cy);
  k_depth<<<grid2(L0.W, L0.H), kBlock2, 0, st>>>(L0.v, c, (float)-h->tp[0], (float)-h->tp[1],
                                                 (float)-h->tp[2], disp, depth);
  FS_LAUNCHED("k_depth");
  return FS_OK;
}

// Record a timing event; inside a stream capture it must become an event
// record node of the graph (cudaEventRecordExternal), not a dependency.
cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(st, &cs);
  if (r != cudaSuccess) return r;
  return cudaEventRecordWithFlags(e, st, cs == cudaStreamCaptureStatusActive
                                             ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// The whole method for one pair on stream st (Algorithm 1 in the pyramid).
// finest_wait / finest_done (may be null): a dependency taken before the
// finest level's work starts and an event recorded once it has ended, which a
// batch uses to bound how many pairs occupy their finest level at once.
// cont: warm start from the finest level's own u and w (fs_solve_continue).
fs_status enqueue_solve(fs_handle* h, const float* I0, const float* I1, const float* init,
                        int warps, int iters, float* disp, float* depth, cudaStream_t st,
                        cudaEvent_t finest_wait = nullptr, cudaEvent_t finest_done = nullptr,
                        bool cont = false) {
  NvtxRange range(init || cont ? "fs warm solve" : "fs solve");
  fs_status s;
  HostLevel& L0 = h->lv[0];
  FS_LAUNCH("k_copy_in_s", launch_copy_in_image(I0, L0.v, 0, st));
  FS_LAUNCH("k_prerotate", launch_prerotate(I1, h->cfield, L0.v, st));
  int top = h->L - 1;
  if (init || cont) {   // warm start: the finest level only
    if (finest_wait) FS_CUDA(cudaStreamWaitEvent(st, finest_wait, 0));
    if (cont) {          // from the level's own last u and w
      FS_LAUNCH("k_continue", launch_continue(L0.v, st));
      if (h->prm.regularizer == FS_REG_TGV) FS_LAUNCH("k_tgv_reset", launch_tgv_reset(L0.v, st));
    } else {             // from the given disparity, w rebuilt along gamma'
      k_copy_in<<<grid2(L0.W, L0.H), kBlock2, 0, st>>>(init, L0.v.u, L0.W, L0.H, L0.P);
      FS_LAUNCHED("k_copy_in");
      if ((s = run_stage(h, 0, FS_STAGE_WARM, 0, st)) != FS_OK) return s;
    }
    if ((s = run_stage(h, 0, FS_STAGE_TENSOR, 0, st)) != FS_OK) return s;
    if ((s = run_stage(h, 0, FS_STAGE_WARP, 0, st)) != FS_OK) return s;
    for (int w = 0; w < warps; ++w) {
      if (h->timing) FS_CUDA(record_event(h->ev[2 * w], st));
      if ((s = run_pd(h, 0, iters, st)) != FS_OK) return s;
      if (h->timing) FS_CUDA(record_event(h->ev[2 * w + 1], st));
      if ((s = clip_then_warp(h, 0, w + 1 < warps, st)) != FS_OK) return s;
    }
    if (h->timing) {
      h->ev_warps = warps;
      h->ev_iters = iters;
      h->ev_levels = 1;
      h->ev_pending = true;
    }
    if (finest_done) FS_CUDA(cudaEventRecord(finest_done, st));
    return enqueue_depth(h, disp, depth, st);
  }
  for (int l = 0; l < top; ++l)
    if ((s = run_stage(h, l, FS_STAGE_DOWNSAMPLE, 0, st)) != FS_OK) return s;
  for (int l = top; l >= 0; --l) {
    static const char* kLevelNames[] = {"fs level 0", "fs level 1", "fs level 2",
                                        "fs level 3", "fs level 4", "fs level 5",
                                        "fs level 6", "fs level 7"};
    NvtxRange level_range(kLevelNames[l < 8 ? l : 7]);
    HostLevel& L = h->lv[l];
    if (l == 0 && finest_wait) FS_CUDA(cudaStreamWaitEvent(st, finest_wait, 0));
    if ((s = run_stage(h, l, FS_STAGE_TENSOR, 0, st)) != FS_OK) return s;
    if (l == top) {
      FS_LAUNCH("k_zero_state", launch_zero_state(L.v, st));
      if (h->prm.regularizer == FS_REG_TGV) FS_LAUNCH("k_tgv_reset", launch_tgv_reset(L.v, st));
    } else if ((s = run_stage(h, l, FS_STAGE_UPSAMPLE, 0, st)) != FS_OK) {
      return s;
    }
    if ((s = run_stage(h, l, FS_STAGE_WARP, 0, st)) != FS_OK) return s;
    for (int w = 0; w < warps; ++w) {
      if (h->timing) FS_CUDA(record_event(h->ev[2 * (l * warps + w)], st));
      if ((s = run_pd(h, l, iters, st)) != FS_OK) return s;
      if (h->timing) FS_CUDA(record_event(h->ev[2 * (l * warps + w) + 1], st));
      if ((s = clip_then_warp(h, l, w + 1 < warps, st)) != FS_OK) return s;
    }
  }
  if (h->timing) {
    h->ev_warps = warps;
    h->ev_iters = iters;
    h->ev_levels = h->L;
    h->ev_pending = true;
  }
  if (finest_done) FS_CUDA(cudaEventRecord(finest_done, st));
  return enqueue_depth(h, disp, depth, st);
}

fs_status prepare_timing(fs_handle* h, int warps) {
  size_t need = (size_t)2 * h->L * warps;
  while (h->ev.size() < need) {
    cudaEvent_t e;
    FS_CUDA(cudaEventCreate(&e));
    h->ev.push_back(e);
  }
  return FS_OK;
}

fs_status check_handle(const fs_handle* h) {
  if (!h) return fail(FS_EINVAL, "null handle");
  return FS_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device bytes of one level: the mask byte plane, 11 FP32 planes (tau,
// sigma, u, ubar, u_w, the ping-pong u, ubar and the primal-dual constants
// dinv, sd, step, c0), 10 planes in the storage
// type (I0, I1, s_x, s_y, p1, p2, I_u, rho0 and the ping-pong p1, p2) and 3
// float2 planes (gamma, w, g); every plane starts on a 256-byte boundary.
size_t level_bytes(int P, int H, int storage, int regularizer) {
  size_t plane = align_up((size_t)P * H * sizeof(float), 256);
  size_t splane = align_up((size_t)P * H * storage_size(storage), 256);
  size_t plane8 = align_up((size_t)P * H, 256);
  // v, vbar, q and the alternate set of the 12 TGV state planes
  size_t tgv = regularizer == FS_REG_TGV ? 20 * plane : 0;
  return plane8 + 11 * plane + 10 * splane + 3 * 2 * plane + tgv;
}

// ------------------------------------------------------------------ persistent schedule

// The device work list of one persistent launch (k_persist.cu) over one or
// more handles' cold solves, and what it was built for.
struct PersistPlan {
  void* dev = nullptr;                   // jobs | phases | items | ctrl | done | level_done
  PersistJob* jobs = nullptr;
  PersistPhase* phases = nullptr;
  int* items = nullptr;
  PersistCtrl* ctrl = nullptr;
  unsigned* done = nullptr;
  unsigned* level_done = nullptr;
  size_t zero_bytes = 0;                 // ctrl .. level_done, cleared before every launch
  int n_items = 0, grid = 0, storage = 0;
  unsigned long long wait_ns = 0;
  int* h_status = nullptr;               // pinned copy of ctrl->status after the launch
  std::vector<long long> key;
};

static void persist_free(PersistPlan* P) {
  if (!P) return;
  if (P->dev) cudaFree(P->dev);
  if (P->h_status) cudaFreeHost(P->h_status);
  delete P;
}

// The footprint and halo depth level l of a persistent solve uses: the
// tuned choice's footprint width (64 -> 64 x 64, 32 -> 32 x 32, both of 1024
// threads) and depth, else block_iters, else 64 x 64 at depth 7 on levels of
// at least 128 x 128 and 32 x 32 at depth 8 below.  The depth is capped at
// 2 fw / 5, so that a footprint reaches at most two tiles to each side
// (B <= 2 (fw - 2 B)): a tile's work items then wait on at most 25 tiles.
static void persist_geometry(const fs_handle* h, int l, int& variant, int& B) {
  const HostLevel& L = h->lv[l];
  int fw = (L.W >= 128 && L.H >= 128) ? 64 : 32;
  B = fw == 64 ? 7 : 8;
  if (h->prm.block_iters > 0) {
    B = h->prm.block_iters;
  } else if (L.tuned >= 1 && L.tuned_variant >= 0) {
    B = L.tuned;
    fw = (L.tuned_variant == PD_TILE_32 || L.tuned_variant == PD_TILE_32_T1024 ||
          L.tuned_variant == PD_TILE_32_T512) ? 32 : 64;
  }
  B = std::max(1, std::min(B, 2 * fw / 5));
  variant = fw == 64 ? PD_TILE_64_T1024 : PD_TILE_32_T1024;
}

// Blocks per warp: ceil(iters / B), raised to an even count of at least 2,
// so the state ends in the primary buffer set (a block may run 0 iterations
// and only copy its interior across).
static int persist_blocks(int iters, int B) {
  int n = (iters + B - 1) / B;
  if (n % 2 == 1) ++n;
  return std::max(n, 2);
}

static std::vector<long long> persist_key(const std::vector<fs_handle*>& hs, int warps, int iters) {
  std::vector<long long> key{warps, iters};
  for (fs_handle* h : hs) {
    key.push_back((long long)(uintptr_t)h);
    key.push_back(h->persist_stall);
    key.push_back((long long)h->wait_ns);
    for (int l = 0; l < h->L; ++l) {
      int v, B;
      persist_geometry(h, l, v, B);
      key.push_back(v * 64 + B);
    }
  }
  return key;
}

// Build (or keep) the work list for the cold solves of hs, every one with
// the same storage type.  Items are ordered by their depth along each pair's
// chain of phases (coarsest level first), ties by pair: every item's
// dependencies then come earlier in the claim order.
static fs_status persist_plan(PersistPlan*& P, const std::vector<fs_handle*>& hs, int warps,
                              int iters) {
  std::vector<long long> key = persist_key(hs, warps, iters);
  if (P && P->key == key) return FS_OK;
  persist_free(P);
  P = nullptr;
  std::vector<PersistJob> jobs;
  struct Ph { long long depth; int pair; PersistPhase p; };
  std::vector<Ph> all;
  int n_done = 0, n_slots = 0;
  unsigned long long wait_ns = ~0ull;
  for (size_t pi = 0; pi < hs.size(); ++pi) {
    fs_handle* h = hs[pi];
    wait_ns = std::min(wait_ns, h->wait_ns);
    long long depth = 0;
    int coarse_slot = -1, coarse_tiles = 0;
    for (int l = h->L - 1; l >= 0; --l) {
      HostLevel& HL = h->lv[l];
      PersistJob J;
      memset(&J, 0, sizeof(J));
      J.L = HL.v;
      if (l + 1 < h->L) J.C = h->lv[l + 1].v;
      J.pp = PDParams{h->prm.lambda, h->prm.huber_eps, h->prm.theta};
      J.top = l == h->L - 1;
      persist_geometry(h, l, J.variant, J.B);
      const int fw = J.variant == PD_TILE_64_T1024 ? 64 : 32;
      J.IW = fw - 2 * J.B;
      J.IH = fw - 2 * J.B;
      J.radius = (J.B + J.IW - 1) / J.IW;          // 1 or 2 (persist_geometry's cap)
      J.tiles_x = (HL.W + J.IW - 1) / J.IW;
      J.tiles_y = (HL.H + J.IH - 1) / J.IH;
      const int tiles = J.tiles_x * J.tiles_y;
      J.done_base = n_done;
      n_done += tiles;
      J.level_slot = n_slots++;
      J.coarse_slot = coarse_slot;
      J.coarse_tiles = coarse_tiles;
      J.beta = h->prm.beta;
      J.eta = h->prm.eta;
      J.du_max = h->prm.du_max;
      J.precond = h->prm.precond;
      J.central = h->prm.deriv == FS_DERIV_CENTRAL;
      J.stall = h->persist_stall && l == 0;
      const int job = (int)jobs.size();
      jobs.push_back(J);
      const int nb = persist_blocks(iters, J.B);
      all.push_back({depth++, (int)pi, PersistPhase{0, job, PERSIST_PRE, 0, 0, 0, 0, 0}});
      for (int w = 0; w < warps; ++w) {
        for (int k = 0, done_it = 0; k < nb; ++k) {
          int n = (iters - done_it) / (nb - k);         // spread the iterations evenly
          if ((iters - done_it) % (nb - k)) ++n;
          done_it += n;
          all.push_back({depth++, (int)pi,
                         PersistPhase{0, job, PERSIST_PD, 1 + w * (nb + 1) + k, k, n, 0, 0}});
        }
        all.push_back({depth++, (int)pi,
                       PersistPhase{0, job, PERSIST_CLIP, 1 + w * (nb + 1) + nb, 0, 0,
                                    w + 1 < warps, w + 1 == warps}});
      }
      coarse_slot = J.level_slot;
      coarse_tiles = tiles;
    }
  }
  std::stable_sort(all.begin(), all.end(), [](const Ph& a, const Ph& b) {
    return a.depth != b.depth ? a.depth < b.depth : a.pair < b.pair;
  });
  std::vector<PersistPhase> phases;
  std::vector<int> items;
  phases.reserve(all.size());
  for (Ph& x : all) {
    const PersistJob& J = jobs[x.p.job];
    x.p.first = (int)items.size();
    const int tiles = J.tiles_x * J.tiles_y;
    if ((long long)items.size() + tiles > INT_MAX / 2)
      return fail(FS_EINVAL, "persistent schedule: too many work items");
    items.insert(items.end(), tiles, (int)phases.size());
    phases.push_back(x.p);
  }
  PersistPlan* Q = new (std::nothrow) PersistPlan();
  if (!Q) return fail(FS_ENOMEM, "host allocation failed");
  const size_t bj = align_up(jobs.size() * sizeof(PersistJob), 256);
  const size_t bp = align_up(phases.size() * sizeof(PersistPhase), 256);
  const size_t bi = align_up(items.size() * sizeof(int), 256);
  const size_t bc = align_up(sizeof(PersistCtrl), 256);
  const size_t bd = align_up((size_t)n_done * sizeof(unsigned), 256);
  const size_t bl = align_up((size_t)n_slots * sizeof(unsigned), 256);
  if (fs_internal_malloc(&Q->dev, bj + bp + bi + bc + bd + bl, "persist") != cudaSuccess) {
    cudaGetLastError();
    Q->dev = nullptr;
    persist_free(Q);
    return fail(FS_ENOMEM, "persistent schedule: work-list allocation failed");
  }
  if (cudaHostAlloc((void**)&Q->h_status, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    Q->h_status = nullptr;
    persist_free(Q);
    return fail(FS_ENOMEM, "persistent schedule: status word allocation failed");
  }
  *Q->h_status = 0;
  char* c = (char*)Q->dev;
  Q->jobs = (PersistJob*)c;
  Q->phases = (PersistPhase*)(c + bj);
  Q->items = (int*)(c + bj + bp);
  Q->ctrl = (PersistCtrl*)(c + bj + bp + bi);
  Q->done = (unsigned*)(c + bj + bp + bi + bc);
  Q->level_done = (unsigned*)(c + bj + bp + bi + bc + bd);
  Q->zero_bytes = bc + bd + bl;
  Q->n_items = (int)items.size();
  Q->storage = hs[0]->prm.storage;
  Q->wait_ns = wait_ns;
  const int cap = persist_max_ctas(Q->storage);
  Q->grid = std::max(1, std::min(cap, Q->n_items));
  cudaError_t e = cudaMemcpy(Q->jobs, jobs.data(), jobs.size() * sizeof(PersistJob),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(Q->phases, phases.data(), phases.size() * sizeof(PersistPhase),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(Q->items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess || cap < 1) {
    persist_free(Q);
    return fail(FS_ECUDA, "persistent schedule: %s",
                e != cudaSuccess ? cudaGetErrorString(e) : "kernel does not fit the device");
  }
  Q->key = key;
  P = Q;
  return FS_OK;
}

// The persistent solve of hs on stream st: per pair the input copy,
// pre-rotation and pyramid, then one launch for every level and warp of
// every pair, the status word to the host, and per pair the depth.
static fs_status enqueue_persist(PersistPlan* P, const std::vector<fs_handle*>& hs,
                                 const float* const* I0, const float* const* I1,
                                 float* const* disp, float* const* depth, cudaStream_t st) {
  fs_status s;
  for (size_t i = 0; i < hs.size(); ++i) {
    fs_handle* h = hs[i];
    FS_LAUNCH("k_copy_in_s", launch_copy_in_image(I0[i], h->lv[0].v, 0, st));
    FS_LAUNCH("k_prerotate", launch_prerotate(I1[i], h->cfield, h->lv[0].v, st));
    for (int l = 0; l + 1 < h->L; ++l)
      if ((s = run_stage(h, l, FS_STAGE_DOWNSAMPLE, 0, st)) != FS_OK) return s;
  }
  FS_CUDA(cudaMemsetAsync(P->ctrl, 0, P->zero_bytes, st));
  // its items derive the iterations' constants themselves and do not write
  // the constant planes
  for (fs_handle* h : hs)
    for (int l = 0; l < h->L; ++l) h->lv[l].consts_stale = true;
  FS_LAUNCH("k_persist", launch_persist(P->storage, P->jobs, P->phases, P->items, P->n_items,
                                        P->ctrl, P->done, P->level_done, P->wait_ns, P->grid,
                                        st));
  FS_CUDA(cudaMemcpyAsync(P->h_status, &P->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost,
                          st));
  for (size_t i = 0; i < hs.size(); ++i)
    if ((s = enqueue_depth(hs[i], disp[i], depth[i], st)) != FS_OK) return s;
  return FS_OK;
}

// Whether a cold solve of h runs the persistent schedule.
static bool persist_applies(const fs_handle* h, bool warm) {
  return h->prm.pd_schedule == FS_SCHED_PERSISTENT && !warm &&
         h->prm.regularizer == FS_REG_HUBER_TV && !(h->prm.accel_gamma > 0);
}


}  // namespace

extern "C" {

const char* fs_last_error(void) { return g_err.c_str(); }

fs_status fs_default_params(fs_params* out) {
  if (!out) return fail(FS_EINVAL, "null params");
  memset(out, 0, sizeof(*out));
  out->lambda = 50.f;
  out->huber_eps = 0.01f;
  out->du_max = 0.2f;
  out->beta = 9.f;
  out->eta = 0.85f;
  out->theta = 1.f;
  out->precond = 1;
  out->block_iters = 0;
  out->use_graph = 0;
  out->regularizer = FS_REG_HUBER_TV;
  out->alpha0 = 17.f;
  out->alpha1 = 1.2f;
  out->deriv = FS_DERIV_FORWARD;
  out->accel_gamma = 0.f;
  return FS_OK;
}

}  // extern "C"

// The argument checks of fs_create, without allocating (also used by the
// server to reject a rig when it is registered).
fs_status fs_internal_validate(const fs_calib cam[2], const fs_pose* pose, int W, int H,
                               int levels, const fs_params* prm) {
  if (!cam || !pose) return fail(FS_EINVAL, "null calibration or pose");
  if (levels < 1 || levels > kMaxLevels) return fail(FS_EINVAL, "levels must be in [1, %d]", kMaxLevels);
  if (W < 4 || H < 4 || W > 32768 || H > 32768) return fail(FS_EINVAL, "bad image size %dx%d", W, H);
  fs_status s;
  if ((s = check_calib(cam[0], 0)) != FS_OK) return s;
  if ((s = check_calib(cam[1], 1)) != FS_OK) return s;
  for (int i = 0; i < 12; ++i) {
    double v = i < 9 ? pose->R[i] : pose->t[i - 9];
    if (!std::isfinite(v)) return fail(FS_EINVAL, "pose has a non-finite entry");
  }
  if (prm) {
    const fs_params& p = *prm;
    if (!(p.lambda > 0) || !(p.huber_eps >= 0) || !(p.du_max > 0) || !(p.beta >= 0) ||
        !(p.eta > 0) || !(p.theta >= 0 && p.theta <= 1) || p.block_iters < 0 ||
        p.block_iters > 8 || p.pd_schedule < 0 || p.pd_schedule > FS_SCHED_PERSISTENT ||
        p.storage < 0 ||
        p.storage > 2 || p.regularizer < 0 || p.regularizer > 1 || p.deriv < 0 || p.deriv > 1)
      return fail(FS_EINVAL, "parameter out of range");
    if (p.regularizer == FS_REG_TGV &&
        (!(p.alpha0 >= 0) || !(p.alpha1 > 0) || !std::isfinite(p.alpha0) ||
         !std::isfinite(p.alpha1) || p.storage != 0))
      return fail(FS_EINVAL, "TGV needs alpha0 >= 0, alpha1 > 0 and FP32 storage");
    if (!(p.accel_gamma >= 0) || !std::isfinite(p.accel_gamma))
      return fail(FS_EINVAL, "accel_gamma must be finite and >= 0");
    if (p.accel_gamma > 0 &&
        (p.precond != 0 || p.regularizer != FS_REG_HUBER_TV || p.storage != 0))
      return fail(FS_EINVAL,
                  "accel_gamma > 0 needs precond = 0, the Huber-TV regulariser and FP32 storage");
    if (p.pd_schedule == FS_SCHED_PERSISTENT &&
        (p.regularizer != FS_REG_HUBER_TV || p.accel_gamma > 0))
      return fail(FS_EINVAL,
                  "the persistent schedule needs the Huber-TV regulariser and accel_gamma = 0");
  }
  size_t bytes = 0;
  return fs_state_bytes(W, H, levels, prm, &bytes);   // level sizes
}

extern "C" {

fs_status fs_create(const fs_calib cam[2], const fs_pose* pose, int W, int H, int levels,
                    const fs_params* prm, void* cuda_stream, fs_handle** out) {
  if (!out) return fail(FS_EINVAL, "null output handle pointer");
  *out = nullptr;
  fs_status s;
  if ((s = fs_internal_validate(cam, pose, W, H, levels, prm)) != FS_OK) return s;
  fs_params p;
  if (prm) p = *prm; else fs_default_params(&p);

  fs_handle* h = new (std::nothrow) fs_handle();
  if (!h) return fail(FS_ENOMEM, "host allocation failed");
  h->cam[0] = cam[0];
  h->cam[1] = cam[1];
  h->pose = *pose;
  h->prm = p;
  h->W = W;
  h->H = H;
  h->L = levels;
  h->stream = (cudaStream_t)cuda_stream;

  // level sizes and scaled calibrations (f 2^-l, (c + 0.5) 2^-l - 0.5)
  size_t bytes = 0;
  for (int l = 0; l < levels; ++l) {
    HostLevel& L = h->lv[l];
    L.W = l == 0 ? W : (h->lv[l - 1].W + 1) / 2;
    L.H = l == 0 ? H : (h->lv[l - 1].H + 1) / 2;
    if (L.W < 4 || L.H < 4) {
      const int lw = L.W, lh = L.H;    // L lives in *h
      delete h;
      return fail(FS_EINVAL, "level %d would be %dx%d (< 4x4): too many levels", l, lw, lh);
    }
    L.P = (int)align_up((size_t)L.W, 32);
    double sc = std::ldexp(1.0, -l);
    L.fx = cam[0].fx * sc;
    L.fy = cam[0].fy * sc;
    L.cx = (cam[0].cx + 0.5) * sc - 0.5;
    L.cy = (cam[0].cy + 0.5) * sc - 0.5;
    bytes += level_bytes(L.P, L.H, p.storage, p.regularizer);
    int cv = pd_cluster_variant(L.W, L.H);
    L.cluster = (cv >= 0 && pd_cluster_fits(cv, L.W, L.H)) ? cv : -1;
  }
  size_t cbytes = align_up((size_t)h->lv[0].P * H * sizeof(float4), 256);
  bytes += cbytes + 256;                                  // + the status word
  const char* genv = std::getenv("FS_GUARD_BANDS");
  if (genv && std::atoi(genv) > 0) {
    // two rows of the widest element (float2) of level 0 on each side
    h->guard = align_up(2 * (size_t)h->lv[0].P * sizeof(float2), 256);
    size_t n_planes = 2;                                  // the calibration field, the status word
    for (int l = 0; l < levels; ++l) n_planes += 25 + (p.regularizer == FS_REG_TGV ? 20 : 0);
    bytes += (n_planes + 1) * h->guard;
  }
  cudaError_t e = fs_internal_malloc(&h->arena, bytes, "arena");
  if (e != cudaSuccess) {
    delete h;
    return fail(FS_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  char* cur = (char*)h->arena;
  // the next plane of `size` bytes, after a guard band in guard-band mode
  auto take = [&](size_t size, int l, const char* name) {
    if (h->guard) {
      h->gband.push_back((unsigned long long)(cur - (char*)h->arena));
      h->gname.push_back(std::string("level ") + std::to_string(l) + " " + name);
      cur += h->guard;
    }
    char* at = cur;
    cur += size;
    return at;
  };
  for (int l = 0; l < levels; ++l) {
    HostLevel& L = h->lv[l];
    size_t plane = align_up((size_t)L.P * L.H * sizeof(float), 256);
    size_t splane = align_up((size_t)L.P * L.H * storage_size(p.storage), 256);
    size_t plane8 = align_up((size_t)L.P * L.H, 256);
    LevelView& v = L.v;
    v.W = L.W; v.H = L.H; v.P = L.P;
    v.st = p.storage;
    v.mask = (const uint8_t*)take(plane8, l, "mask");
    float** fl[] = {&v.tau, &v.sig, &v.u, &v.ubar, &v.uw, &v.u_alt, &v.ubar_alt,
                    &v.dinv, &v.sd, &v.step, &v.c0};
    const char* nfl[] = {"tau", "sigma", "u", "ubar", "u_w", "u (ping-pong)", "ubar (ping-pong)",
                         "dinv", "sigma dinv", "L1 step", "c0"};
    for (int j = 0; j < 11; ++j) *fl[j] = (float*)take(plane, l, nfl[j]);
    v.I0lo = v.u_alt;
    v.I1lo = v.ubar_alt;
    SPlane* sp[] = {&v.I0, &v.I1, &v.sx, &v.sy, &v.p1, &v.p2, &v.Iu, &v.rho0, &v.p1_alt,
                    &v.p2_alt};
    const char* nsp[] = {"I0", "I1", "s_x", "s_y", "p1", "p2", "I_u", "rho0",
                         "p1 (ping-pong)", "p2 (ping-pong)"};
    for (int j = 0; j < 10; ++j) sp[j]->p = take(splane, l, nsp[j]);
    float2** f2[] = {&v.gamma, &v.w, &v.g};
    const char* nf2[] = {"gamma'", "w", "g"};
    for (int j = 0; j < 3; ++j) *f2[j] = (float2*)take(2 * plane, l, nf2[j]);
    if (p.regularizer == FS_REG_TGV) {
      float** ft[] = {&v.v1, &v.v2, &v.vb1, &v.vb2, &v.q11, &v.q12, &v.q21, &v.q22};
      const char* nft[] = {"v1", "v2", "vbar1", "vbar2", "q11", "q12", "q21", "q22"};
      for (int j = 0; j < 8; ++j) *ft[j] = (float*)take(plane, l, nft[j]);
      for (int j = 0; j < 12; ++j) v.tgv_alt[j] = (float*)take(plane, l, "TGV ping-pong");
    }
  }
  h->cfield = (float4*)take(cbytes, 0, "calibration field");
  h->pd_status = (int*)take(256, 0, "status word");
  for (int l = 0; l < levels; ++l) build_tma_maps(h->lv[l]);
  if (h->guard) {                                         // the band after the last plane
    h->gband.push_back((unsigned long long)(cur - (char*)h->arena));
    h->gname.push_back("end of the arena");
    cur += h->guard;
  }
  e = cudaMemsetAsync(h->arena, 0, bytes, h->stream);
  for (size_t j = 0; e == cudaSuccess && j < h->gband.size(); ++j)
    e = cudaMemsetAsync((char*)h->arena + h->gband[j], 0xFF, h->guard, h->stream);
  if (e == cudaSuccess && h->guard) {
    e = fs_internal_malloc((void**)&h->gband_dev,
                           h->gband.size() * sizeof(unsigned long long) + sizeof(int), "guard");
    if (e != cudaSuccess) {
      h->gband_dev = nullptr;
      cudaStreamSynchronize(h->stream);
      cudaFree(h->arena);
      delete h;
      return fail(FS_ENOMEM, "guard-band table allocation failed: %s", cudaGetErrorString(e));
    }
    h->gflag = (int*)(h->gband_dev + h->gband.size());
    e = cudaMemcpyAsync(h->gband_dev, h->gband.data(),
                        h->gband.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                        h->stream);
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(h->stream);
    if (h->gband_dev) cudaFree(h->gband_dev);
    cudaFree(h->arena);
    delete h;
    return fail(FS_ECUDA, "arena initialisation failed: %s", cudaGetErrorString(e));
  }
  std::vector<uint8_t> host;
  if ((s = upload_masks(h, host)) != FS_OK || (s = build_fields(h)) != FS_OK) {
    cudaStreamSynchronize(h->stream);
    if (h->gband_dev) cudaFree(h->gband_dev);
    cudaFree(h->arena);
    delete h;
    return s;
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    if (h->gband_dev) cudaFree(h->gband_dev);
    cudaFree(h->arena);
    delete h;
    return fail(FS_ECUDA, "fs_create: %s", cudaGetErrorString(e));
  }
  *out = h;
  return FS_OK;
}

fs_status fs_state_bytes(int W, int H, int levels, const fs_params* prm, size_t* out) {
  if (!out) return fail(FS_EINVAL, "null output");
  if (levels < 1 || levels > kMaxLevels) return fail(FS_EINVAL, "levels must be in [1, %d]", kMaxLevels);
  if (W < 4 || H < 4 || W > 32768 || H > 32768) return fail(FS_EINVAL, "bad image size %dx%d", W, H);
  const int storage = prm ? prm->storage : 0;
  const int reg = prm ? prm->regularizer : 0;
  if (storage < 0 || storage > 2 || reg < 0 || reg > 1)
    return fail(FS_EINVAL, "parameter out of range");
  size_t bytes = 0;
  int lw = W, lh = H;
  for (int l = 0; l < levels; ++l) {
    if (l > 0) { lw = (lw + 1) / 2; lh = (lh + 1) / 2; }
    if (lw < 4 || lh < 4)
      return fail(FS_EINVAL, "level %d would be %dx%d (< 4x4): too many levels", l, lw, lh);
    bytes += level_bytes((int)align_up((size_t)lw, 32), lh, storage, reg);
  }
  bytes += align_up(align_up((size_t)W, 32) * H * sizeof(float4), 256);
  bytes += 256;                                   // the status word
  *out = bytes;
  return FS_OK;
}

fs_status fs_set_pose(fs_handle* h, const fs_pose* pose) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!pose) return fail(FS_EINVAL, "null pose");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(i < 9 ? pose->R[i] : pose->t[i - 9]))
      return fail(FS_EINVAL, "pose has a non-finite entry");
  fs_pose old = h->pose;
  h->pose = *pose;
  if ((s = build_fields(h)) != FS_OK) {
    h->pose = old;
    return s;
  }
  if (h->gexec) {  // the graph captured the old depth constants
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return FS_OK;
}

fs_status fs_level_size(const fs_handle* h, int level, int* W, int* H) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (level < 0 || level >= h->L) return fail(FS_EINVAL, "level %d out of range", level);
  if (W) *W = h->lv[level].W;
  if (H) *H = h->lv[level].H;
  return FS_OK;
}

fs_status fs_trajectory_field(fs_handle* h, int level, float* d_out) {
  return fs_buffer_read(h, level, FS_BUF_GAMMA, d_out);
}

}  // extern "C"

extern "C" fs_status fs_guard_check(fs_handle* h) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!h->guard) return fail(FS_EINVAL, "the handle was created without FS_GUARD_BANDS");
  const int none = INT_MAX;
  int first = none;
  FS_CUDA(cudaMemcpyAsync(h->gflag, &none, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  fs::k_guard_check<<<(unsigned)h->gband.size(), 256, 0, h->stream>>>(
      (const uint32_t*)h->arena, h->gband_dev, (int)h->gband.size(), h->guard / 4, h->gflag);
  FS_CUDA(cudaGetLastError());
  FS_CUDA(cudaMemcpyAsync(&first, h->gflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  FS_CUDA(cudaStreamSynchronize(h->stream));
  if (first != none)
    return fail(FS_ECUDA, "guard band before %s overwritten", h->gname[first].c_str());
  return FS_OK;
}

extern "C" fs_status fs_guard_clobber(fs_handle* h, int band, size_t offset, int* out) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!h->guard) return fail(FS_EINVAL, "the handle was created without FS_GUARD_BANDS");
  if (out) *out = (int)h->gband.size();
  if (band == -1) return FS_OK;
  if (band < 0 || band >= (int)h->gband.size() || offset >= h->guard)
    return fail(FS_EINVAL, "no guard band %d or offset %zu", band, offset);
  FS_CUDA(cudaMemsetAsync((char*)h->arena + h->gband[band] + offset, 0, 1, h->stream));
  FS_CUDA(cudaStreamSynchronize(h->stream));
  return FS_OK;
}

// fs_solve and fs_solve_continue: direct launches, or a CUDA graph captured
// once per set of buffers and replayed.  In guard-band mode every solve ends
// with fs_guard_check (which synchronises the stream).
// A cold solve in the persistent schedule: the work list for (warps, iters)
// and the handle's tuned geometry, the launch sequence (in the handle's
// graph when use_graph is set), then the wait for it and its status.
static fs_status solve_persist(fs_handle* h, const float* d_I0, const float* d_I1, int warps,
                               int iters, float* d_disp, float* d_depth) {
  fs_status s;
  std::vector<fs_handle*> hs{h};
  PersistPlan* before = h->plan;
  if ((s = persist_plan(h->plan, hs, warps, iters)) != FS_OK) return s;
  h->has_state = false;
  if (!h->prm.use_graph) {
    s = enqueue_persist(h->plan, hs, &d_I0, &d_I1, &d_disp, &d_depth, h->stream);
  } else {
    const void* key[7] = {d_I0, d_I1, nullptr, d_disp, d_depth, (const void*)2, h->plan};
    bool hit = h->gexec && before == h->plan && warps == h->gwarps && iters == h->giters &&
               memcmp(key, h->gkey, sizeof(key)) == 0;
    if (!hit) {
      if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
      if (!h->cap_stream) FS_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      FS_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      s = enqueue_persist(h->plan, hs, &d_I0, &d_I1, &d_disp, &d_depth, h->cap_stream);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
      if (s != FS_OK) { if (g) cudaGraphDestroy(g); return s; }
      if (e != cudaSuccess) return fail(FS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&h->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { h->gexec = nullptr; return fail(FS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
      memcpy(h->gkey, key, sizeof(key));
      h->gwarps = warps;
      h->giters = iters;
    }
    FS_CUDA(cudaGraphLaunch(h->gexec, h->stream));
  }
  if (s != FS_OK) return s;
  FS_CUDA(cudaStreamSynchronize(h->stream));
  if (*h->plan->h_status != 0)
    return fail((fs_status)*h->plan->h_status,
                "persistent schedule: a wait ran out after %.3f s (neighbour or coarser level "
                "not finished)", (double)h->plan->wait_ns * 1e-9);
  h->has_state = true;
  return FS_OK;
}

static fs_status solve_launch(fs_handle* h, const float* d_I0, const float* d_I1,
                            const float* d_init, bool cont, int warps, int iters, float* d_disp,
                            float* d_depth) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!d_I0 || !d_I1) return fail(FS_EINVAL, "null input image");
  if (warps < 1 || iters < 1) return fail(FS_EINVAL, "warps and iters must be >= 1");
  if (cont && !h->has_state) return fail(FS_EINVAL, "fs_solve_continue: the handle holds no result");
  if (h->timing && (s = prepare_timing(h, warps)) != FS_OK) return s;
  if ((s = ensure_schedule(h, iters)) != FS_OK) return s;
  if (persist_applies(h, d_init || cont)) return solve_persist(h, d_I0, d_I1, warps, iters,
                                                               d_disp, d_depth);
  if (!h->prm.use_graph) {
    h->has_state = false;
    s = enqueue_solve(h, d_I0, d_I1, d_init, warps, iters, d_disp, d_depth, h->stream, nullptr,
                      nullptr, cont);
    h->has_state = s == FS_OK;
    return s;
  }

  const void* key[7] = {d_I0, d_I1, d_init, d_disp, d_depth, cont ? (const void*)1 : nullptr,
                        nullptr};
  bool hit = h->gexec && warps == h->gwarps && iters == h->giters &&
             memcmp(key, h->gkey, sizeof(key)) == 0;
  if (!hit) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (!h->cap_stream) FS_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    FS_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    s = enqueue_solve(h, d_I0, d_I1, d_init, warps, iters, d_disp, d_depth, h->cap_stream,
                      nullptr, nullptr, cont);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (s != FS_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return fail(FS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->gexec = nullptr; return fail(FS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    memcpy(h->gkey, key, sizeof(key));
    h->gwarps = warps;
    h->giters = iters;
  }
  h->has_state = false;
  FS_CUDA(cudaGraphLaunch(h->gexec, h->stream));
  h->has_state = true;
  if (h->timing) {              // the replay re-records the captured events
    h->ev_warps = warps;
    h->ev_iters = iters;
    h->ev_levels = (d_init || cont) ? 1 : h->L;
    h->ev_pending = true;
  }
  return FS_OK;
}

static fs_status solve_impl(fs_handle* h, const float* d_I0, const float* d_I1,
                            const float* d_init, bool cont, int warps, int iters, float* d_disp,
                            float* d_depth) {
  fs_status s = solve_launch(h, d_I0, d_I1, d_init, cont, warps, iters, d_disp, d_depth);
  if (s == FS_OK && h->guard) s = fs_guard_check(h);
  return s;
}

extern "C" {

fs_status fs_solve(fs_handle* h, const float* d_I0, const float* d_I1, const float* d_init,
                   int warps, int iters, float* d_disp, float* d_depth) {
  return solve_impl(h, d_I0, d_I1, d_init, false, warps, iters, d_disp, d_depth);
}

fs_status fs_solve_continue(fs_handle* h, const float* d_I0, const float* d_I1, int warps,
                            int iters, float* d_disp, float* d_depth) {
  return solve_impl(h, d_I0, d_I1, nullptr, true, warps, iters, d_disp, d_depth);
}

fs_status fs_solve_host(fs_handle* h, const float* h_I0, const float* h_I1, const float* h_init,
                        int warps, int iters, float* h_disp, float* h_depth) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!h_I0 || !h_I1) return fail(FS_EINVAL, "null input image");
  size_t n = (size_t)h->W * h->H;
  if (!h->stage) {
    cudaError_t e = fs_internal_malloc((void**)&h->stage, 5 * n * sizeof(float), "stage");
    if (e != cudaSuccess) { h->stage = nullptr; return fail(FS_ENOMEM, "staging allocation failed"); }
  }
  float *dI0 = h->stage, *dI1 = h->stage + n, *dinit = h->stage + 2 * n;
  float *ddisp = h->stage + 3 * n, *ddepth = h->stage + 4 * n;
  FS_CUDA(cudaMemcpyAsync(dI0, h_I0, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  FS_CUDA(cudaMemcpyAsync(dI1, h_I1, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  if (h_init) FS_CUDA(cudaMemcpyAsync(dinit, h_init, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  if ((s = fs_solve(h, dI0, dI1, h_init ? dinit : nullptr, warps, iters, h_disp ? ddisp : nullptr,
                    h_depth ? ddepth : nullptr)) != FS_OK)
    return s;
  if (h_disp) FS_CUDA(cudaMemcpyAsync(h_disp, ddisp, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  if (h_depth) FS_CUDA(cudaMemcpyAsync(h_depth, ddepth, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  FS_CUDA(cudaStreamSynchronize(h->stream));
  return uses_tma(h) ? fs_check_waits(h) : FS_OK;
}

fs_status fs_destroy(fs_handle* h) {
  if (!h) return FS_OK;
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->stage) cudaFree(h->stage);
  if (h->eacc) cudaFree(h->eacc);
  if (h->gband_dev) cudaFree(h->gband_dev);
  if (h->sched) cudaFree(h->sched);
  persist_free(h->plan);
  if (h->arena) cudaFree(h->arena);
  delete h;
  return FS_OK;
}

// ------------------------------------------------------------------ batches

struct fs_batch {
  std::vector<fs_handle*> h;
  cudaStream_t stream = nullptr;          // user stream the graph is launched on
  cudaStream_t origin = nullptr;          // capture origin
  std::vector<cudaStream_t> lanes;        // one per pair
  std::vector<cudaEvent_t> joins;
  std::vector<cudaEvent_t> finest;        // pair i's finest level has ended
  int finest_limit = 0;                   // pairs on their finest level at once (0: all)
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> key;
  int warps = 0, iters = 0;
  PersistPlan* plan = nullptr;            // the persistent schedule's work list
};

static void batch_free(fs_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  persist_free(b->plan);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  for (cudaEvent_t e : b->finest) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t s : b->lanes) cudaStreamDestroy(s);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

extern "C" fs_status fs_batch_create(fs_handle* const* handles, int n, void* cuda_stream,
                                     fs_batch** out) {
  if (!out) return fail(FS_EINVAL, "null output batch pointer");
  *out = nullptr;
  if (!handles || n < 1) return fail(FS_EINVAL, "a batch needs n >= 1 handles");
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return fail(FS_EINVAL, "batch handle %d is null", i);
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(FS_EINVAL, "handle %d appears twice", i);
  }
  fs_batch* b = new (std::nothrow) fs_batch();
  if (!b) return fail(FS_ENOMEM, "host allocation failed");
  b->h.assign(handles, handles + n);
  b->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    cudaStream_t s;
    cudaEvent_t j;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->lanes.push_back(s);
    e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->joins.push_back(j);
    e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->finest.push_back(j);
  }
  if (e != cudaSuccess) {
    batch_free(b);
    return fail(FS_ECUDA, "fs_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return FS_OK;
}

extern "C" fs_status fs_batch_solve(fs_batch* b, const float* const* d_I0,
                                    const float* const* d_I1, const float* const* d_init,
                                    int warps, int iters, float* const* d_disp,
                                    float* const* d_depth) {
  if (!b) return fail(FS_EINVAL, "null batch");
  if (!d_I0 || !d_I1 || !d_disp || !d_depth) return fail(FS_EINVAL, "null pointer array");
  if (warps < 1 || iters < 1) return fail(FS_EINVAL, "warps and iters must be >= 1");
  const int n = (int)b->h.size();
  std::vector<const void*> key;
  key.reserve(7 * n);
  for (int i = 0; i < n; ++i) {
    if (!d_I0[i] || !d_I1[i]) return fail(FS_EINVAL, "null input image for pair %d", i);
    fs_status s;
    if ((s = ensure_schedule(b->h[i], iters)) != FS_OK) return s;
    key.push_back(b->h[i]->sched);
    key.push_back((const void*)(uintptr_t)b->h[i]->sched_gen);
    key.push_back(d_I0[i]);
    key.push_back(d_I1[i]);
    key.push_back(d_init ? d_init[i] : nullptr);
    key.push_back(d_disp[i]);
    key.push_back(d_depth[i]);
  }
  // every pair cold, in the persistent schedule, one storage type: one
  // persistent launch for the whole batch
  bool persist = true;
  for (int i = 0; i < n; ++i)
    persist = persist && persist_applies(b->h[i], d_init && d_init[i]) &&
              b->h[i]->prm.storage == b->h[0]->prm.storage;
  if (persist) {
    PersistPlan* before = b->plan;
    fs_status s;
    if ((s = persist_plan(b->plan, b->h, warps, iters)) != FS_OK) return s;
    key.push_back(b->plan);
    bool phit = b->gexec && before == b->plan && warps == b->warps && iters == b->iters &&
                key == b->key;
    if (!phit) {
      if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
      FS_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
      s = enqueue_persist(b->plan, b->h, d_I0, d_I1, d_disp, d_depth, b->origin);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->origin, &g);
      if (s != FS_OK) { if (g) cudaGraphDestroy(g); return s; }
      if (e != cudaSuccess) return fail(FS_ECUDA, "batch capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { b->gexec = nullptr; return fail(FS_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e)); }
      b->key = key;
      b->warps = warps;
      b->iters = iters;
    }
    for (int i = 0; i < n; ++i) b->h[i]->has_state = false;
    FS_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    FS_CUDA(cudaStreamSynchronize(b->stream));
    if (*b->plan->h_status != 0)
      return fail((fs_status)*b->plan->h_status,
                  "persistent schedule: a wait ran out after %.3f s (neighbour or coarser level "
                  "not finished)", (double)b->plan->wait_ns * 1e-9);
    for (int i = 0; i < n; ++i) b->h[i]->has_state = true;
    return FS_OK;
  }
  bool hit = b->gexec && warps == b->warps && iters == b->iters && key == b->key;
  if (!hit) {
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    for (int i = 0; i < n; ++i) {
      fs_status s;
      if (b->h[i]->timing && (s = prepare_timing(b->h[i], warps)) != FS_OK) return s;
    }
    FS_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    fs_status s = FS_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    for (int i = 0; i < n && s == FS_OK && e == cudaSuccess; ++i) {
      e = cudaStreamWaitEvent(b->lanes[i], b->fork, 0);
      if (e != cudaSuccess) break;
      // pair i enters its finest level once pair i - k has left its own
      const int k = b->finest_limit;
      cudaEvent_t wait = (k > 0 && i >= k) ? b->finest[i - k] : nullptr;
      cudaEvent_t done = k > 0 ? b->finest[i] : nullptr;
      s = enqueue_solve(b->h[i], d_I0[i], d_I1[i], d_init ? d_init[i] : nullptr, warps, iters,
                        d_disp[i], d_depth[i], b->lanes[i], wait, done);
      if (s != FS_OK) break;
      e = cudaEventRecord(b->joins[i], b->lanes[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
    if (s != FS_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(FS_ECUDA, "batch capture failed: %s",
                  cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->gexec = nullptr; return fail(FS_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e)); }
    b->key = key;
    b->warps = warps;
    b->iters = iters;
  }
  FS_CUDA(cudaGraphLaunch(b->gexec, b->stream));
  for (int i = 0; i < n; ++i) {
    fs_handle* h = b->h[i];
    h->has_state = true;
    if (h->timing) {
      h->ev_warps = warps;
      h->ev_iters = iters;
      h->ev_levels = (d_init && d_init[i]) ? 1 : h->L;
      h->ev_pending = true;
    }
  }
  return FS_OK;
}

extern "C" fs_status fs_batch_set_finest_limit(fs_batch* b, int k) {
  if (!b) return fail(FS_EINVAL, "null batch");
  if (k < 0) return fail(FS_EINVAL, "finest-level limit must be >= 0");
  if (k != b->finest_limit && b->gexec) {   // the cached schedule no longer applies
    cudaStreamSynchronize(b->stream);
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->finest_limit = k;
  return FS_OK;
}

// The common coarse-level schedules fs_batch_autotune tries besides every
// handle's own: blocking depth 8 on 64 x 64 footprints of 1024 threads,
// depth 6 on 64 x 48 of 768, depth 8 on 64 x 64 of 512, depth 5 on 32 x 32
// of 512 -- few, large footprints with little halo, which is what many
// pairs sharing the GPU want, where a pair alone wants short dependent
// chains per launch.
static const int kBatchCoarseChoices[] = {32, 69, 8, 45};

extern "C" fs_status fs_batch_autotune(fs_batch* b, int iters, int* choice) {
  if (!b) return fail(FS_EINVAL, "null batch");
  if (iters < 1) return fail(FS_EINVAL, "iters must be >= 1");
  if (choice) *choice = -1;
  const int n = (int)b->h.size();
  // every handle's own coarse choices (to restore when they win)
  std::vector<std::vector<std::pair<int, int>>> own(n);
  bool any = false;
  for (int i = 0; i < n; ++i) {
    fs_handle* h = b->h[i];
    if (h->prm.regularizer == FS_REG_TGV)
      return fail(FS_EINVAL, "fs_batch_autotune: TGV handles are tuned alone (fs_autotune)");
    fs_status s;
    if ((s = ensure_schedule(h, iters)) != FS_OK) return s;
    for (int l = 2; l < h->L; ++l) {
      own[i].push_back({h->lv[l].tuned, h->lv[l].tuned_variant});
      any = true;
    }
  }
  if (!any) return FS_OK;
  FS_CUDA(cudaStreamSynchronize(b->stream));
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  auto apply = [&](int c) {
    for (int i = 0; i < n; ++i) {
      fs_handle* h = b->h[i];
      if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
      ++h->sched_gen;
      h->has_state = false;                     // the trials overwrite the coarse levels
      for (int l = 2; l < h->L; ++l) {
        HostLevel& L = h->lv[l];
        if (c < 0) {
          L.tuned = own[i][l - 2].first;
          L.tuned_variant = own[i][l - 2].second;
        } else {
          decode_choice(c, false, L.tuned, L.tuned_variant);
        }
      }
    }
  };
  // `iters` iterations on every coarse level of every pair, each pair on its
  // own lane (coarsest first), all pairs at once: one graph per candidate,
  // best of three replays after one
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](float& best) -> fs_status {
    for (int i = 0; i < n; ++i)                 // constants current before the capture
      for (int l = 2; l < b->h[i]->L; ++l) b->h[i]->lv[l].consts_stale = true;
    FS_CUDA(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    fs_status s = FS_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    for (int i = 0; i < n && s == FS_OK && e == cudaSuccess; ++i) {
      e = cudaStreamWaitEvent(b->lanes[i], b->fork, 0);
      for (int l = b->h[i]->L - 1; l >= 2 && s == FS_OK && e == cudaSuccess; --l)
        s = run_pd(b->h[i], l, iters, b->lanes[i]);
      if (s == FS_OK && e == cudaSuccess) e = cudaEventRecord(b->joins[i], b->lanes[i]);
      if (s == FS_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
    if (s != FS_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(FS_ECUDA, "fs_batch_autotune capture: %s",
                  cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(FS_ECUDA, "fs_batch_autotune: %s", cudaGetErrorString(e));
    best = 3.4e38f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, b->stream);
      if (e == cudaSuccess) e = cudaGraphLaunch(x, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    cudaGraphExecDestroy(x);
    if (e != cudaSuccess) return fail(FS_ECUDA, "fs_batch_autotune: %s", cudaGetErrorString(e));
    return FS_OK;
  };
  fs_status st = FS_OK;
  float best_ms = 3.4e38f;
  int best_c = -1;
  const int n_cand = 1 + (int)(sizeof(kBatchCoarseChoices) / sizeof(int));
  for (int k = 0; k < n_cand && st == FS_OK; ++k) {
    const int c = k == 0 ? -1 : kBatchCoarseChoices[k - 1];
    apply(c);
    float ms = 0.f;
    if ((st = time_it(ms)) == FS_OK && ms < best_ms) {
      best_ms = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply(st == FS_OK ? best_c : -1);
  if (st == FS_OK && choice) *choice = best_c;
  return st;
}

extern "C" fs_status fs_batch_destroy(fs_batch* b) {
  if (!b) return FS_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return FS_OK;
}

// ------------------------------------------------------------------ stages

// Where a buffer lives: FP32 planes (kind 0), interleaved float2 (kind 1) or
// planes in the level's storage (kind 2).
struct BufLoc {
  int kind = 0, planes = 1;
  float* f[4] = {nullptr, nullptr, nullptr, nullptr};
  SPlane s[2] = {{nullptr}, {nullptr}};
};

static fs_status buffer_loc(fs_handle* h, int level, int buffer, BufLoc& b) {
  LevelView& v = h->lv[level].v;
  switch (buffer) {
    case FS_BUF_I0: b.kind = 2; b.s[0] = v.I0; break;
    case FS_BUF_I1: b.kind = 2; b.s[0] = v.I1; break;
    case FS_BUF_GAMMA: b.kind = 1; b.planes = 2; b.f[0] = (float*)v.gamma; break;
    case FS_BUF_U: b.f[0] = v.u; break;
    case FS_BUF_UBAR: b.f[0] = v.ubar; break;
    case FS_BUF_UW: b.f[0] = v.uw; break;
    case FS_BUF_P: b.kind = 2; b.planes = 2; b.s[0] = v.p1; b.s[1] = v.p2; break;
    case FS_BUF_W: b.kind = 1; b.planes = 2; b.f[0] = (float*)v.w; break;
    case FS_BUF_IU: b.kind = 2; b.s[0] = v.Iu; break;
    case FS_BUF_RHO0: b.kind = 2; b.s[0] = v.rho0; break;
    case FS_BUF_G: b.kind = 1; b.planes = 2; b.f[0] = (float*)v.g; break;
    case FS_BUF_V: case FS_BUF_VBAR: case FS_BUF_Q:
      if (!v.v1) return fail(FS_EINVAL, "buffer %d exists on TGV handles only", buffer);
      if (buffer == FS_BUF_V) { b.planes = 2; b.f[0] = v.v1; b.f[1] = v.v2; }
      else if (buffer == FS_BUF_VBAR) { b.planes = 2; b.f[0] = v.vb1; b.f[1] = v.vb2; }
      else { b.planes = 4; b.f[0] = v.q11; b.f[1] = v.q12; b.f[2] = v.q21; b.f[3] = v.q22; }
      break;
    default: return fail(FS_EINVAL, "buffer %d cannot be accessed this way", buffer);
  }
  return FS_OK;
}

extern "C" fs_status fs_buffer_read(fs_handle* h, int level, int buffer, float* d_out) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (level < 0 || level >= h->L) return fail(FS_EINVAL, "level %d out of range", level);
  if (!d_out) return fail(FS_EINVAL, "null output");
  HostLevel& L = h->lv[level];
  size_t n = (size_t)L.W * L.H;
  cudaStream_t st = h->stream;
  if (buffer == FS_BUF_MASK) {
    k_mask_to_float<<<grid2(L.W, L.H), kBlock2, 0, st>>>(L.v.mask, d_out, L.W, L.H, L.P);
    FS_LAUNCHED("k_mask_to_float");
    return FS_OK;
  }
  if (buffer == FS_BUF_TENSOR) {
    FS_LAUNCH("k_tensor_abc", launch_tensor_abc(L.v, d_out, st));
    return FS_OK;
  }
  if (buffer == FS_BUF_STEPS) {
    k_pack<<<grid2(L.W, L.H), kBlock2, 0, st>>>(L.v.tau, 1, d_out, L.W, L.H, L.P);
    k_pack<<<grid2(L.W, L.H), kBlock2, 0, st>>>(L.v.sig, 1, d_out + n, L.W, L.H, L.P);
    FS_LAUNCHED("k_pack");
    return FS_OK;
  }
  BufLoc b;
  if ((s = buffer_loc(h, level, buffer, b)) != FS_OK) return s;
  for (int c = 0; c < b.planes; ++c) {
    if (b.kind == 2) {
      FS_LAUNCH("k_pack_s", launch_pack_s(b.s[c], L.v.st, d_out + c * n, L.W, L.H, L.P, st));
      continue;
    }
    k_pack<<<grid2(L.W, L.H), kBlock2, 0, st>>>(b.kind == 1 ? b.f[0] + c : b.f[c],
                                                b.kind == 1 ? 2 : 1, d_out + c * n, L.W, L.H,
                                                L.P);
    FS_LAUNCHED("k_pack");
  }
  return FS_OK;
}

extern "C" fs_status fs_buffer_write(fs_handle* h, int level, int buffer, const float* d_in) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (level < 0 || level >= h->L) return fail(FS_EINVAL, "level %d out of range", level);
  if (!d_in) return fail(FS_EINVAL, "null input");
  if (buffer == FS_BUF_MASK || buffer == FS_BUF_TENSOR || buffer == FS_BUF_STEPS)
    return fail(FS_EINVAL, "buffer %d is derived and read-only", buffer);
  HostLevel& L = h->lv[level];
  L.consts_stale = true;
  size_t n = (size_t)L.W * L.H;
  if (buffer == FS_BUF_I0 || buffer == FS_BUF_I1) {   // with the pyramid's low part
    FS_LAUNCH("k_copy_in_s", launch_copy_in_image(d_in, L.v, buffer == FS_BUF_I0 ? 0 : 1,
                                                  h->stream));
    return FS_OK;
  }
  BufLoc b;
  if ((s = buffer_loc(h, level, buffer, b)) != FS_OK) return s;
  for (int c = 0; c < b.planes; ++c) {
    if (b.kind == 2) {
      FS_LAUNCH("k_unpack_s",
                launch_unpack_s(d_in + c * n, b.s[c], L.v.st, L.W, L.H, L.P, h->stream));
      continue;
    }
    k_unpack<<<grid2(L.W, L.H), kBlock2, 0, h->stream>>>(
        d_in + c * n, b.kind == 1 ? b.f[0] + c : b.f[c], b.kind == 1 ? 2 : 1, L.W, L.H, L.P);
    FS_LAUNCHED("k_unpack");
  }
  return FS_OK;
}

extern "C" fs_status fs_run_stage(fs_handle* h, int level, int stage, int count) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (level < 0 || level >= h->L) return fail(FS_EINVAL, "level %d out of range", level);
  h->has_state = false;
  return run_stage(h, level, stage, count, h->stream);
}

extern "C" fs_status fs_stage_prerotate(fs_handle* h, const float* d_I1) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!d_I1) return fail(FS_EINVAL, "null input");
  HostLevel& L0 = h->lv[0];
  FS_LAUNCH("k_prerotate", launch_prerotate(d_I1, h->cfield, L0.v, h->stream));
  return FS_OK;
}

extern "C" fs_status fs_timing_enable(fs_handle* h, int enable) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if ((enable != 0) != (h->timing != 0) && h->gexec) {  // captured graph has / lacks the events
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  h->timing = enable != 0;
  h->ev_pending = false;
  return FS_OK;
}

extern "C" fs_status fs_timing_read(fs_handle* h, double* ms, long long* launches,
                                    double* pixel_iters, int reset) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (h->ev_pending) {
    FS_CUDA(cudaStreamSynchronize(h->stream));
    for (int l = 0; l < h->ev_levels; ++l) {
      int B = pd_block(h, l);
      for (int w = 0; w < h->ev_warps; ++w) {
        float t = 0.f;
        FS_CUDA(cudaEventElapsedTime(&t, h->ev[2 * (l * h->ev_warps + w)],
                                     h->ev[2 * (l * h->ev_warps + w) + 1]));
        h->t_ms[l] += t;
      }
      h->t_launch[l] += use_cluster(h, l)
                            ? (long long)h->ev_warps
                            : (long long)h->ev_warps * pd_launches(h->ev_iters, B);
      h->t_pxit[l] += (double)h->lv[l].W * h->lv[l].H * h->ev_warps * h->ev_iters;
    }
    h->ev_pending = false;
  }
  for (int l = 0; l < kMaxLevels; ++l) {
    if (ms) ms[l] = h->t_ms[l];
    if (launches) launches[l] = h->t_launch[l];
    if (pixel_iters) pixel_iters[l] = h->t_pxit[l];
    if (reset) { h->t_ms[l] = 0; h->t_launch[l] = 0; h->t_pxit[l] = 0; }
  }
  return FS_OK;
}

extern "C" fs_status fs_autotune(fs_handle* h, int iters, int* choice) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (iters < 1) return fail(FS_EINVAL, "iters must be >= 1");
  if ((s = ensure_schedule(h, iters)) != FS_OK) return s;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  ++h->sched_gen;
  h->has_state = false;   // the trial runs overwrite every level's state
  cudaEvent_t e0, e1;
  FS_CUDA(cudaEventCreate(&e0));
  FS_CUDA(cudaEventCreate(&e1));
  const int saved_block = h->prm.block_iters, saved_sched = h->prm.pd_schedule;
  fs_status st = FS_OK;
  for (int l = 0; l < h->L && st == FS_OK; ++l) {
    HostLevel& L = h->lv[l];
    L.tuned = -1;
    L.tuned_variant = -1;
    float best = 3.4e38f;
    int best_c = -1;
    std::vector<float> timed(kMaxChoice + 1, -1.f);
    // best of 3 timed runs after a warm-up, each candidate once
    auto try_cand = [&](int cand) {
      if (st != FS_OK || timed[cand] >= 0.f) return;
      h->prm.pd_schedule = cand == 0 ? 0 : 1;
      h->prm.block_iters = saved_block;
      decode_choice(cand, h->prm.regularizer == FS_REG_TGV, L.tuned, L.tuned_variant);
      float t = 3.4e38f;
      for (int rep = 0; rep < 4 && st == FS_OK; ++rep) {
        cudaError_t e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess && (st = run_pd(h, l, iters, h->stream)) != FS_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) { st = fail(FS_ECUDA, "fs_autotune: %s", cudaGetErrorString(e)); break; }
        if (rep > 0 && ms < t) t = ms;
      }
      timed[cand] = t;
      if (st == FS_OK && t < best) { best = t; best_c = cand; }
    };
    if (h->prm.regularizer == FS_REG_TGV) {
      // 0 = a launch per step, then every depth 1..8 on each footprint
      for (int cand = 0; cand <= kMaxTgvChoice; ++cand) try_cand(cand);
    } else {
      // 0 = cluster where the level fits one, then every depth 1..8 on every
      // footprint.  (Timing each footprint at a few depths first and only
      // the winner at all depths picked a 30 % slower level-0 schedule on
      // the 1024 x 1024 workload: the best depth, 7, lies between the
      // sampled ones, where another footprint was faster.)
      if (L.cluster >= 0 && !(h->prm.accel_gamma > 0)) try_cand(0);
      for (int cand = 1; cand <= kMaxChoice; ++cand)
        if (L.tma_ok || !is_tma_choice(cand, false)) try_cand(cand);
    }
    decode_choice(best_c, h->prm.regularizer == FS_REG_TGV, L.tuned, L.tuned_variant);
    if (choice) choice[l] = best_c;
  }
  h->prm.block_iters = saved_block;
  h->prm.pd_schedule = saved_sched;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

extern "C" fs_status fs_energy(fs_handle* h, int level, double out[4]) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (level < 0 || level >= h->L) return fail(FS_EINVAL, "level %d out of range", level);
  if (!out) return fail(FS_EINVAL, "null output");
  if (!h->eacc) {
    cudaError_t e = fs_internal_malloc((void**)&h->eacc, 3 * sizeof(double), "energy");
    if (e != cudaSuccess) { h->eacc = nullptr; return fail(FS_ENOMEM, "energy accumulator: %s", cudaGetErrorString(e)); }
  }
  double acc[3];
  FS_CUDA(cudaMemsetAsync(h->eacc, 0, sizeof(acc), h->stream));
  const bool tgv = h->prm.regularizer == FS_REG_TGV;
  FS_LAUNCH("k_energy", launch_energy(h->lv[level].v, h->prm.lambda, tgv ? 0.f : h->prm.huber_eps,
                                      tgv ? 1 : 0, h->prm.alpha0, h->prm.alpha1, h->eacc,
                                      h->stream));
  FS_CUDA(cudaMemcpyAsync(acc, h->eacc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
  FS_CUDA(cudaStreamSynchronize(h->stream));
  out[0] = acc[0] + acc[1];
  out[1] = acc[0];
  out[2] = acc[1];
  out[3] = acc[2];
  return FS_OK;
}

extern "C" fs_status fs_set_schedule(fs_handle* h, const int* choice) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!choice) return fail(FS_EINVAL, "null schedule");
  const bool tgv = h->prm.regularizer == FS_REG_TGV;
  for (int l = 0; l < h->L; ++l) {
    int c = choice[l];
    if (c < -1 || c > (tgv ? kMaxTgvChoice : kMaxChoice))
      return fail(FS_EINVAL, "level %d: schedule %d out of range", l, c);
    if (c == 0 && !tgv && (h->lv[l].cluster < 0 || h->prm.accel_gamma > 0))
      return fail(FS_EINVAL, "level %d does not fit one thread-block cluster", l);
    if (is_tma_choice(c, tgv) && !h->lv[l].tma_ok)
      return fail(FS_EINVAL, "level %d: no tensor maps for the TMA footprints", l);
  }
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  ++h->sched_gen;
  for (int l = 0; l < h->L; ++l) {
    int c = choice[l];
    HostLevel& L = h->lv[l];
    decode_choice(c, tgv, L.tuned, L.tuned_variant);
  }
  return FS_OK;
}

extern "C" fs_status fs_set_wait_limit(fs_handle* h, double seconds) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  if (!(seconds > 0 && seconds <= 3600)) return fail(FS_EINVAL, "wait limit must be in (0, 3600] s");
  h->wait_ns = (unsigned long long)(seconds * 1e9);
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }   // captured the old bound
  ++h->sched_gen;
  return FS_OK;
}

extern "C" fs_status fs_persist_stall(fs_handle* h, int stall) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  h->persist_stall = stall ? 1 : 0;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  ++h->sched_gen;
  return FS_OK;
}

extern "C" fs_status fs_check_waits(fs_handle* h) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  int v = 0;
  FS_CUDA(cudaMemcpyAsync(&v, h->pd_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  FS_CUDA(cudaStreamSynchronize(h->stream));
  if (v == 0) return FS_OK;
  FS_CUDA(cudaMemsetAsync(h->pd_status, 0, sizeof(int), h->stream));
  FS_CUDA(cudaStreamSynchronize(h->stream));
  return fail(FS_ETIMEOUT,
              "a copy wait of the TMA-staged primal-dual footprints ran out (limit %.3g s); "
              "the level state is unspecified",
              (double)h->wait_ns * 1e-9);
}

extern "C" fs_status fs_stage_depth(fs_handle* h, float* d_disp, float* d_depth) {
  fs_status s;
  if ((s = check_handle(h)) != FS_OK) return s;
  return enqueue_depth(h, d_disp, d_depth, h->stream);
}

}  // extern "C"
