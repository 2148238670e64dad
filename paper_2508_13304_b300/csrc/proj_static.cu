// Allocation-free variant of the forward pose gradient.
//
// Who needs it: code that may not allocate device memory at all - for
// example a plug-in running inside a host application that owns every
// device allocation, a real-time loop whose memory budget is frozen after
// start-up, or a caller whose allocator is not CUDA's.  Such callers can hand
// over input and output buffers but cannot call cudaMalloc for a plan or a
// workspace.  This entry point therefore needs no plan and no workspace: its
// scratch (geometry tables, the prepared (mu, grad mu) volume and the
// reduction records) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads this library keeps until the process exits.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "proj_internal.cuh"

using namespace projk;

namespace {

// Limits of the static scratch (see include/proj.h).
constexpr int kMaxPadVoxels = 74 * 70 * 68;  // pitched (mu, grad mu) volume of a 64^3 grid
constexpr int kMaxInst = 64;
constexpr int kMaxPose = 64;
constexpr int kMaxViews = 64;
constexpr int kMaxRecords = 4096;            // n_inst x ray tiles of 16 x 16 pixels

constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffStatus = 0;
constexpr size_t kOffViews = al(kOffStatus + sizeof(int));
constexpr size_t kOffInstView = al(kOffViews + sizeof(double) * 12 * kMaxViews);
constexpr size_t kOffInstPose = al(kOffInstView + sizeof(int) * kMaxInst);
constexpr size_t kOffPosePtr = al(kOffInstPose + sizeof(int) * kMaxInst);
constexpr size_t kOffPoseIdx = al(kOffPosePtr + sizeof(int) * (kMaxPose + 1));
constexpr size_t kOffInst = al(kOffPoseIdx + sizeof(int) * kMaxInst);
constexpr size_t kOffPtab = al(kOffInst + sizeof(InstTable) * kMaxInst);
constexpr size_t kOffVol4 = al(kOffPtab + sizeof(PoseTable) * kMaxPose);
constexpr size_t kOffPart = al(kOffVol4 + sizeof(float4) * (size_t)kMaxPadVoxels);
constexpr size_t kScratchBytes = al(kOffPart + sizeof(float) * kRec * (size_t)kMaxRecords);
static_assert(kScratchBytes <= (6.5 * (1 << 20)), "static scratch is documented as 6.2 MiB");

// The scratch itself.  In host code this name is only a host-side stand-in;
// its device address comes from cudaGetSymbolAddress (per device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Messages go to the library's per-thread error string (proj_last_error).
int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  record_error(buf);
  return code;
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device, looked up once per
// device with that device current.  The cached address belongs to the
// context that was current then: a cudaDeviceReset after the first call
// (which unloads this module) is not supported.
int scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PROJ_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PROJ_E_UNSUPPORTED, "device index %d not supported", dev);
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail(PROJ_E_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return PROJ_OK;
}

}  // namespace

extern "C" {

int proj_forward_pose_grad_static(const proj_geometry* geom, int n_pose, int n_inst, const int* inst_view,
                                  const int* inst_pose, const float* d_mu, const float* d_pose, int loss,
                                  const float* d_ref, float* d_grad, float* d_loss, proj_stream stream) {
  record_error("");
  if (!geom || !inst_view || !inst_pose || !d_mu || !d_pose || !d_ref || !d_grad)
    return fail(PROJ_E_ARG, "NULL argument");
  const proj_geometry& G = *geom;
  if (loss != PROJ_LOSS_RESIDUAL && loss != PROJ_LOSS_L2 && loss != PROJ_LOSS_NCC)
    return fail(PROJ_E_ARG, "unknown loss mode %d", loss);
  if (G.nx < 1 || G.ny < 1 || G.nz < 1 || G.nu < 1 || G.nv < 1 || G.n_views < 1 || !G.views || n_pose < 1 ||
      n_inst < 1)
    return fail(PROJ_E_ARG, "sizes must be >= 1 and the view table non-NULL");
  if (!(std::isfinite(G.vx) && G.vx > 0 && std::isfinite(G.vy) && G.vy > 0 && std::isfinite(G.vz) && G.vz > 0 &&
        std::isfinite(G.step) && G.step > 0))
    return fail(PROJ_E_ARG, "voxel pitch and ray step must be finite and > 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(G.vol_offset[a])) return fail(PROJ_E_ARG, "volume offset must be finite");
  // Size limits of the static scratch.
  int pqx, pqy, pqz;
  volume_pitches(G.nx, G.ny, G.nz, &pqx, &pqy, &pqz);
  const long long npad = (long long)pqx * pqy * pqz;
  const long long n_tiles = (long long)ceil_div(G.nu, kTileU) * ceil_div(G.nv, kTileV);
  if (npad > kMaxPadVoxels)
    return fail(PROJ_E_ARG, "volume %d x %d x %d exceeds the static scratch limit (%lld padded voxels > %d)", G.nx,
                G.ny, G.nz, npad, kMaxPadVoxels);
  if (n_inst > kMaxInst) return fail(PROJ_E_ARG, "n_inst %d exceeds the static scratch limit of %d", n_inst, kMaxInst);
  if (n_pose > kMaxPose) return fail(PROJ_E_ARG, "n_pose %d exceeds the static scratch limit of %d", n_pose, kMaxPose);
  if (G.n_views > kMaxViews)
    return fail(PROJ_E_ARG, "n_views %d exceeds the static scratch limit of %d", G.n_views, kMaxViews);
  if (n_inst * n_tiles > kMaxRecords)
    return fail(PROJ_E_ARG, "n_inst x detector tiles (%lld) exceeds the static scratch limit of %d",
                (long long)n_inst * n_tiles, kMaxRecords);
  for (int v = 0; v < G.n_views; ++v) {
    const double* w = G.views + 12 * v;
    for (int a = 0; a < 12; ++a)
      if (!std::isfinite(w[a])) return fail(PROJ_E_ARG, "view %d has a non-finite entry", v);
    double q00[3], B[9];
    for (int a = 0; a < 3; ++a) {
      q00[a] = w[3 + a] - 0.5 * (G.nu - 1) * w[6 + a] - 0.5 * (G.nv - 1) * w[9 + a];
      B[3 * a] = w[6 + a];
      B[3 * a + 1] = w[9 + a];
      B[3 * a + 2] = q00[a] - w[a];
    }
    const double det = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                       B[2] * (B[3] * B[7] - B[4] * B[6]);
    const double scale = std::sqrt(B[0] * B[0] + B[3] * B[3] + B[6] * B[6]) *
                         std::sqrt(B[1] * B[1] + B[4] * B[4] + B[7] * B[7]) *
                         std::sqrt(B[2] * B[2] + B[5] * B[5] + B[8] * B[8]);
    if (!(std::fabs(det) > 1e-12 * scale)) return fail(PROJ_E_ARG, "view %d: singular detector basis", v);
  }
  int ptr[kMaxPose + 1] = {0}, idx[kMaxInst], fill[kMaxPose];
  for (int i = 0; i < n_inst; ++i) {
    if (inst_view[i] < 0 || inst_view[i] >= G.n_views || inst_pose[i] < 0 || inst_pose[i] >= n_pose)
      return fail(PROJ_E_ARG, "instance %d: view %d / pose %d out of range", i, inst_view[i], inst_pose[i]);
    ptr[inst_pose[i] + 1]++;
  }
  for (int q = 0; q < n_pose; ++q) ptr[q + 1] += ptr[q];
  for (int q = 0; q < n_pose; ++q) fill[q] = ptr[q];
  for (int i = 0; i < n_inst; ++i) idx[fill[inst_pose[i]]++] = i;

  Geo g;
  g.nx = G.nx;
  g.ny = G.ny;
  g.nz = G.nz;
  g.px = G.nx + 2;
  g.py = G.ny + 2;
  g.pz = G.nz + 2;
  volume_pitches(G.nx, G.ny, G.nz, &g.qx, &g.qy, &g.qz);
  volume_pitches_yfast(G.nx, G.ny, &g.rqx, &g.rqy);  // no y-fast copy here: every instance marches vol4
  g.vx = (float)G.vx;
  g.vy = (float)G.vy;
  g.vz = (float)G.vz;
  g.hx = 0.5f * (G.nx + 1);
  g.hy = 0.5f * (G.ny + 1);
  g.hz = 0.5f * (G.nz + 1);
  g.gx = 0.5f * (G.nx + 3);
  g.gy = 0.5f * (G.ny + 3);
  g.gz = 0.5f * (G.nz + 3);
  g.cx = 0.5f * (G.nx - 1);
  g.cy = 0.5f * (G.ny - 1);
  g.cz = 0.5f * (G.nz - 1);
  g.offx = (float)G.vol_offset[0];
  g.offy = (float)G.vol_offset[1];
  g.offz = (float)G.vol_offset[2];
  g.nu = G.nu;
  g.nv = G.nv;
  g.step = (float)G.step;

  // Each call copies its host tables (the caller's view table and instance
  // maps, and CSR arrays on this function's stack) with cudaMemcpyAsync.
  // A graph captured from such a call would read those host buffers again
  // at every replay, long after they are gone, so a capturing stream is
  // refused before anything is enqueued.
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess) return fail(PROJ_E_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(ce));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(PROJ_E_ARG, "the stream is capturing a CUDA graph; this entry point cannot be captured");

  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  int* status = reinterpret_cast<int*>(base + kOffStatus);
  double* views = reinterpret_cast<double*>(base + kOffViews);
  int* d_iv = reinterpret_cast<int*>(base + kOffInstView);
  int* d_ip = reinterpret_cast<int*>(base + kOffInstPose);
  int* d_ptr = reinterpret_cast<int*>(base + kOffPosePtr);
  int* d_idx = reinterpret_cast<int*>(base + kOffPoseIdx);
  InstTable* inst = reinterpret_cast<InstTable*>(base + kOffInst);
  PoseTable* ptab = reinterpret_cast<PoseTable*>(base + kOffPtab);
  float4* vol4 = reinterpret_cast<float4*>(base + kOffVol4);
  float* part = reinterpret_cast<float*>(base + kOffPart);

  // Host tables into the scratch (pageable sources: each copy returns once
  // its source has been read).  The status word starts each call at zero.
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(views, G.views, sizeof(double) * 12 * G.n_views, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_iv, inst_view, sizeof(int) * n_inst, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ip, inst_pose, sizeof(int) * n_inst, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ptr, ptr, sizeof(int) * (n_pose + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_idx, idx, sizeof(int) * n_inst, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(PROJ_E_CUDA, "table upload: %s", cudaGetErrorString(e));
  e = launch_volume_prep(d_mu, g, nullptr, vol4, s);
  if (e == cudaSuccess) e = launch_setup(d_pose, n_pose, views, d_iv, d_ip, n_inst, g, inst, ptab, status, s);
  if (e == cudaSuccess) e = launch_forward_grad(inst, n_inst, g, vol4, nullptr, loss, d_ref, nullptr, part, s);
  if (e == cudaSuccess)
    e = launch_forward_grad_reduce(inst, ptab, n_pose, d_ptr, d_idx, (int)n_tiles, g, loss, part, d_grad, d_loss, s);
  if (e != cudaSuccess) return fail(PROJ_E_CUDA, "launch: %s", cudaGetErrorString(e));
  return PROJ_OK;
}

}  // extern "C"
