// C ABI of the projector library (declared in include/proj.h): plan
// creation, host-side argument validation, workspace layout and the
// launch sequence of each operation.  No entry point allocates device
// memory except proj_plan_create (the plan's small tables).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "proj_internal.cuh"
#include "proj_optim.cuh"

using namespace projk;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(PROJ_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

void projk::record_error(const char* msg) { g_last_error = msg; }

struct proj_plan_s {
  Geo geo;
  int n_views, n_pose, n_inst, ops;
  int device;
  int n_tiles;        // ray tiles per instance
  int ipp = 1;        // most instances of any one pose (grid slots per pose of a pose list)
  int bp_blocks;      // most voxel bricks of the back-projection gradient over the brick shapes (records per instance)
  int bp_shape = 3;   // brick shape of the back-projection gradient (0..kBrickShapes-1)
  std::vector<double> views;
  std::vector<int> inst_view, inst_pose;
  // device tables owned by the plan
  double* d_views = nullptr;
  int* d_inst_view = nullptr;
  int* d_inst_pose = nullptr;
  int* d_pose_ptr = nullptr;
  int* d_pose_idx = nullptr;
  FdkView* d_fdk = nullptr;  // per instance
  // rays per warp row in the fused pose-gradient march (2, 4, 8 or 16)
  int warp_width = 4;
  // empty-space skipping in the forward marches: log2 of the occupancy brick edge (3: 8 cells, 4: 16), 0 = off
  int skip_shift = 3;
  // and the per-sample test of the cell map in the fused march: 0 off, 1 on, 2 automatic (default; decided
  // on the device by proj_set_volume from the volume's cells, see k_cell_decide)
  int skip_cells = 2;
  // optional timing of the main kernel of each call
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // workspace layout (byte offsets; 0 = buffer absent, the status word sits at 0)
  size_t off_status = 0, off_inst = 0, off_ptab = 0, off_volq = 0, off_volqy = 0, off_vol4 = 0, off_vol4y = 0, off_part_f = 0,
         off_det4 = 0,
         off_part_b = 0, off_detq = 0, off_acc = 0, off_sharp_m = 0, off_sharp_part = 0, off_occ8 = 0, off_occ16 = 0,
         off_nbits = 0, off_cells = 0, off_cstat = 0, off_volb = 0,
         ws_bytes = 0;
};

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

struct WsView {
  int* status = nullptr;
  InstTable* inst = nullptr;
  PoseTable* ptab = nullptr;
  float4* volq = nullptr;
  float4* volqy = nullptr;
  float4* vol4 = nullptr;
  float4* vol4y = nullptr;
  float* part_f = nullptr;
  float4* det4 = nullptr;
  float* part_b = nullptr;
  float4* acc = nullptr;
  float4* detq = nullptr;
  unsigned char* occ8 = nullptr;
  unsigned char* occ16 = nullptr;
  unsigned* nbits = nullptr;
  unsigned* cells = nullptr;
  void* cstat = nullptr;
  float4* volb = nullptr;
};

int check_ws(const proj_plan_s* p, void* d_ws, size_t ws_bytes, WsView* w) {
  if (!d_ws) return fail(PROJ_E_WORKSPACE, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(d_ws) % kAlign) return fail(PROJ_E_WORKSPACE, "workspace is not 256-byte aligned");
  if (ws_bytes < p->ws_bytes)
    return fail(PROJ_E_WORKSPACE, "workspace has %zu bytes, plan needs %zu", ws_bytes, p->ws_bytes);
  char* b = static_cast<char*>(d_ws);
  w->status = reinterpret_cast<int*>(b + p->off_status);
  w->inst = reinterpret_cast<InstTable*>(b + p->off_inst);
  w->ptab = reinterpret_cast<PoseTable*>(b + p->off_ptab);
  w->volq = p->off_volq ? reinterpret_cast<float4*>(b + p->off_volq) : nullptr;
  w->volqy = p->off_volqy ? reinterpret_cast<float4*>(b + p->off_volqy) : nullptr;
  w->vol4 = p->off_vol4 ? reinterpret_cast<float4*>(b + p->off_vol4) : nullptr;
  w->vol4y = p->off_vol4y ? reinterpret_cast<float4*>(b + p->off_vol4y) : nullptr;
  w->part_f = p->off_part_f ? reinterpret_cast<float*>(b + p->off_part_f) : nullptr;
  w->det4 = p->off_det4 ? reinterpret_cast<float4*>(b + p->off_det4) : nullptr;
  w->part_b = p->off_part_b ? reinterpret_cast<float*>(b + p->off_part_b) : nullptr;
  w->acc = p->off_acc ? reinterpret_cast<float4*>(b + p->off_acc) : nullptr;
  w->detq = p->off_detq ? reinterpret_cast<float4*>(b + p->off_detq) : nullptr;
  w->occ8 = p->off_occ8 ? reinterpret_cast<unsigned char*>(b + p->off_occ8) : nullptr;
  w->occ16 = p->off_occ16 ? reinterpret_cast<unsigned char*>(b + p->off_occ16) : nullptr;
  w->nbits = p->off_nbits ? reinterpret_cast<unsigned*>(b + p->off_nbits) : nullptr;
  w->cells = p->off_cells ? reinterpret_cast<unsigned*>(b + p->off_cells) : nullptr;
  w->cstat = p->off_cstat ? static_cast<void*>(b + p->off_cstat) : nullptr;
  w->volb = p->off_volb ? reinterpret_cast<float4*>(b + p->off_volb) : nullptr;
  return PROJ_OK;
}

// The occupancy bricks (edge 2^shift; shift 0: none) and the cell map the forward marches skip with; cells:
// 0 no cell test, 1 always, 2 as decided for the volume by proj_set_volume.
Occ occ_of(const proj_plan_s* p, const WsView& w, int shift, int cells) {
  Occ o{};
  if (cells && w.cells) {
    o.cells = w.cells;
    o.cw = cell_words(p->geo.nx);
    o.ch = p->geo.ny + 3;
    o.cells_flag = cells == 2 ? cell_flag_of(w.cstat) : nullptr;
  }
  unsigned char* m = shift == 3 ? w.occ8 : (shift == 4 ? w.occ16 : nullptr);
  if (!m) return o;
  o.map = m;
  o.shift = shift;
  o.nb[0] = occ_bricks(p->geo.nx, shift);
  o.nb[1] = occ_bricks(p->geo.ny, shift);
  o.nb[2] = occ_bricks(p->geo.nz, shift);
  return o;
}

// The plan's own setting.
Occ occ_of(const proj_plan_s* p, const WsView& w) { return occ_of(p, w, p->skip_shift, p->skip_cells); }

int need_op(const proj_plan_s* p, int op, const char* name) {
  if (!(p->ops & op)) return fail(PROJ_E_UNSUPPORTED, "%s: operation not enabled when the plan was created", name);
  return PROJ_OK;
}

int setup(const proj_plan_s* p, const float* d_pose, const WsView& w, cudaStream_t s) {
  cudaError_t e = launch_setup(d_pose, p->n_pose, p->d_views, p->d_inst_view, p->d_inst_pose, p->n_inst, p->geo,
                               w.inst, w.ptab, w.status, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "pose set-up launch");
}

void mark(const proj_plan_s* p, bool before, cudaStream_t s) {
  if (p->timing) cudaEventRecord(before ? p->ev0 : p->ev1, s);
}

int check_device(const proj_plan_s* p) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != p->device) return fail(PROJ_E_ARG, "current device %d differs from the plan's device %d", dev, p->device);
  return PROJ_OK;
}

}  // namespace

extern "C" {

const char* proj_last_error(void) { return g_last_error.c_str(); }

const char* proj_version(void) { return "b300-diffproj 0.1 (sm_103a)"; }

int proj_plan_create(const proj_geometry* geom, int n_pose, int n_inst, const int* inst_view, const int* inst_pose,
                     int ops, proj_plan* out) {
  g_last_error.clear();
  if (!out) return fail(PROJ_E_ARG, "out is NULL");
  *out = nullptr;
  if (!geom) return fail(PROJ_E_ARG, "geometry is NULL");
  const proj_geometry& G = *geom;
  if (G.nx < 1 || G.ny < 1 || G.nz < 1) return fail(PROJ_E_ARG, "volume size %d x %d x %d", G.nx, G.ny, G.nz);
  if (G.nu < 1 || G.nv < 1) return fail(PROJ_E_ARG, "detector size %d x %d", G.nu, G.nv);
  const long long npad = (long long)(G.nx + 2) * (G.ny + 2) * (G.nz + 2);
  int qx, qy, qz;
  volume_pitches(G.nx, G.ny, G.nz, &qx, &qy, &qz);
  const long long npad2 = (long long)qx * qy * qz;
  if (npad2 >= (1LL << 31)) return fail(PROJ_E_ARG, "volume too large (padded voxel count %lld >= 2^31)", npad2);
  int rqx, rqy;
  volume_pitches_yfast(G.nx, G.ny, &rqx, &rqy);
  const long long npad2y = (long long)rqx * rqy * qz;
  if (npad2y >= (1LL << 31)) return fail(PROJ_E_ARG, "volume too large (padded voxel count %lld >= 2^31)", npad2y);
  if ((long long)(G.nu + 4) * (G.nv + 4) >= (1LL << 31)) return fail(PROJ_E_ARG, "detector too large");
  if (!finite_pos(G.vx) || !finite_pos(G.vy) || !finite_pos(G.vz))
    return fail(PROJ_E_ARG, "voxel pitch must be finite and > 0");
  if (!finite_pos(G.step)) return fail(PROJ_E_ARG, "ray step must be finite and > 0");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(G.vol_offset[a])) return fail(PROJ_E_ARG, "volume offset must be finite");
  if (G.n_views < 1 || !G.views) return fail(PROJ_E_ARG, "need n_views >= 1 and a view table");
  if (n_pose < 1) return fail(PROJ_E_ARG, "n_pose must be >= 1");
  if (n_inst < 1 || !inst_view || !inst_pose) return fail(PROJ_E_ARG, "need n_inst >= 1 and instance maps");
  if ((ops & PROJ_OP_ALL) == 0 || (ops & ~(PROJ_OP_ALL | PROJ_FLAG_ONE_COPY | PROJ_FLAG_BRICKS)))
    return fail(PROJ_E_ARG, "ops must be a non-empty OR of PROJ_OP_* (plus PROJ_FLAG_* options)");
  // launch grids put volume rows / slices, detector rows and (for the detector stack) instances in
  // the y and z grid dimensions
  if (G.ny > 65000 || G.nz > 65000 || G.nv > 65000) return fail(PROJ_E_ARG, "ny, nz and nv must be <= 65000");
  if ((ops & (PROJ_OP_BACK | PROJ_OP_BACK_GRAD)) && n_inst > 65535)
    return fail(PROJ_E_ARG, "PROJ_OP_BACK and PROJ_OP_BACK_GRAD support at most 65535 instances per plan");
  for (int v = 0; v < G.n_views; ++v) {
    const double* w = G.views + 12 * v;
    for (int a = 0; a < 12; ++a)
      if (!std::isfinite(w[a])) return fail(PROJ_E_ARG, "view %d has a non-finite entry", v);
    // detector basis B = [U | V | q00 - s] must be invertible
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
  for (int i = 0; i < n_inst; ++i) {
    if (inst_view[i] < 0 || inst_view[i] >= G.n_views)
      return fail(PROJ_E_ARG, "instance %d: view %d out of range [0, %d)", i, inst_view[i], G.n_views);
    if (inst_pose[i] < 0 || inst_pose[i] >= n_pose)
      return fail(PROJ_E_ARG, "instance %d: pose %d out of range [0, %d)", i, inst_pose[i], n_pose);
  }

  proj_plan_s* p = new proj_plan_s();
  Geo& g = p->geo;
  g.nx = G.nx;
  g.ny = G.ny;
  g.nz = G.nz;
  g.px = G.nx + 2;
  g.py = G.ny + 2;
  g.pz = G.nz + 2;
  volume_pitches(G.nx, G.ny, G.nz, &g.qx, &g.qy, &g.qz);
  volume_pitches_yfast(G.nx, G.ny, &g.rqx, &g.rqy);
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
  p->n_views = G.n_views;
  p->n_pose = n_pose;
  p->n_inst = n_inst;
  p->ops = ops;
  p->views.assign(G.views, G.views + 12 * (size_t)G.n_views);
  p->inst_view.assign(inst_view, inst_view + n_inst);
  p->inst_pose.assign(inst_pose, inst_pose + n_inst);
  p->n_tiles = ceil_div(G.nu, kTileU) * ceil_div(G.nv, kTileV);

  // CSR list of instances per pose (ascending instance order).
  std::vector<int> ptr(n_pose + 1, 0), idx(n_inst);
  int p_ipp = 1;
  for (int i = 0; i < n_inst; ++i) ptr[inst_pose[i] + 1]++;
  for (int q = 0; q < n_pose; ++q) ptr[q + 1] += ptr[q];
  for (int q = 0; q < n_pose; ++q) p_ipp = std::max(p_ipp, ptr[q + 1] - ptr[q]);
  {
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < n_inst; ++i) idx[fill[inst_pose[i]]++] = i;
  }
  p->ipp = p_ipp;

  cudaError_t e = cudaGetDevice(&p->device);
  int n_sm = 148;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "device query");
  }
  // records of the back-projection gradient: one per voxel brick and instance
  p->bp_blocks = 0;
  for (int b = 0; b < kBrickShapes; ++b) p->bp_blocks = std::max(p->bp_blocks, back_grad_blocks(p->geo, b));
  (void)n_sm;

  // Workspace layout.
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  p->off_status = take(sizeof(int));
  p->off_inst = take(sizeof(InstTable) * (size_t)n_inst);
  p->off_ptab = take(sizeof(PoseTable) * (size_t)n_pose);
  const size_t npad_sz = (size_t)npad;
  const size_t nrec = (size_t)(G.nx + 2) * (G.ny + 2) * record_slices(G.nz);
  p->off_volq = (ops & PROJ_OP_FORWARD) ? take(sizeof(float4) * nrec) : 0;
  const bool bricks = (ops & PROJ_FLAG_BRICKS) != 0;
  const bool two_copies = !(ops & PROJ_FLAG_ONE_COPY);
  p->off_volqy = ((ops & PROJ_OP_FORWARD) && two_copies) ? take(sizeof(float4) * nrec) : 0;
  p->off_vol4 = (ops & PROJ_OP_FORWARD_GRAD) ? take(sizeof(float4) * (size_t)npad2) : 0;
  p->off_vol4y = ((ops & PROJ_OP_FORWARD_GRAD) && two_copies && !bricks) ? take(sizeof(float4) * (size_t)npad2y) : 0;
  p->off_volb = ((ops & PROJ_OP_FORWARD_GRAD) && bricks)
                    ? take(sizeof(float4) * (size_t)vb_n(G.nx) * vb_n(G.ny) * vb_n(G.nz) * kVbElems)
                    : 0;
  p->off_part_f = (ops & PROJ_OP_FORWARD_GRAD) ? take(sizeof(float) * kRec * (size_t)n_inst * p->n_tiles) : 0;
  // the detector scratch of proj_back (cell records) and of proj_back_pose_grad (the (l, d_u l, d_v l)
  // stack) are never needed by the same call: one region serves both
  {
    const size_t det4_bytes = (ops & PROJ_OP_BACK_GRAD) ? sizeof(float4) * (size_t)n_inst * (G.nu + 4) * (G.nv + 4) : 0;
    const size_t detq_bytes = (ops & PROJ_OP_BACK) ? sizeof(float4) * (size_t)n_inst * (G.nu + 1) * (G.nv + 1) : 0;
    const size_t off_det = (det4_bytes || detq_bytes) ? take(std::max(det4_bytes, detq_bytes)) : 0;
    p->off_det4 = det4_bytes ? off_det : 0;
    p->off_detq = detq_bytes ? off_det : 0;
  }
  p->off_part_b = (ops & PROJ_OP_BACK_GRAD) ? take(sizeof(float) * 12 * (size_t)n_inst * p->bp_blocks) : 0;
  p->off_acc = (ops & PROJ_OP_ADJOINT) ? take(sizeof(float4) * npad_sz) : 0;
  if (ops & (PROJ_OP_FORWARD | PROJ_OP_FORWARD_GRAD)) {
    p->off_occ8 = take((size_t)occ_bricks(G.nx, 3) * occ_bricks(G.ny, 3) * occ_bricks(G.nz, 3));
    p->off_occ16 = take((size_t)occ_bricks(G.nx, 4) * occ_bricks(G.ny, 4) * occ_bricks(G.nz, 4));
    p->off_nbits = take(sizeof(unsigned) * (size_t)nbits_words(p->geo.qx) * p->geo.qy * p->geo.qz);
    p->off_cells = take(sizeof(unsigned) * (size_t)cell_words(G.nx) * (G.ny + 3) * (G.nz + 3));
    p->off_cstat = take(kCellStatBytes);
  }
  if (ops & PROJ_OP_SHARPNESS) {
    p->off_sharp_m = take(sizeof(float) * (size_t)G.nx * G.ny * G.nz);
    p->off_sharp_part = take(sizeof(double) * (2 * (size_t)sharpness_blocks(g) + 2));
  }
  p->ws_bytes = off;

  // FDK constants per instance (FP64 on the host).
  std::vector<FdkView> fdk(n_inst);
  for (int i = 0; i < n_inst; ++i) {
    const double* w = G.views + 12 * inst_view[i];
    const double *sv = w, *cv = w + 3, *U = w + 6, *V = w + 9;
    double nrm[3] = {U[1] * V[2] - U[2] * V[1], U[2] * V[0] - U[0] * V[2], U[0] * V[1] - U[1] * V[0]};
    const double nl = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
    for (int a = 0; a < 3; ++a) nrm[a] /= nl;
    double sdd = 0, sad = 0;
    for (int a = 0; a < 3; ++a) {
      sdd += (cv[a] - sv[a]) * nrm[a];
      sad += -sv[a] * nrm[a];
    }
    if (sdd < 0) {
      sdd = -sdd;
      sad = -sad;
      for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
    }
    // principal point: foot of the perpendicular from the source, in pixel
    // indices (q00 + pu U + pv V, solved in the detector basis)
    double q00[3], d[3];
    for (int a = 0; a < 3; ++a) {
      q00[a] = cv[a] - 0.5 * (G.nu - 1) * U[a] - 0.5 * (G.nv - 1) * V[a];
      d[a] = sv[a] + sdd * nrm[a] - q00[a];
    }
    const double uu = U[0] * U[0] + U[1] * U[1] + U[2] * U[2], vv = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    const double uvd = U[0] * V[0] + U[1] * V[1] + U[2] * V[2];
    const double du_ = d[0] * U[0] + d[1] * U[1] + d[2] * U[2], dv_ = d[0] * V[0] + d[1] * V[1] + d[2] * V[2];
    const double det = uu * vv - uvd * uvd;
    FdkView f;
    f.pu = (float)((du_ * vv - dv_ * uvd) / det);
    f.pv = (float)((dv_ * uu - du_ * uvd) / det);
    f.sad = (float)sad;
    f.du = (float)(std::sqrt(uu) * sad / sdd);
    f.dv = (float)(std::sqrt(vv) * sad / sdd);
    f.pad[0] = f.pad[1] = f.pad[2] = 0.f;
    fdk[i] = f;
  }

  e = cudaMalloc(&p->d_views, sizeof(double) * p->views.size());
  if (e == cudaSuccess) e = cudaMalloc(&p->d_inst_view, sizeof(int) * n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_inst_pose, sizeof(int) * n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_pose_ptr, sizeof(int) * (n_pose + 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_pose_idx, sizeof(int) * n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_fdk, sizeof(FdkView) * n_inst);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_fdk, fdk.data(), sizeof(FdkView) * n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_views, p->views.data(), sizeof(double) * p->views.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_inst_view, inst_view, sizeof(int) * n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_inst_pose, inst_pose, sizeof(int) * n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_pose_ptr, ptr.data(), sizeof(int) * (n_pose + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_pose_idx, idx.data(), sizeof(int) * n_inst, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    proj_plan_destroy(p);
    return cuda_fail(e, "plan table allocation");
  }
  *out = p;
  return PROJ_OK;
}

int proj_plan_destroy(proj_plan p) {
  if (!p) return PROJ_OK;
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  cudaFree(p->d_views);
  cudaFree(p->d_inst_view);
  cudaFree(p->d_inst_pose);
  cudaFree(p->d_pose_ptr);
  cudaFree(p->d_pose_idx);
  cudaFree(p->d_fdk);
  delete p;
  return PROJ_OK;
}

int proj_workspace_size(proj_plan p, size_t* bytes) {
  if (!p || !bytes) return fail(PROJ_E_ARG, "plan or bytes is NULL");
  *bytes = p->ws_bytes;
  return PROJ_OK;
}

int proj_set_volume(proj_plan p, const float* d_mu, void* d_ws, size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_mu) return fail(PROJ_E_ARG, "d_mu is NULL");
  if (!(p->ops & (PROJ_OP_FORWARD | PROJ_OP_FORWARD_GRAD)))
    return fail(PROJ_E_UNSUPPORTED, "proj_set_volume: no ray-driven operation enabled");
  WsView w;
  int rc = check_ws(p, d_ws, ws_bytes, &w);
  if (rc) return rc;
  if ((rc = check_device(p))) return rc;
  cudaError_t e = launch_volume_prep(d_mu, p->geo, w.volq, w.vol4, (cudaStream_t)stream, w.nbits, w.vol4y);
  if (e == cudaSuccess && w.cells)
    e = launch_cell_bits(w.nbits, p->geo, w.cells, w.occ8, w.occ16, w.cstat, (cudaStream_t)stream);
  if (e == cudaSuccess && w.volb) e = launch_volume_bricks(w.vol4, p->geo, w.volb, (cudaStream_t)stream);
  if (e == cudaSuccess && w.volqy) e = launch_records_yfast(w.volq, p->geo, w.volqy, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "volume preparation launch");
}

int proj_forward(proj_plan p, const float* d_pose, float* d_proj, void* d_ws, size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_proj) return fail(PROJ_E_ARG, "proj_forward: NULL pose or output");
  int rc = need_op(p, PROJ_OP_FORWARD, "proj_forward");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  mark(p, true, s);
  cudaError_t e = launch_forward(w.inst, p->n_inst, p->geo, w.volq, w.volqy, d_proj, s, occ_of(p, w));
  mark(p, false, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "forward launch");
}

int proj_count_samples(proj_plan p, const float* d_pose, long long* d_count, void* d_ws, size_t ws_bytes,
                       proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_count) return fail(PROJ_E_ARG, "proj_count_samples: NULL pose or output");
  WsView w;
  int rc = check_ws(p, d_ws, ws_bytes, &w);
  if (rc) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  cudaError_t e = launch_count(w.inst, p->n_inst, p->geo, d_count, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "count launch");
}

int proj_forward_pose_grad(proj_plan p, const float* d_pose, int loss, const float* d_ref, float* d_grad,
                           float* d_loss, float* d_proj, void* d_ws, size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_ref || !d_grad) return fail(PROJ_E_ARG, "proj_forward_pose_grad: NULL pose, reference or grad");
  if (loss != PROJ_LOSS_RESIDUAL && loss != PROJ_LOSS_L2 && loss != PROJ_LOSS_NCC)
    return fail(PROJ_E_ARG, "unknown loss mode %d", loss);
  int rc = need_op(p, PROJ_OP_FORWARD_GRAD, "proj_forward_pose_grad");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  mark(p, true, s);
  cudaError_t e =
      launch_forward_grad(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, loss, d_ref, d_proj, w.part_f, s, p->warp_width,
                          nullptr, occ_of(p, w), w.volb);
  mark(p, false, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward pose-gradient launch");
  e = launch_forward_grad_reduce(w.inst, w.ptab, p->n_pose, p->d_pose_ptr, p->d_pose_idx, p->n_tiles, p->geo, loss,
                                 w.part_f, d_grad, d_loss, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "forward pose-gradient reduction launch");
}

int proj_forward_pose_grad_list(proj_plan p, const float* d_pose, const int* d_pose_list, int n_list, int loss,
                                const float* d_ref, float* d_grad, float* d_loss, float* d_proj, void* d_ws,
                                size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_pose_list || !d_ref || !d_grad)
    return fail(PROJ_E_ARG, "proj_forward_pose_grad_list: NULL pose, pose list, reference or grad");
  if (n_list < 1) return fail(PROJ_E_ARG, "proj_forward_pose_grad_list: n_list must be >= 1");
  if ((long long)n_list * p->ipp * p->n_tiles > 0x7fffffffLL)
    return fail(PROJ_E_ARG, "proj_forward_pose_grad_list: n_list x instances per pose x tiles exceeds 2^31 - 1");
  if (loss != PROJ_LOSS_RESIDUAL && loss != PROJ_LOSS_L2 && loss != PROJ_LOSS_NCC)
    return fail(PROJ_E_ARG, "unknown loss mode %d", loss);
  int rc = need_op(p, PROJ_OP_FORWARD_GRAD, "proj_forward_pose_grad_list");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  PoseList L{d_pose_list, n_list, p->ipp, p->n_pose, p->d_pose_ptr, p->d_pose_idx, w.status};
  mark(p, true, s);
  cudaError_t e = launch_forward_grad(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, loss, d_ref, d_proj, w.part_f, s,
                                      p->warp_width, &L, occ_of(p, w), w.volb);
  mark(p, false, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward pose-gradient launch");
  e = launch_forward_grad_reduce(w.inst, w.ptab, p->n_pose, p->d_pose_ptr, p->d_pose_idx, p->n_tiles, p->geo, loss,
                                 w.part_f, d_grad, d_loss, s, d_pose_list, n_list);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "forward pose-gradient reduction launch");
}

int proj_back(proj_plan p, const float* d_proj, const float* d_pose, int weight, float* d_vol, void* d_ws,
              size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_proj || !d_pose || !d_vol) return fail(PROJ_E_ARG, "proj_back: NULL input or output");
  if (weight != PROJ_W_NONE && weight != PROJ_W_FDK && weight != PROJ_W_FDK_CONST)
    return fail(PROJ_E_ARG, "unknown weight %d", weight);
  int rc = need_op(p, PROJ_OP_BACK, "proj_back");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  mark(p, true, s);
  cudaError_t e = launch_back(w.inst, p->n_inst, p->geo, weight, d_proj, w.detq, d_vol, s);
  mark(p, false, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "back-projection launch");
}

int proj_back_adjoint(proj_plan p, const float* d_vol, const float* d_pose, int weight, float* d_proj, void* d_ws,
                      size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_vol || !d_pose || !d_proj) return fail(PROJ_E_ARG, "proj_back_adjoint: NULL argument");
  if (weight != PROJ_W_NONE && weight != PROJ_W_FDK && weight != PROJ_W_FDK_CONST)
    return fail(PROJ_E_ARG, "unknown weight %d", weight);
  int rc = need_op(p, PROJ_OP_BACK, "proj_back_adjoint");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  mark(p, true, s);
  cudaError_t e = launch_back_adjoint(w.inst, p->n_inst, p->geo, weight, d_vol, w.detq, d_proj, s);
  mark(p, false, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "back-projection adjoint launch");
}

int proj_back_pose_grad(proj_plan p, const float* d_proj, const float* d_pose, int weight, const float* d_vol_resid,
                        float* d_grad, void* d_ws, size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_proj || !d_pose || !d_vol_resid || !d_grad) return fail(PROJ_E_ARG, "proj_back_pose_grad: NULL argument");
  if (weight != PROJ_W_NONE && weight != PROJ_W_FDK && weight != PROJ_W_FDK_CONST)
    return fail(PROJ_E_ARG, "unknown weight %d", weight);
  int rc = need_op(p, PROJ_OP_BACK_GRAD, "proj_back_pose_grad");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  cudaError_t e = launch_detector_prep(d_proj, p->n_inst, p->geo, w.det4, s);
  if (e != cudaSuccess) return cuda_fail(e, "detector-gradient launch");
  mark(p, true, s);
  e = launch_back_grad(w.inst, p->n_inst, p->geo, weight, w.det4, d_vol_resid, w.part_b, p->bp_shape, s);
  mark(p, false, s);
  if (e != cudaSuccess) return cuda_fail(e, "back-projection gradient launch");
  e = launch_back_grad_reduce(w.ptab, p->n_pose, p->d_pose_ptr, p->d_pose_idx, p->n_inst,
                              back_grad_blocks(p->geo, p->bp_shape), p->geo,
                              w.part_b, d_grad, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "back-projection gradient reduction launch");
}

int proj_forward_adjoint(proj_plan p, const float* d_y, const float* d_pose, float* d_vol, void* d_ws,
                         size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_y || !d_pose || !d_vol) return fail(PROJ_E_ARG, "proj_forward_adjoint: NULL argument");
  int rc = need_op(p, PROJ_OP_ADJOINT, "proj_forward_adjoint");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  mark(p, true, s);
  cudaError_t e = launch_forward_adjoint(w.inst, p->n_inst, p->geo, d_y, w.acc, d_vol, s);
  mark(p, false, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "forward adjoint launch");
}

int proj_gather_probe(proj_plan p, const float* d_pose, void* d_ws, size_t ws_bytes, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose) return fail(PROJ_E_ARG, "proj_gather_probe: NULL pose");
  int rc = need_op(p, PROJ_OP_FORWARD_GRAD, "proj_gather_probe");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  mark(p, true, s);
  cudaError_t e = launch_gather_probe(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, w.part_f, s,
                                      occ_of(p, w), w.volb);
  mark(p, false, s);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "gather probe launch");
}

int proj_set_warp_shape(proj_plan p, int warp_width) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (warp_width != 2 && warp_width != 4 && warp_width != 8 && warp_width != 16)
    return fail(PROJ_E_ARG, "warp width %d is not one of 2, 4, 8, 16", warp_width);
  p->warp_width = warp_width;
  return PROJ_OK;
}

int proj_get_warp_shape(proj_plan p, int* warp_width) {
  if (!p || !warp_width) return fail(PROJ_E_ARG, "plan or warp_width is NULL");
  *warp_width = p->warp_width;
  return PROJ_OK;
}

int proj_set_brick_shape(proj_plan p, int shape) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (shape < 0 || shape >= kBrickShapes) return fail(PROJ_E_ARG, "brick shape %d is not in 0..%d", shape, kBrickShapes - 1);
  p->bp_shape = shape;
  return PROJ_OK;
}

int proj_get_brick_shape(proj_plan p, int* shape) {
  if (!p || !shape) return fail(PROJ_E_ARG, "plan or shape is NULL");
  *shape = p->bp_shape;
  return PROJ_OK;
}

int proj_autotune_back_grad(proj_plan p, const float* d_proj, const float* d_pose, int weight,
                            const float* d_vol_resid, void* d_ws, size_t ws_bytes, proj_stream stream, int reps,
                            float* times_ms, int* shape) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_proj || !d_pose || !d_vol_resid) return fail(PROJ_E_ARG, "proj_autotune_back_grad: NULL argument");
  if (weight != PROJ_W_NONE && weight != PROJ_W_FDK && weight != PROJ_W_FDK_CONST)
    return fail(PROJ_E_ARG, "unknown weight %d", weight);
  if (reps < 1 || reps > 1000) return fail(PROJ_E_ARG, "reps must be in 1..1000");
  int rc = need_op(p, PROJ_OP_BACK_GRAD, "proj_autotune_back_grad");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  cudaError_t e = launch_detector_prep(d_proj, p->n_inst, p->geo, w.det4, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = 0.f;
  int pick = p->bp_shape;
  for (int i = 0; i < kBrickShapes && e == cudaSuccess; ++i) {
    e = launch_back_grad(w.inst, p->n_inst, p->geo, weight, w.det4, d_vol_resid, w.part_b, i, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
      e = launch_back_grad(w.inst, p->n_inst, p->geo, weight, w.det4, d_vol_resid, w.part_b, i, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    ms /= (float)reps;
    if (times_ms) times_ms[i] = ms;
    if (e == cudaSuccess && (i == 0 || ms < best)) {
      best = ms;
      pick = i;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "brick-shape autotune launches");
  p->bp_shape = pick;
  if (shape) *shape = pick;
  return PROJ_OK;
}

int proj_autotune_forward_grad(proj_plan p, const float* d_pose, int loss, const float* d_ref, void* d_ws,
                               size_t ws_bytes, proj_stream stream, int reps, float* times_ms, int* warp_width) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_ref) return fail(PROJ_E_ARG, "proj_autotune_forward_grad: NULL pose or reference");
  if (loss != PROJ_LOSS_RESIDUAL && loss != PROJ_LOSS_L2 && loss != PROJ_LOSS_NCC)
    return fail(PROJ_E_ARG, "unknown loss mode %d", loss);
  if (reps < 1 || reps > 1000) return fail(PROJ_E_ARG, "reps must be in 1..1000");
  int rc = need_op(p, PROJ_OP_FORWARD_GRAD, "proj_autotune_forward_grad");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int widths[4] = {2, 4, 8, 16};
  float best = 0.f;
  int pick = p->warp_width;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    const Occ occ = occ_of(p, w);
    e = launch_forward_grad(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, loss, d_ref, nullptr, w.part_f, s,
                            widths[i], nullptr, occ, w.volb);
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r)
      e = launch_forward_grad(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, loss, d_ref, nullptr, w.part_f, s,
                              widths[i], nullptr, occ, w.volb);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    ms /= (float)reps;
    if (times_ms) times_ms[i] = ms;
    if (e == cudaSuccess && (i == 0 || ms < best)) {
      best = ms;
      pick = widths[i];
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "autotune launches");
  p->warp_width = pick;
  if (warp_width) *warp_width = pick;
  return PROJ_OK;
}

int proj_count_marched_samples(proj_plan p, const float* d_pose, long long* d_count, void* d_ws, size_t ws_bytes,
                               proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_count) return fail(PROJ_E_ARG, "proj_count_marched_samples: NULL pose or output");
  int rc = need_op(p, PROJ_OP_FORWARD_GRAD, "proj_count_marched_samples");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  // the fused march's samples: the gradient grid's box, clipped to the occupied bricks when skipping is on
  cudaError_t e = launch_count(w.inst, p->n_inst, p->geo, d_count, s, occ_of(p, w), 1);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "count launch");
}

int proj_set_skip_brick(proj_plan p, int edge) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (edge != 0 && edge != 8 && edge != 16) return fail(PROJ_E_ARG, "brick edge %d is not one of 0, 8, 16", edge);
  p->skip_shift = edge == 8 ? 3 : (edge == 16 ? 4 : 0);
  return PROJ_OK;
}

int proj_get_skip_brick(proj_plan p, int* edge) {
  if (!p || !edge) return fail(PROJ_E_ARG, "plan or edge is NULL");
  *edge = p->skip_shift ? 1 << p->skip_shift : 0;
  return PROJ_OK;
}

int proj_set_skip_cells(proj_plan p, int mode) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (mode < 0 || mode > 2) return fail(PROJ_E_ARG, "skip_cells mode must be 0, 1 or 2, got %d", mode);
  p->skip_cells = mode;
  return PROJ_OK;
}

int proj_get_skip_cells(proj_plan p, int* mode) {
  if (!p || !mode) return fail(PROJ_E_ARG, "plan or mode is NULL");
  *mode = p->skip_cells;
  return PROJ_OK;
}

int proj_autotune_march(proj_plan p, const float* d_pose, int loss, const float* d_ref, void* d_ws, size_t ws_bytes,
                        proj_stream stream, int reps, float* times_ms, int* warp_width, int* brick_edge,
                        int* skip_cells) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_pose || !d_ref) return fail(PROJ_E_ARG, "proj_autotune_march: NULL pose or reference");
  if (loss != PROJ_LOSS_RESIDUAL && loss != PROJ_LOSS_L2 && loss != PROJ_LOSS_NCC)
    return fail(PROJ_E_ARG, "unknown loss mode %d", loss);
  if (reps < 1 || reps > 1000) return fail(PROJ_E_ARG, "reps must be in 1..1000");
  int rc = need_op(p, PROJ_OP_FORWARD_GRAD, "proj_autotune_march");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = setup(p, d_pose, w, s))) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int widths[4] = {2, 4, 8, 16};
  const int shifts[3] = {0, 3, 4};
  float best = 0.f;
  int pick_w = p->warp_width, pick_s = p->skip_shift;
  int pick_c = p->skip_cells;
  bool have = false;
  // j = 2 * (brick edge position) + cell test
  for (int j = 0; j < 6 && e == cudaSuccess; ++j) {
    const Occ occ = occ_of(p, w, shifts[j >> 1], j & 1);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
      e = launch_forward_grad(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, loss, d_ref, nullptr, w.part_f, s,
                              widths[i], nullptr, occ, w.volb);
      if (e == cudaSuccess) e = cudaEventRecord(a, s);
      for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = launch_forward_grad(w.inst, p->n_inst, p->geo, w.vol4, w.vol4y, loss, d_ref, nullptr, w.part_f, s,
                                widths[i], nullptr, occ, w.volb);
      if (e == cudaSuccess) e = cudaEventRecord(b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      ms /= (float)reps;
      if (times_ms) times_ms[4 * j + i] = ms;
      if (e == cudaSuccess && (!have || ms < best)) {
        best = ms;
        pick_w = widths[i];
        pick_s = shifts[j >> 1];
        pick_c = j & 1;
        have = true;
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "autotune launches");
  p->warp_width = pick_w;
  p->skip_shift = pick_s;
  p->skip_cells = pick_c;
  if (warp_width) *warp_width = pick_w;
  if (brick_edge) *brick_edge = pick_s ? 1 << pick_s : 0;
  if (skip_cells) *skip_cells = pick_c;
  return PROJ_OK;
}

int proj_enable_kernel_timing(proj_plan p, int enable) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (enable && !p->ev0) {
    cudaError_t e = cudaEventCreate(&p->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
    if (e != cudaSuccess) return cuda_fail(e, "timing event creation");
  }
  p->timing = enable != 0;
  return PROJ_OK;
}

int proj_kernel_time_ms(proj_plan p, float* ms) {
  if (!p || !ms) return fail(PROJ_E_ARG, "plan or ms is NULL");
  if (!p->ev0) return fail(PROJ_E_UNSUPPORTED, "kernel timing was never enabled");
  cudaError_t e = cudaEventSynchronize(p->ev1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, p->ev0, p->ev1);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "kernel timing");
}

int proj_fdk_filter(proj_plan p, const float* d_proj, float scale, float* d_out, proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_proj || !d_out) return fail(PROJ_E_ARG, "proj_fdk_filter: NULL argument");
  if (d_proj == d_out) return fail(PROJ_E_ARG, "proj_fdk_filter: input and output must differ");
  if (!std::isfinite(scale)) return fail(PROJ_E_ARG, "proj_fdk_filter: scale must be finite");
  if ((size_t)p->geo.nu * sizeof(float) > 200 * 1024) return fail(PROJ_E_UNSUPPORTED, "detector rows too long");
  int rc = check_device(p);
  if (rc) return rc;
  cudaError_t e = launch_fdk_filter(p->d_fdk, p->n_inst, p->geo, scale, d_proj, d_out, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "FDK filter launch");
}

int proj_sharpness(proj_plan p, const float* d_vol, float* d_loss, float* d_grad, void* d_ws, size_t ws_bytes,
                   proj_stream stream) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  if (!d_vol || !d_loss) return fail(PROJ_E_ARG, "proj_sharpness: NULL volume or loss");
  int rc = need_op(p, PROJ_OP_SHARPNESS, "proj_sharpness");
  if (rc) return rc;
  WsView w;
  if ((rc = check_ws(p, d_ws, ws_bytes, &w))) return rc;
  if ((rc = check_device(p))) return rc;
  char* b = static_cast<char*>(d_ws);
  float* m = reinterpret_cast<float*>(b + p->off_sharp_m);
  double* part = reinterpret_cast<double*>(b + p->off_sharp_part);
  double* stats = part + 2 * (size_t)sharpness_blocks(p->geo);
  cudaError_t e = launch_sharpness(d_vol, p->geo, m, part, stats, d_loss, d_grad, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "sharpness launch");
}

int proj_pose_adam(float* d_pose, const float* d_grad, float* d_m, float* d_v, float* d_t,
                   const unsigned char* d_active, int n, const float* lr, float b1, float b2, float eps,
                   proj_stream stream) {
  if (n < 0) return fail(PROJ_E_ARG, "proj_pose_adam: n = %d", n);
  if (n == 0) return PROJ_OK;
  if (!d_pose || !d_grad || !d_m || !d_v || !d_t || !lr) return fail(PROJ_E_ARG, "proj_pose_adam: NULL argument");
  if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps >= 0.f))
    return fail(PROJ_E_ARG, "proj_pose_adam: need 0 <= b1, b2 < 1 and eps >= 0");
  PoseAdam h;
  for (int j = 0; j < 6; ++j) h.lr[j] = lr[j];
  h.b1 = b1;
  h.a1 = (float)(1.0 - (double)b1);
  h.b2 = b2;
  h.a2 = (float)(1.0 - (double)b2);
  h.eps = eps;
  cudaError_t e = launch_pose_adam(d_pose, d_grad, d_m, d_v, d_t, d_active, n, h, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "pose Adam launch");
}

int proj_registration_step(int n, int n_slots, float* d_pose, const float* d_grad, const float* d_loss, float* d_last,
                           float* d_m, float* d_v, float* d_t, unsigned char* d_alive, long long* d_iters,
                           int* d_slots, long long* d_next, const float* d_truth, int n_truth,
                           unsigned char* d_hit_any, unsigned char* d_listed, const proj_reg_params* prm,
                           proj_stream stream) {
  if (n < 0 || n_slots < 0) return fail(PROJ_E_ARG, "proj_registration_step: n = %d, n_slots = %d", n, n_slots);
  if (n == 0 || n_slots == 0) return PROJ_OK;
  if (!d_pose || !d_grad || !d_loss || !d_last || !d_m || !d_v || !d_t || !d_alive || !d_iters || !d_slots ||
      !d_next || !d_listed || !prm)
    return fail(PROJ_E_ARG, "proj_registration_step: NULL argument");
  if (d_truth && (n_truth != 1 && n_truth != n))
    return fail(PROJ_E_ARG, "proj_registration_step: n_truth = %d must be 1 or n = %d", n_truth, n);
  if (d_truth && !d_hit_any) return fail(PROJ_E_ARG, "proj_registration_step: a truth needs d_hit_any");
  if (!(prm->b1 >= 0.f && prm->b1 < 1.f && prm->b2 >= 0.f && prm->b2 < 1.f && prm->eps >= 0.f))
    return fail(PROJ_E_ARG, "proj_registration_step: need 0 <= b1, b2 < 1 and eps >= 0");
  RegStep r;
  r.n = n;
  r.n_slots = n_slots;
  r.pose = d_pose;
  r.grad = d_grad;
  r.loss = d_loss;
  r.last = d_last;
  r.m = d_m;
  r.v = d_v;
  r.t = d_t;
  r.alive = d_alive;
  r.iters = d_iters;
  r.slots = d_slots;
  r.next = d_next;
  r.truth = d_truth;
  r.n_truth = n_truth;
  r.hit_any = d_hit_any;
  r.listed = d_listed;
  r.ncc_stop = prm->ncc_stop;
  r.dloss_stop = prm->dloss_stop;
  r.tol_mm = prm->tol_mm;
  r.tol_deg = prm->tol_deg;
  r.max_iter = prm->max_iter;
  for (int j = 0; j < 6; ++j) r.adam.lr[j] = prm->lr[j];
  r.adam.b1 = prm->b1;
  r.adam.a1 = (float)(1.0 - (double)prm->b1);
  r.adam.b2 = prm->b2;
  r.adam.a2 = (float)(1.0 - (double)prm->b2);
  r.adam.eps = prm->eps;
  cudaError_t e = launch_registration_step(r, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "registration step launch");
}

}  // extern "C"

struct proj_batch_s {
  int n = 0;
  int device = -1;
  long long n_items = 0;
  int n_blocks = 0;
  std::vector<proj_plan> plans;
  std::vector<int> loss;
  std::vector<const float*> pose;
  std::vector<float*> grad, loss_out;
  std::vector<void*> ws;
  std::vector<size_t> ws_bytes;
  BatchProblem* d_probs = nullptr;
  unsigned long long* d_counter = nullptr;
  int loss_all = -1;  // the loss every problem shares, or -1
};

extern "C" {

int proj_batch_create(int n, const proj_plan* plans, const int* loss, const float* const* d_pose,
                      const float* const* d_ref, float* const* d_grad, float* const* d_loss, void* const* d_ws,
                      const size_t* ws_bytes, proj_batch* out) {
  g_last_error.clear();
  if (!out) return fail(PROJ_E_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !plans || !loss || !d_pose || !d_ref || !d_grad || !d_ws || !ws_bytes)
    return fail(PROJ_E_ARG, "proj_batch_create: need n >= 1 and all per-problem arrays");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::vector<BatchProblem> probs(n);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    const proj_plan p = plans[i];
    if (!p) return fail(PROJ_E_ARG, "problem %d: plan is NULL", i);
    if (!(p->ops & PROJ_OP_FORWARD_GRAD))
      return fail(PROJ_E_UNSUPPORTED, "problem %d: plan lacks PROJ_OP_FORWARD_GRAD", i);
    if (p->device != dev) return fail(PROJ_E_ARG, "problem %d: plan is on device %d, current is %d", i, p->device, dev);
    if (loss[i] != PROJ_LOSS_RESIDUAL && loss[i] != PROJ_LOSS_L2 && loss[i] != PROJ_LOSS_NCC)
      return fail(PROJ_E_ARG, "problem %d: unknown loss %d", i, loss[i]);
    if (!d_pose[i] || !d_ref[i] || !d_grad[i]) return fail(PROJ_E_ARG, "problem %d: NULL pose, reference or grad", i);
    WsView w;
    int rc = check_ws(p, d_ws[i], ws_bytes[i], &w);
    if (rc) return fail(rc, "problem %d: %s", i, g_last_error.c_str());
    for (int j = 0; j < i; ++j)
      if (d_ws[j] == d_ws[i]) return fail(PROJ_E_ARG, "problems %d and %d share a workspace", j, i);
    BatchProblem& B = probs[i];
    B.geo = p->geo;
    B.inst = w.inst;
    B.vol4 = w.vol4;
    B.vol4y = w.vol4y;
    B.occ = occ_of(p, w);
    B.ref = d_ref[i];
    B.part = w.part_f;
    B.n_tiles = p->n_tiles;
    B.tiles_u = ceil_div(p->geo.nu, kTileU);
    B.loss = loss[i];
    B.n_inst = p->n_inst;
    // per-tile cost ~ samples per ray ~ volume diagonal / step
    const double dx = p->geo.nx * (double)p->geo.vx, dy = p->geo.ny * (double)p->geo.vy,
                 dz = p->geo.nz * (double)p->geo.vz;
    cost[i] = std::sqrt(dx * dx + dy * dy + dz * dz) / p->geo.step;
  }
  // longest tiles first
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  proj_batch_s* b = new proj_batch_s();
  b->n = n;
  b->device = dev;
  std::vector<BatchProblem> sorted(n);
  long long items = 0;
  for (int k = 0; k < n; ++k) {
    const int i = order[k];
    sorted[k] = probs[i];
    sorted[k].item_begin = items;
    items += (long long)plans[i]->n_inst * plans[i]->n_tiles;
    b->plans.push_back(plans[i]);
    b->loss.push_back(loss[i]);
    b->pose.push_back(d_pose[i]);
    b->grad.push_back(d_grad[i]);
    b->loss_out.push_back(d_loss ? d_loss[i] : nullptr);
    b->ws.push_back(d_ws[i]);
    b->ws_bytes.push_back(ws_bytes[i]);
  }
  b->n_items = items;
  b->loss_all = loss[0];
  for (int i = 1; i < n; ++i)
    if (loss[i] != loss[0]) b->loss_all = -1;
  int n_sm = 148;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const long long cap = (long long)n_sm * forward_grad_batch_blocks_per_sm(b->loss_all);
  b->n_blocks = (int)(items < cap ? items : cap);
  e = cudaMalloc(&b->d_probs, sizeof(BatchProblem) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_probs, sorted.data(), sizeof(BatchProblem) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    proj_batch_destroy(b);
    return cuda_fail(e, "batch table allocation");
  }
  *out = b;
  return PROJ_OK;
}

int proj_batch_destroy(proj_batch b) {
  if (!b) return PROJ_OK;
  cudaFree(b->d_probs);
  cudaFree(b->d_counter);
  delete b;
  return PROJ_OK;
}

int proj_batch_run(proj_batch b, proj_stream stream) {
  if (!b) return fail(PROJ_E_ARG, "batch is NULL");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != b->device) return fail(PROJ_E_ARG, "current device %d differs from the batch's device %d", dev, b->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<WsView> w(b->n);
  for (int k = 0; k < b->n; ++k) {
    int rc = check_ws(b->plans[k], b->ws[k], b->ws_bytes[k], &w[k]);
    if (rc) return rc;
    if ((rc = setup(b->plans[k], b->pose[k], w[k], s))) return rc;
  }
  e = launch_forward_grad_batch(b->d_probs, b->n, b->n_items, b->d_counter, b->n_blocks, b->loss_all, s);
  if (e != cudaSuccess) return cuda_fail(e, "batched pose-gradient launch");
  for (int k = 0; k < b->n; ++k) {
    const proj_plan p = b->plans[k];
    e = launch_forward_grad_reduce(w[k].inst, w[k].ptab, p->n_pose, p->d_pose_ptr, p->d_pose_idx,
                                   p->n_tiles, p->geo, b->loss[k], w[k].part_f, b->grad[k],
                                   b->loss_out[k], s);
    if (e != cudaSuccess) return cuda_fail(e, "batched reduction launch");
  }
  return PROJ_OK;
}

int proj_check(proj_plan p, void* d_ws, size_t ws_bytes, proj_stream stream, int* status) {
  if (!p) return fail(PROJ_E_ARG, "plan is NULL");
  WsView w;
  int rc = check_ws(p, d_ws, ws_bytes, &w);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, w.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.status, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (status) *status = h;
  if (h) return fail(PROJ_E_DEVICE, "device status bits 0x%x", h);
  return PROJ_OK;
}

}  // extern "C"
