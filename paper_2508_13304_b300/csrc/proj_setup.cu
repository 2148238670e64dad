// Pose set-up kernel: theta -> R, t, dR/dgamma (Table I) and, per (view,
// pose) instance, the FP32 tables the march and back-projection kernels
// read.  Runs in FP64 once per call; one thread per pose / instance.
#include "proj_internal.cuh"

namespace projk {

namespace {

__device__ void mul3(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// R = Rz(gz) Ry(gy) Rx(gx) and its derivatives in the three angles.
__device__ bool pose_matrices(const float* th, double* R, double* dR, double* t) {
  bool ok = true;
  double p[6];
  for (int a = 0; a < 6; ++a) {
    p[a] = (double)th[a];
    ok = ok && isfinite(p[a]);
  }
  if (!ok) {
    for (int a = 0; a < 9; ++a) R[a] = (a % 4 == 0) ? 1.0 : 0.0;
    for (int a = 0; a < 27; ++a) dR[a] = 0.0;
    t[0] = t[1] = t[2] = 0.0;
    return false;
  }
  double sx, cx, sy, cy, sz, cz;
  sincos(p[3], &sx, &cx);
  sincos(p[4], &sy, &cy);
  sincos(p[5], &sz, &cz);
  const double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  const double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  const double dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
  const double dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
  const double dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
  double YX[9], T[9];
  mul3(Ry, Rx, YX);
  mul3(Rz, YX, R);
  mul3(Ry, dRx, T);
  mul3(Rz, T, dR);
  mul3(dRy, Rx, T);
  mul3(Rz, T, dR + 9);
  mul3(dRz, YX, dR + 18);
  t[0] = p[0];
  t[1] = p[1];
  t[2] = p[2];
  return true;
}

__global__ void k_setup(const float* __restrict__ pose, int n_pose, const double* __restrict__ views,
                        const int* __restrict__ inst_view, const int* __restrict__ inst_pose, int n_inst, Geo g,
                        InstTable* __restrict__ inst, PoseTable* __restrict__ ptab, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pose) {
    PoseTable pt;
    pt.valid = pose_matrices(pose + 6 * i, pt.R, pt.dR, pt.t) ? 1 : 0;
    pt.pad = 0;
    ptab[i] = pt;
    if (!pt.valid) atomicOr(status, PROJ_STATUS_BAD_POSE);
  }
  if (i >= n_inst) return;

  double R[9], dR[27], t[3];
  const int p = inst_pose[i], v = inst_view[i];
  const bool valid = pose_matrices(pose + 6 * p, R, dR, t);
  const double* vw = views + 12 * v;
  const double s[3] = {vw[0], vw[1], vw[2]};
  const double U[3] = {vw[6], vw[7], vw[8]};
  const double V[3] = {vw[9], vw[10], vw[11]};
  double q00[3];
  for (int a = 0; a < 3; ++a) q00[a] = vw[3 + a] - 0.5 * (g.nu - 1) * U[a] - 0.5 * (g.nv - 1) * V[a];
  const double off[3] = {g.offx, g.offy, g.offz};
  const double vox[3] = {g.vx, g.vy, g.vz};

  InstTable T;
  // Ray-driven part: source in centred object index coordinates, pixel
  // direction basis rotated into the object frame (R^T x).
  for (int b = 0; b < 3; ++b) {
    double sp = 0, c0 = 0, uo = 0, vo = 0;
    for (int a = 0; a < 3; ++a) {
      sp += R[3 * a + b] * (s[a] - t[a]);
      c0 += R[3 * a + b] * (q00[a] - s[a]);
      uo += R[3 * a + b] * U[a];
      vo += R[3 * a + b] * V[a];
    }
    T.A[b] = (float)((sp - off[b]) / vox[b]);
    T.C0[b] = (float)c0;
    T.Uo[b] = (float)uo;
    T.Vo[b] = (float)vo;
  }
  // Projection matrix P = [B^-1 | -B^-1 s], B = [U | V | q00 - s] (Eq.
  // projmatrix), then Q = P [R | t] applied to r' = off + f~ * vox.
  double B[9];
  for (int a = 0; a < 3; ++a) {
    B[3 * a + 0] = U[a];
    B[3 * a + 1] = V[a];
    B[3 * a + 2] = q00[a] - s[a];
  }
  const double det = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                     B[2] * (B[3] * B[7] - B[4] * B[6]);
  const double id = 1.0 / det;
  const double Bi[9] = {(B[4] * B[8] - B[5] * B[7]) * id, (B[2] * B[7] - B[1] * B[8]) * id,
                        (B[1] * B[5] - B[2] * B[4]) * id, (B[5] * B[6] - B[3] * B[8]) * id,
                        (B[0] * B[8] - B[2] * B[6]) * id, (B[2] * B[3] - B[0] * B[5]) * id,
                        (B[3] * B[7] - B[4] * B[6]) * id, (B[1] * B[6] - B[0] * B[7]) * id,
                        (B[0] * B[4] - B[1] * B[3]) * id};
  double P4[3];
  for (int a = 0; a < 3; ++a) P4[a] = -(Bi[3 * a] * s[0] + Bi[3 * a + 1] * s[1] + Bi[3 * a + 2] * s[2]);
  double PR[9];
  mul3(Bi, R, PR);
  double Roff_t[3];
  for (int a = 0; a < 3; ++a) Roff_t[a] = R[3 * a] * off[0] + R[3 * a + 1] * off[1] + R[3 * a + 2] * off[2] + t[a];
  for (int col = 0; col < 3; ++col)
    for (int row = 0; row < 3; ++row) T.Q[3 * col + row] = (float)(PR[3 * row + col] * vox[col]);
  for (int row = 0; row < 3; ++row)
    T.Q[9 + row] = (float)(Bi[3 * row] * Roff_t[0] + Bi[3 * row + 1] * Roff_t[1] + Bi[3 * row + 2] * Roff_t[2] +
                           P4[row]);
  for (int a = 0; a < 9; ++a) T.P3[a] = (float)Bi[a];
  T.w0 = (float)P4[2];
  T.view = v;
  T.pose = p;
  T.valid = valid ? 1 : 0;
  // neighbouring pixels along u are neighbouring rays: march the copy of the
  // volume whose rows run along the index axis (x or y) closest to u
  T.yfast = fabs(T.Uo[1] / vox[1]) > fabs(T.Uo[0] / vox[0]) ? 1 : 0;
  T.pad[0] = T.pad[1] = 0;
  inst[i] = T;
}

}  // namespace

cudaError_t launch_setup(const float* d_pose, int n_pose, const double* d_views, const int* d_inst_view,
                         const int* d_inst_pose, int n_inst, Geo geo, InstTable* d_inst, PoseTable* d_ptab,
                         int* d_status, cudaStream_t s) {
  // one thread per instance runs a long dependent chain of FP64 operations (FP64 runs at a small
  // fraction of the FP32 rate here): blocks of 8 threads spread the instances over many SMs
  constexpr int kSetupThreads = 8;
  const int n = n_pose > n_inst ? n_pose : n_inst;
  k_setup<<<ceil_div(n, kSetupThreads), kSetupThreads, 0, s>>>(d_pose, n_pose, d_views, d_inst_view, d_inst_pose,
                                                               n_inst, geo, d_inst, d_ptab, d_status);
  return cudaGetLastError();
}

}  // namespace projk
