/* A C program (no Python, no torch) that runs the projector through the C
 * ABI on the GPU: plan, caller-owned workspace, volume, forward projection,
 * fused L2 pose gradient.  Checks, with the CUDA runtime only:
 *   - the fused loss equals sum (l - b)^2 formed on the host from
 *     proj_forward's output (same rays, same FP32 march);
 *   - dL/dtx and dL/dgz match central differences of that loss;
 *   - the status word is clear.
 * Prints "abi_gpu ok" and returns 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "proj.h"

#define CK(x)                                                            \
  do {                                                                   \
    int rc_ = (x);                                                       \
    if (rc_ != 0) {                                                      \
      printf("FAILED: %s -> %d (%s)\n", #x, rc_, proj_last_error());     \
      return 1;                                                          \
    }                                                                    \
  } while (0)

#define CU(x)                                                            \
  do {                                                                   \
    cudaError_t e_ = (x);                                                \
    if (e_ != cudaSuccess) {                                             \
      printf("FAILED: %s -> %s\n", #x, cudaGetErrorString(e_));          \
      return 1;                                                          \
    }                                                                    \
  } while (0)

enum { NX = 40, NY = 36, NZ = 32, NU = 48, NV = 40, NVIEW = 2 };

/* proj_forward at pose_h into out_h (host); 0 on success */
static int project(proj_plan plan, const float *pose_h, float *d_pose, float *d_proj, float *out_h, void *d_ws,
                   size_t ws_bytes) {
  if (cudaMemcpy(d_pose, pose_h, 6 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return 1;
  if (proj_forward(plan, d_pose, d_proj, d_ws, ws_bytes, NULL) != PROJ_OK) return 1;
  return cudaMemcpy(out_h, d_proj, sizeof(float) * NVIEW * NU * NV, cudaMemcpyDeviceToHost) != cudaSuccess;
}

/* sum (l - b)^2 over both views, l = proj_forward at pose_h, in FP64 on the host */
static double loss_of(proj_plan plan, const float *pose_h, float *d_pose, float *d_proj, const float *target,
                      float *proj_h, void *d_ws, size_t ws_bytes) {
  if (project(plan, pose_h, d_pose, d_proj, proj_h, d_ws, ws_bytes)) return NAN;
  double L = 0.0;
  for (int i = 0; i < NVIEW * NU * NV; ++i) {
    const double d = (double)proj_h[i] - (double)target[i];
    L += d * d;
  }
  return L;
}

int main(void) {
  /* two views of a circular orbit, 1 mm voxels, 1.6 mm pixels */
  double views[12 * NVIEW];
  for (int v = 0; v < NVIEW; ++v) {
    const double b = 1.3 * v, c = cos(b), s = sin(b), sad = 200.0, sdd = 320.0, du = 1.6;
    double *w = views + 12 * v;
    w[0] = sad * c, w[1] = sad * s, w[2] = 0.0;
    w[3] = -(sdd - sad) * c, w[4] = -(sdd - sad) * s, w[5] = 0.0;
    w[6] = -du * s, w[7] = du * c, w[8] = 0.0;
    w[9] = 0.0, w[10] = 0.0, w[11] = du;
  }
  proj_geometry geo = {0};
  geo.nx = NX, geo.ny = NY, geo.nz = NZ;
  geo.vx = geo.vy = geo.vz = 1.0;
  geo.nu = NU, geo.nv = NV, geo.n_views = NVIEW;
  geo.views = views;
  geo.step = 0.5;
  int iv[NVIEW] = {0, 1}, ip[NVIEW] = {0, 0};
  proj_plan plan = NULL;
  CK(proj_plan_create(&geo, 1, NVIEW, iv, ip, PROJ_OP_FORWARD | PROJ_OP_FORWARD_GRAD, &plan));
  size_t ws_bytes = 0;
  CK(proj_workspace_size(plan, &ws_bytes));
  void *d_ws = NULL;
  CU(cudaMalloc(&d_ws, ws_bytes));
  CU(cudaMemset(d_ws, 0, ws_bytes));

  /* a smooth blob volume */
  float *mu_h = (float *)malloc(sizeof(float) * NX * NY * NZ);
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const double x = i - 0.5 * (NX - 1) - 3.0, y = j - 0.5 * (NY - 1) + 2.0, z = k - 0.5 * (NZ - 1);
        mu_h[(k * NY + j) * NX + i] = (float)(0.02 * exp(-(x * x + 0.7 * y * y + 1.3 * z * z) / 60.0));
      }
  float *d_mu = NULL, *d_pose = NULL, *d_proj = NULL, *d_ref = NULL, *d_grad = NULL, *d_loss = NULL;
  CU(cudaMalloc((void **)&d_mu, sizeof(float) * NX * NY * NZ));
  CU(cudaMalloc((void **)&d_pose, 6 * sizeof(float)));
  CU(cudaMalloc((void **)&d_proj, sizeof(float) * NVIEW * NU * NV));
  CU(cudaMalloc((void **)&d_ref, sizeof(float) * NVIEW * NU * NV));
  CU(cudaMalloc((void **)&d_grad, 6 * sizeof(float)));
  CU(cudaMalloc((void **)&d_loss, sizeof(float)));
  CU(cudaMemcpy(d_mu, mu_h, sizeof(float) * NX * NY * NZ, cudaMemcpyHostToDevice));
  CK(proj_set_volume(plan, d_mu, d_ws, ws_bytes, NULL));

  /* target: projections at a reference pose */
  float *target = (float *)malloc(sizeof(float) * NVIEW * NU * NV);
  float *proj_h = (float *)malloc(sizeof(float) * NVIEW * NU * NV);
  const float pose_t[6] = {1.0f, -0.5f, 0.3f, 0.04f, -0.03f, 0.05f};
  if (project(plan, pose_t, d_pose, d_proj, target, d_ws, ws_bytes)) {
    printf("FAILED: target projection (%s)\n", proj_last_error());
    return 1;
  }
  CU(cudaMemcpy(d_ref, target, sizeof(float) * NVIEW * NU * NV, cudaMemcpyHostToDevice));

  /* fused loss and gradient at another pose */
  float pose[6] = {0.2f, 0.4f, -0.6f, -0.02f, 0.03f, -0.04f};
  CU(cudaMemcpy(d_pose, pose, 6 * sizeof(float), cudaMemcpyHostToDevice));
  CK(proj_forward_pose_grad(plan, d_pose, PROJ_LOSS_L2, d_ref, d_grad, d_loss, NULL, d_ws, ws_bytes, NULL));
  float grad[6], loss = 0.f;
  CU(cudaMemcpy(grad, d_grad, sizeof(grad), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(&loss, d_loss, sizeof(float), cudaMemcpyDeviceToHost));
  const double L0 = loss_of(plan, pose, d_pose, d_proj, target, proj_h, d_ws, ws_bytes);
  int fails = 0;
  if (!(fabs(loss - L0) <= 1e-4 * L0)) {
    printf("FAILED: fused loss %g vs host sum of squares %g\n", loss, L0);
    ++fails;
  }
  /* central differences of the loss in tx (mm) and gz (rad) */
  const int comp[2] = {0, 5};
  const float h[2] = {0.05f, 5e-4f};
  for (int c = 0; c < 2; ++c) {
    float pp[6], pm[6];
    for (int a = 0; a < 6; ++a) pp[a] = pm[a] = pose[a];
    pp[comp[c]] += h[c];
    pm[comp[c]] -= h[c];
    const double fd = (loss_of(plan, pp, d_pose, d_proj, target, proj_h, d_ws, ws_bytes) -
                       loss_of(plan, pm, d_pose, d_proj, target, proj_h, d_ws, ws_bytes)) /
                      (double)(pp[comp[c]] - pm[comp[c]]);
    if (!(fabs(grad[comp[c]] - fd) <= 0.02 * fabs(fd) + 1e-9)) {
      printf("FAILED: dL/dtheta[%d] = %g vs central difference %g\n", comp[c], grad[comp[c]], fd);
      ++fails;
    }
  }
  int status = -1;
  CK(proj_check(plan, d_ws, ws_bytes, NULL, &status));
  if (status != 0) {
    printf("FAILED: status word %d\n", status);
    ++fails;
  }
  CK(proj_plan_destroy(plan));
  cudaFree(d_ws);
  cudaFree(d_mu);
  cudaFree(d_pose);
  cudaFree(d_proj);
  cudaFree(d_ref);
  cudaFree(d_grad);
  cudaFree(d_loss);
  free(mu_h);
  free(target);
  free(proj_h);
  if (fails) return 1;
  printf("abi_gpu ok\n");
  return 0;
}
