/* A C program (no Python, no torch) against the C ABI of libproj.so:
 * the headers compile as C, the library links, and calls that must fail on
 * the host fail with the documented codes and a message.  Needs no GPU. */
#include <stdio.h>
#include <string.h>

#include "posenet.h"
#include "proj.h"

static int fails = 0;

static void expect(int cond, const char *what) {
  if (!cond) {
    printf("FAILED: %s\n", what);
    ++fails;
  }
}

int main(void) {
  const char *v = proj_version();
  expect(v != NULL && strstr(v, "sm_103a") != NULL, "proj_version names sm_103a");

  proj_plan plan = NULL;
  expect(proj_plan_create(NULL, 1, 1, NULL, NULL, PROJ_OP_ALL, &plan) == PROJ_E_ARG, "NULL geometry");
  expect(plan == NULL, "no plan on failure");
  expect(proj_last_error()[0] != '\0', "error message set");

  /* a valid-looking geometry with a zero ray step is rejected before any CUDA call */
  double views[12] = {800, 0, 0, -400, 0, 0, 0, 1, 0, 0, 0, 1};
  int iv = 0, ip = 0;
  proj_geometry g;
  memset(&g, 0, sizeof(g));
  g.nx = g.ny = g.nz = 8;
  g.vx = g.vy = g.vz = 1.0;
  g.nu = g.nv = 16;
  g.n_views = 1;
  g.views = views;
  g.step = 0.0;
  expect(proj_plan_create(&g, 1, 1, &iv, &ip, PROJ_OP_ALL, &plan) == PROJ_E_ARG, "zero step");
  expect(strstr(proj_last_error(), "step") != NULL, "message names the step");
  g.step = 0.5;
  iv = 3;
  expect(proj_plan_create(&g, 1, 1, &iv, &ip, PROJ_OP_ALL, &plan) == PROJ_E_ARG, "view index out of range");

  size_t n = 0;
  expect(proj_workspace_size(NULL, &n) == PROJ_E_ARG, "workspace size of NULL plan");
  expect(proj_forward(NULL, NULL, NULL, NULL, 0, NULL) == PROJ_E_ARG, "forward on NULL plan");
  expect(proj_batch_run(NULL, NULL) == PROJ_E_ARG, "batch run of NULL batch");
  expect(proj_plan_destroy(NULL) == PROJ_OK, "destroying NULL is a no-op");

  expect(pn_gemm_bf16(0, 8, 8, NULL, 8, NULL, 8, NULL, NULL, 0, 0, NULL, NULL, 8, 1, NULL, NULL) == PROJ_E_ARG,
         "empty GEMM");
  expect(pn_transpose_bf16(NULL, 1, 1, NULL, 1, NULL) == PROJ_E_ARG, "transpose of NULL");
  expect(pn_mse_loss(NULL, 1, 6, 8, NULL, NULL, NULL, 8, NULL) == PROJ_E_ARG, "loss of NULL");
  expect(pn_colsum_scratch_floats(0, 4) == 0, "scratch size of an empty matrix");

  printf(fails ? "%d failures\n" : "ok\n", fails);
  return fails != 0;
}
