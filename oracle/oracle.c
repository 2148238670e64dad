/*
 * FP64 CPU oracle for the cone-beam projector pair and its rigid-pose
 * gradients.  TEST INFRASTRUCTURE ONLY: it is called by the tests, by
 * __graft_entry__.smoke() and by the benchmark's CPU-baseline leg, never by
 * the product path.  It shares no code, header or table with the CUDA
 * library.  It is written for readability, not speed: every quantity is
 * recomputed from its definition where it is used.
 *
 * Notation follows the paper (Table I): pose theta = (tx,ty,tz,gx,gy,gz),
 * M = [R | t], r = R r' + t, r' = R^T (r - t); projection matrix P (Eq.
 * projmatrix) maps a world point to (u', v', w') and d = (u'/w', v'/w').
 *
 * Readings of points the paper leaves open (also listed in the design notes):
 *  - R = Rz(gz) Ry(gy) Rx(gx), right-handed, angles in rad.
 *  - Forward model (Eq. forward, discretised as in Sec. II-C.1): a ray-driven
 *    march with trilinear interpolation and zero padding,
 *        l_i = step * sum_{k in K_i} mu~(r'_k),  r_k = s + k*step*e_i,
 *    where K_i holds every integer k >= 0 whose object-frame index
 *    coordinate lies in the open box (-1, n)^3 (mu~ vanishes on its faces).
 *  - Forward pose gradient (Eq. final_forward / for_int / dis_forward):
 *    G_f evaluated at every integration point; grad mu = trilinear
 *    interpolation of the central-difference grid of the zero-padded volume,
 *    defined on the extended index grid [-1, n]^3 (mode OR_GRAD_ANALYTIC),
 *    or the exact derivative of mu~ (mode OR_GRAD_EXACT); mode
 *    OR_GRAD_VOXEL_CENTRE reads the paper's three-step recipe literally and
 *    interpolates G = grad mu (x) (r - t) formed at voxel centres (reported,
 *    not graded: it differs from the graded reading at second order).  Each channel of
 *    G_f is projected by the same ray march over the support of its own
 *    interpolant: the open box (-2, n+1)^3 for the analytic gradient grid
 *    (mu~ itself is zero outside (-1, n)^3), which keeps the gradient
 *    continuous in the pose.
 *  - Back-projection (Eq. back, discretised as in Sec. II-C.2): voxel-driven
 *        mu_j = sum_inst W(r_j) * l~(p(R r'_j + t)),
 *    l~ bilinear with zero padding in pixel-index units; voxels with w' <= 0
 *    (behind the source) receive nothing.  W = 1, or the FDK distance weight
 *    W = (w'(0) / w'(r))^2 with w'(0) the value at the world origin.
 *  - Back-projection pose gradient (Eq. back_derive / final_back / back_int
 *    / dis_back): grad_d l = bilinear interpolation of central-difference
 *    detector images on the extended grid [-1,nu] x [-1,nv] with zero
 *    padding (analytic; its interpolant lives on (-2,nu+1) x (-2,nv+1)) or
 *    the exact derivative of l~ (exact); the FDK weight contributes
 *    l~ * grad W unless the paper-literal constant-weight variant is
 *    requested.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int nx, ny, nz;
  double vx, vy, vz;
  double off[3];
  int nu, nv;
  int n_views;
  const double *views; /* [n_views][12]: s, c, U, V */
  double step;
} or_geom;

enum { OR_GRAD_ANALYTIC = 0, OR_GRAD_EXACT = 1, OR_GRAD_VOXEL_CENTRE = 2 };
enum { OR_W_NONE = 0, OR_W_FDK = 1, OR_W_FDK_CONST = 2 };

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- matrices */

static void mat3_mul(const double A[9], const double B[9], double C[9]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}

/* Rotation R = Rz Ry Rx and its three partial derivatives dR/dg_j
 * (Table I: R(gamma)). */
void or_rotation(const double th[6], double R[9], double dR[27]) {
  double cx = cos(th[3]), sx = sin(th[3]);
  double cy = cos(th[4]), sy = sin(th[4]);
  double cz = cos(th[5]), sz = sin(th[5]);
  double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
  double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
  double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
  double dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
  double dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
  double dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
  double T[9];
  mat3_mul(Ry, Rx, T);
  mat3_mul(Rz, T, R);
  if (dR) {
    double U[9];
    mat3_mul(Ry, dRx, U);
    mat3_mul(Rz, U, dR + 0);
    mat3_mul(dRy, Rx, U);
    mat3_mul(Rz, U, dR + 9);
    mat3_mul(dRz, T, dR + 18);
  }
}

/* Projection matrix P (3x4, row major) of one view in pixel-index units
 * (Eq. projmatrix).  With B = [U | V | q00 - s] (columns; q00 = centre of
 * pixel (0,0)), a point r on the ray from s through pixel (iu, iv) satisfies
 * B^{-1} (r - s) = lambda (iu, iv, 1), so P = [B^{-1} | -B^{-1} s].
 * Returns 0, or -1 when B is singular. */
int or_projection_matrix(const double view[12], int nu, int nv, double P[12]) {
  const double *s = view, *c = view + 3, *U = view + 6, *V = view + 9;
  double q00[3], B[9], Bi[9];
  for (int a = 0; a < 3; ++a)
    q00[a] = c[a] - 0.5 * (nu - 1) * U[a] - 0.5 * (nv - 1) * V[a];
  for (int a = 0; a < 3; ++a) {
    B[3 * a + 0] = U[a];
    B[3 * a + 1] = V[a];
    B[3 * a + 2] = q00[a] - s[a];
  }
  /* inverse by cofactors */
  double det = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
               B[2] * (B[3] * B[7] - B[4] * B[6]);
  if (det == 0.0 || !isfinite(det)) return -1;
  Bi[0] = (B[4] * B[8] - B[5] * B[7]) / det;
  Bi[1] = (B[2] * B[7] - B[1] * B[8]) / det;
  Bi[2] = (B[1] * B[5] - B[2] * B[4]) / det;
  Bi[3] = (B[5] * B[6] - B[3] * B[8]) / det;
  Bi[4] = (B[0] * B[8] - B[2] * B[6]) / det;
  Bi[5] = (B[2] * B[3] - B[0] * B[5]) / det;
  Bi[6] = (B[3] * B[7] - B[4] * B[6]) / det;
  Bi[7] = (B[1] * B[6] - B[0] * B[7]) / det;
  Bi[8] = (B[0] * B[4] - B[1] * B[3]) / det;
  for (int a = 0; a < 3; ++a) {
    P[4 * a + 0] = Bi[3 * a + 0];
    P[4 * a + 1] = Bi[3 * a + 1];
    P[4 * a + 2] = Bi[3 * a + 2];
    P[4 * a + 3] = -(Bi[3 * a + 0] * s[0] + Bi[3 * a + 1] * s[1] + Bi[3 * a + 2] * s[2]);
  }
  return 0;
}

/* ------------------------------------------------------------ volume access */

static double vox(const double *mu, const or_geom *g, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz) return 0.0;
  return mu[((size_t)k * g->ny + j) * g->nx + i];
}

/* Central-difference gradient (per mm) of the zero-padded volume at integer
 * index point (i,j,k) of the extended grid [-1,n]^3 (Sec. II-C.1); zero
 * outside the extended grid. */
static void grad_grid(const double *mu, const or_geom *g, int i, int j, int k, double out[3]) {
  if (i < -1 || j < -1 || k < -1 || i > g->nx || j > g->ny || k > g->nz) {
    out[0] = out[1] = out[2] = 0.0;
    return;
  }
  out[0] = (vox(mu, g, i + 1, j, k) - vox(mu, g, i - 1, j, k)) / (2.0 * g->vx);
  out[1] = (vox(mu, g, i, j + 1, k) - vox(mu, g, i, j - 1, k)) / (2.0 * g->vy);
  out[2] = (vox(mu, g, i, j, k + 1) - vox(mu, g, i, j, k - 1)) / (2.0 * g->vz);
}

/* Trilinear interpolation of the zero-padded volume at index point f. */
static double trilinear(const double *mu, const or_geom *g, const double f[3]) {
  int i0 = (int)floor(f[0]), j0 = (int)floor(f[1]), k0 = (int)floor(f[2]);
  double ax = f[0] - i0, ay = f[1] - j0, az = f[2] - k0;
  double s = 0.0;
  for (int c = 0; c < 8; ++c) {
    int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
    double w = (di ? ax : 1.0 - ax) * (dj ? ay : 1.0 - ay) * (dk ? az : 1.0 - az);
    s += w * vox(mu, g, i0 + di, j0 + dj, k0 + dk);
  }
  return s;
}

/* Object-frame spatial gradient (per mm) at index point f:
 * analytic = trilinear interpolation of grad_grid; exact = derivative of
 * the trilinear interpolant itself. */
static void gradient_at(const double *mu, const or_geom *g, const double f[3], int mode, double out[3]) {
  int i0 = (int)floor(f[0]), j0 = (int)floor(f[1]), k0 = (int)floor(f[2]);
  double ax = f[0] - i0, ay = f[1] - j0, az = f[2] - k0;
  out[0] = out[1] = out[2] = 0.0;
  for (int c = 0; c < 8; ++c) {
    int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
    double wx = di ? ax : 1.0 - ax, wy = dj ? ay : 1.0 - ay, wz = dk ? az : 1.0 - az;
    if (mode == OR_GRAD_ANALYTIC) {
      double gg[3];
      grad_grid(mu, g, i0 + di, j0 + dj, k0 + dk, gg);
      double w = wx * wy * wz;
      out[0] += w * gg[0];
      out[1] += w * gg[1];
      out[2] += w * gg[2];
    } else {
      double m = vox(mu, g, i0 + di, j0 + dj, k0 + dk);
      double sx = di ? 1.0 : -1.0, sy = dj ? 1.0 : -1.0, sz = dk ? 1.0 : -1.0;
      out[0] += m * sx * wy * wz / g->vx;
      out[1] += m * wx * sy * wz / g->vy;
      out[2] += m * wx * wy * sz / g->vz;
    }
  }
}

/* ------------------------------------------------------------- ray geometry */

/* Object-frame index coordinate of world point r under pose (R, t). */
static void world_to_index(const or_geom *g, const double R[9], const double t[3], const double r[3],
                           double f[3]) {
  double d[3] = {r[0] - t[0], r[1] - t[1], r[2] - t[2]};
  double rp[3];
  for (int b = 0; b < 3; ++b) rp[b] = R[0 * 3 + b] * d[0] + R[1 * 3 + b] * d[1] + R[2 * 3 + b] * d[2];
  f[0] = (rp[0] - g->off[0]) / g->vx + 0.5 * (g->nx - 1);
  f[1] = (rp[1] - g->off[1]) / g->vy + 0.5 * (g->ny - 1);
  f[2] = (rp[2] - g->off[2]) / g->vz + 0.5 * (g->nz - 1);
}

/* Open box (-m, n - 1 + m)^3 in index coordinates: m = 1 is the support of
 * mu~, m = 2 the support of the interpolated central-difference grid. */
static int inside_box_m(const or_geom *g, const double f[3], int m) {
  return f[0] > -m && f[0] < g->nx - 1 + m && f[1] > -m && f[1] < g->ny - 1 + m && f[2] > -m &&
         f[2] < g->nz - 1 + m;
}

static int inside_box(const or_geom *g, const double f[3]) { return inside_box_m(g, f, 1); }

/* Source and unit direction of the ray through the centre of pixel (iu,iv). */
static void pixel_ray(const or_geom *g, const double *view, int iu, int iv, double s[3], double e[3]) {
  double q[3], L = 0.0;
  for (int a = 0; a < 3; ++a) {
    s[a] = view[a];
    q[a] = view[3 + a] + (iu - 0.5 * (g->nu - 1)) * view[6 + a] + (iv - 0.5 * (g->nv - 1)) * view[9 + a];
    e[a] = q[a] - s[a];
    L += e[a] * e[a];
  }
  L = sqrt(L);
  for (int a = 0; a < 3; ++a) e[a] /= L;
}

/* Range [k_lo, k_hi] of sample indices whose index coordinate can lie in the
 * open box (-m, n - 1 + m)^3; returns 0 when the ray misses.  Samples are
 * re-tested one by one, so this only bounds the loop. */
static int sample_range_m(const or_geom *g, const double R[9], const double t[3], const double s[3],
                          const double e[3], int m, long *k_lo, long *k_hi) {
  double f0[3], f1[3], p1[3];
  world_to_index(g, R, t, s, f0);
  for (int a = 0; a < 3; ++a) p1[a] = s[a] + e[a];
  world_to_index(g, R, t, p1, f1);
  double lo = 0.0, hi = INFINITY;
  const int n[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a) {
    double df = f1[a] - f0[a]; /* index units per mm of arc length */
    if (fabs(df) < 1e-300) {
      if (!(f0[a] > -m && f0[a] < n[a] - 1 + m)) return 0;
      continue;
    }
    double s1 = (-(double)m - f0[a]) / df, s2 = (n[a] - 1 + m - f0[a]) / df;
    double a1 = s1 < s2 ? s1 : s2, a2 = s1 < s2 ? s2 : s1;
    if (a1 > lo) lo = a1;
    if (a2 < hi) hi = a2;
  }
  if (!(hi > lo)) return 0;
  *k_lo = (long)floor(lo / g->step) - 1;
  if (*k_lo < 0) *k_lo = 0;
  *k_hi = (long)ceil(hi / g->step) + 1;
  return 1;
}

static int sample_range(const or_geom *g, const double R[9], const double t[3], const double s[3],
                        const double e[3], long *k_lo, long *k_hi) {
  return sample_range_m(g, R, t, s, e, 1, k_lo, k_hi);
}

static void pose_of(const double *poses, int p, double R[9], double dR[27], double t[3]) {
  or_rotation(poses + 6 * p, R, dR);
  t[0] = poses[6 * p + 0];
  t[1] = poses[6 * p + 1];
  t[2] = poses[6 * p + 2];
}

/* -------------------------------------------------------- forward projector */

/* l_i for every pixel of every instance; proj is [n_inst][nv][nu].
 * nsamples (optional) receives |K_i| summed per instance. */
void or_forward(const or_geom *g, const double *mu, const double *poses, int n_inst, const int *inst_view,
                const int *inst_pose, double *proj, long long *nsamples) {
  const long npix = (long)g->nu * g->nv;
  for (int n = 0; n < n_inst; ++n) {
    double R[9], t[3];
    pose_of(poses, inst_pose[n], R, NULL, t);
    const double *view = g->views + 12 * inst_view[n];
    long long count = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : count)
    for (long p = 0; p < npix; ++p) {
      int iu = (int)(p % g->nu), iv = (int)(p / g->nu);
      double s[3], e[3];
      pixel_ray(g, view, iu, iv, s, e);
      long klo, khi;
      double acc = 0.0;
      if (sample_range(g, R, t, s, e, &klo, &khi)) {
        for (long k = klo; k <= khi; ++k) {
          double r[3], f[3];
          for (int a = 0; a < 3; ++a) r[a] = s[a] + (double)k * g->step * e[a];
          world_to_index(g, R, t, r, f);
          if (!inside_box(g, f)) continue;
          acc += trilinear(mu, g, f);
          ++count;
        }
      }
      proj[(size_t)n * npix + p] = g->step * acc;
    }
    if (nsamples) nsamples[n] = count;
  }
}

/* Contract dL/dM (3x4 per pose) with dM/dtheta: translations read column 4,
 * rotations sum dL/dR_ab * (dR/dg_j)_ab. */
static void contract_pose(const double gM[12], const double dR[27], double gth[6]) {
  for (int a = 0; a < 3; ++a) gth[a] = gM[4 * a + 3];
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s += gM[4 * a + b] * dR[9 * j + 3 * a + b];
    gth[3 + j] = s;
  }
}

/* Forward pose gradient of L given w = dL/dl ([n_inst][nv][nu]):
 *   dL/dM_ab = sum_i w_i step sum_k g_b(r'_k) (r_k - t)_a        (b < 3)
 *   dL/dM_a4 = -sum_i w_i step sum_k sum_b R_ab g_b(r'_k)
 * (Eq. for_grad and the matrices of grad_M x', y', z'; Eq. dis_forward).
 * gM: [n_pose][12] (row-major 3x4), gth: [n_pose][6]; both overwritten. */
void or_forward_grad(const or_geom *g, const double *mu, const double *poses, int n_pose, int n_inst,
                     const int *inst_view, const int *inst_pose, const double *w, int mode, double *gM,
                     double *gth) {
  const long npix = (long)g->nu * g->nv;
  memset(gM, 0, sizeof(double) * 12 * (size_t)n_pose);
  double *ray = (double *)malloc(sizeof(double) * 12 * (size_t)npix);
  for (int n = 0; n < n_inst; ++n) {
    double R[9], t[3];
    pose_of(poses, inst_pose[n], R, NULL, t);
    const double *view = g->views + 12 * inst_view[n];
    const double *wn = w + (size_t)n * npix;
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < npix; ++p) {
      double acc[12] = {0};
      int iu = (int)(p % g->nu), iv = (int)(p / g->nu);
      double s[3], e[3];
      pixel_ray(g, view, iu, iv, s, e);
      long klo, khi;
      const int m = (mode == OR_GRAD_EXACT) ? 1 : 2;
      if (wn[p] != 0.0 && sample_range_m(g, R, t, s, e, m, &klo, &khi)) {
        for (long k = klo; k <= khi; ++k) {
          double r[3], f[3], gr[3];
          for (int a = 0; a < 3; ++a) r[a] = s[a] + (double)k * g->step * e[a];
          world_to_index(g, R, t, r, f);
          if (!inside_box_m(g, f, m)) continue;
          if (mode == OR_GRAD_VOXEL_CENTRE) {
            /* the paper's recipe read literally: G = grad mu (x) (r - t) formed at the
             * voxel centres of the gradient grid, then interpolated like mu */
            int i0 = (int)floor(f[0]), j0 = (int)floor(f[1]), k0 = (int)floor(f[2]);
            double ax = f[0] - i0, ay = f[1] - j0, az = f[2] - k0;
            for (int c = 0; c < 8; ++c) {
              int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
              double wgt = (di ? ax : 1.0 - ax) * (dj ? ay : 1.0 - ay) * (dk ? az : 1.0 - az);
              double gg[3], rp[3], rc[3];
              grad_grid(mu, g, i0 + di, j0 + dj, k0 + dk, gg);
              rp[0] = g->off[0] + (i0 + di - 0.5 * (g->nx - 1)) * g->vx;
              rp[1] = g->off[1] + (j0 + dj - 0.5 * (g->ny - 1)) * g->vy;
              rp[2] = g->off[2] + (k0 + dk - 0.5 * (g->nz - 1)) * g->vz;
              for (int a = 0; a < 3; ++a) rc[a] = R[3 * a + 0] * rp[0] + R[3 * a + 1] * rp[1] + R[3 * a + 2] * rp[2];
              for (int a = 0; a < 3; ++a) {
                for (int b = 0; b < 3; ++b) acc[4 * a + b] += wgt * gg[b] * rc[a];
                acc[4 * a + 3] -= wgt * (R[3 * a + 0] * gg[0] + R[3 * a + 1] * gg[1] + R[3 * a + 2] * gg[2]);
              }
            }
            continue;
          }
          gradient_at(mu, g, f, mode, gr);
          for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) acc[4 * a + b] += gr[b] * (r[a] - t[a]);
            acc[4 * a + 3] -= R[3 * a + 0] * gr[0] + R[3 * a + 1] * gr[1] + R[3 * a + 2] * gr[2];
          }
        }
      }
      for (int q = 0; q < 12; ++q) ray[12 * p + q] = wn[p] * g->step * acc[q];
    }
    double *dst = gM + 12 * (size_t)inst_pose[n];
    for (long p = 0; p < npix; ++p)
      for (int q = 0; q < 12; ++q) dst[q] += ray[12 * p + q];
  }
  free(ray);
  for (int p = 0; p < n_pose; ++p) {
    double R[9], dR[27], t[3];
    pose_of(poses, p, R, dR, t);
    contract_pose(gM + 12 * p, dR, gth + 6 * p);
  }
}

/* Exact transpose of or_forward: each sample spreads step * y_i over the 8
 * trilinear corners inside the grid.  vol ([nz][ny][nx]) is overwritten. */
void or_forward_adjoint(const or_geom *g, const double *y, const double *poses, int n_inst,
                        const int *inst_view, const int *inst_pose, double *vol) {
  const long npix = (long)g->nu * g->nv;
  memset(vol, 0, sizeof(double) * (size_t)g->nx * g->ny * g->nz);
  for (int n = 0; n < n_inst; ++n) {
    double R[9], t[3];
    pose_of(poses, inst_pose[n], R, NULL, t);
    const double *view = g->views + 12 * inst_view[n];
    for (long p = 0; p < npix; ++p) {
      double yi = y[(size_t)n * npix + p];
      if (yi == 0.0) continue;
      int iu = (int)(p % g->nu), iv = (int)(p / g->nu);
      double s[3], e[3];
      pixel_ray(g, view, iu, iv, s, e);
      long klo, khi;
      if (!sample_range(g, R, t, s, e, &klo, &khi)) continue;
      for (long k = klo; k <= khi; ++k) {
        double r[3], f[3];
        for (int a = 0; a < 3; ++a) r[a] = s[a] + (double)k * g->step * e[a];
        world_to_index(g, R, t, r, f);
        if (!inside_box(g, f)) continue;
        int i0 = (int)floor(f[0]), j0 = (int)floor(f[1]), k0 = (int)floor(f[2]);
        double ax = f[0] - i0, ay = f[1] - j0, az = f[2] - k0;
        for (int c = 0; c < 8; ++c) {
          int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
          int ii = i0 + di, jj = j0 + dj, kk = k0 + dk;
          if (ii < 0 || jj < 0 || kk < 0 || ii >= g->nx || jj >= g->ny || kk >= g->nz) continue;
          double wgt = (di ? ax : 1.0 - ax) * (dj ? ay : 1.0 - ay) * (dk ? az : 1.0 - az);
          vol[((size_t)kk * g->ny + jj) * g->nx + ii] += g->step * yi * wgt;
        }
      }
    }
  }
}

/* ------------------------------------------------------------ detector side */

static double pix(const double *img, const or_geom *g, int iu, int iv) {
  if (iu < 0 || iv < 0 || iu >= g->nu || iv >= g->nv) return 0.0;
  return img[(size_t)iv * g->nu + iu];
}

static double bilinear(const double *img, const or_geom *g, double u, double v) {
  int i0 = (int)floor(u), j0 = (int)floor(v);
  double au = u - i0, av = v - j0;
  return (1 - au) * (1 - av) * pix(img, g, i0, j0) + au * (1 - av) * pix(img, g, i0 + 1, j0) +
         (1 - au) * av * pix(img, g, i0, j0 + 1) + au * av * pix(img, g, i0 + 1, j0 + 1);
}

/* Central-difference detector gradient (per pixel index) of the zero-padded
 * image at integer point (iu, iv) of the extended grid [-1,nu]x[-1,nv]. */
static void det_grad_grid(const double *img, const or_geom *g, int iu, int iv, double out[2]) {
  if (iu < -1 || iv < -1 || iu > g->nu || iv > g->nv) {
    out[0] = out[1] = 0.0;
    return;
  }
  out[0] = 0.5 * (pix(img, g, iu + 1, iv) - pix(img, g, iu - 1, iv));
  out[1] = 0.5 * (pix(img, g, iu, iv + 1) - pix(img, g, iu, iv - 1));
}

/* Detector gradient at (u, v): the bilinear interpolant of the
 * central-difference images (zero outside their grid [-1,nu] x [-1,nv]) or
 * the exact derivative of l~. */
static void det_gradient_at(const double *img, const or_geom *g, double u, double v, int mode, double out[2]) {
  int i0 = (int)floor(u), j0 = (int)floor(v);
  double au = u - i0, av = v - j0;
  out[0] = out[1] = 0.0;
  for (int c = 0; c < 4; ++c) {
    int di = c & 1, dj = (c >> 1) & 1;
    double wu = di ? au : 1 - au, wv = dj ? av : 1 - av;
    if (mode == OR_GRAD_ANALYTIC) {
      double gg[2];
      det_grad_grid(img, g, i0 + di, j0 + dj, gg);
      out[0] += wu * wv * gg[0];
      out[1] += wu * wv * gg[1];
    } else {
      double m = pix(img, g, i0 + di, j0 + dj);
      out[0] += m * (di ? 1.0 : -1.0) * wv;
      out[1] += m * wu * (dj ? 1.0 : -1.0);
    }
  }
}

/* World position of voxel (i,j,k) moved by (R, t): r = R r' + t. Also returns r'. */
static void voxel_world(const or_geom *g, const double R[9], const double t[3], int i, int j, int k,
                        double rp[3], double r[3]) {
  rp[0] = g->off[0] + (i - 0.5 * (g->nx - 1)) * g->vx;
  rp[1] = g->off[1] + (j - 0.5 * (g->ny - 1)) * g->vy;
  rp[2] = g->off[2] + (k - 0.5 * (g->nz - 1)) * g->vz;
  for (int a = 0; a < 3; ++a) r[a] = R[3 * a] * rp[0] + R[3 * a + 1] * rp[1] + R[3 * a + 2] * rp[2] + t[a];
}

static void apply_P(const double P[12], const double r[3], double h[3]) {
  for (int a = 0; a < 3; ++a) h[a] = P[4 * a] * r[0] + P[4 * a + 1] * r[1] + P[4 * a + 2] * r[2] + P[4 * a + 3];
}

static double distance_weight(const double P[12], double wp, int weight) {
  if (weight == OR_W_NONE) return 1.0;
  double w0 = P[11]; /* w' of the world origin */
  return (w0 / wp) * (w0 / wp);
}

/* Voxel-driven back-projection; proj is [n_inst][nv][nu], vol overwritten. */
void or_back(const or_geom *g, const double *proj, const double *poses, int n_inst, const int *inst_view,
             const int *inst_pose, int weight, double *vol) {
  const long npix = (long)g->nu * g->nv;
  memset(vol, 0, sizeof(double) * (size_t)g->nx * g->ny * g->nz);
  for (int n = 0; n < n_inst; ++n) {
    double R[9], t[3], P[12];
    pose_of(poses, inst_pose[n], R, NULL, t);
    or_projection_matrix(g->views + 12 * inst_view[n], g->nu, g->nv, P);
    const double *img = proj + (size_t)n * npix;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          double rp[3], r[3], h[3];
          voxel_world(g, R, t, i, j, k, rp, r);
          apply_P(P, r, h);
          if (!(h[2] > 0.0)) continue;
          double u = h[0] / h[2], v = h[1] / h[2];
          vol[((size_t)k * g->ny + j) * g->nx + i] += distance_weight(P, h[2], weight) * bilinear(img, g, u, v);
        }
  }
}

/* Exact transpose of or_back: each voxel spreads W * y_j over the 4
 * bilinear corners inside the detector; proj [n_inst][nv][nu] overwritten. */
void or_back_adjoint(const or_geom *g, const double *y, const double *poses, int n_inst, const int *inst_view,
                     const int *inst_pose, int weight, double *proj) {
  const long npix = (long)g->nu * g->nv;
  memset(proj, 0, sizeof(double) * (size_t)n_inst * npix);
  for (int n = 0; n < n_inst; ++n) {
    double R[9], t[3], P[12];
    pose_of(poses, inst_pose[n], R, NULL, t);
    or_projection_matrix(g->views + 12 * inst_view[n], g->nu, g->nv, P);
    double *img = proj + (size_t)n * npix;
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          double yj = y[((size_t)k * g->ny + j) * g->nx + i];
          if (yj == 0.0) continue;
          double rp[3], r[3], h[3];
          voxel_world(g, R, t, i, j, k, rp, r);
          apply_P(P, r, h);
          if (!(h[2] > 0.0)) continue;
          double u = h[0] / h[2], v = h[1] / h[2];
          double W = distance_weight(P, h[2], weight);
          int i0 = (int)floor(u), j0 = (int)floor(v);
          double au = u - i0, av = v - j0;
          for (int c = 0; c < 4; ++c) {
            int di = c & 1, dj = (c >> 1) & 1;
            int iu = i0 + di, iv = j0 + dj;
            if (iu < 0 || iv < 0 || iu >= g->nu || iv >= g->nv) continue;
            img[(size_t)iv * g->nu + iu] += W * yj * (di ? au : 1 - au) * (dj ? av : 1 - av);
          }
        }
  }
}

/* Back-projection pose gradient given wvol = dL/dmu ([nz][ny][nx]):
 *   dL/dM_ab = sum_inst sum_j wvol_j rho_a (x', y', z', 1)_b
 *   rho = W (d_u l~, d_v l~) J_p(r_j) + l~ grad_r W
 * with J_p the 2x3 Jacobian of d = p(r) (Eq. back_derive and the Jacobian
 * of the 3D-2D mapping; Eq. dis_back).  gM: [n_pose][12], gth [n_pose][6]. */
void or_back_grad(const or_geom *g, const double *proj, const double *poses, int n_pose, int n_inst,
                  const int *inst_view, const int *inst_pose, int weight, int mode, const double *wvol,
                  double *gM, double *gth) {
  const long npix = (long)g->nu * g->nv;
  memset(gM, 0, sizeof(double) * 12 * (size_t)n_pose);
  double *slab = (double *)malloc(sizeof(double) * 12 * (size_t)g->nz);
  for (int n = 0; n < n_inst; ++n) {
    double R[9], t[3], P[12];
    pose_of(poses, inst_pose[n], R, NULL, t);
    or_projection_matrix(g->views + 12 * inst_view[n], g->nu, g->nv, P);
    const double *img = proj + (size_t)n * npix;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < g->nz; ++k) {
      double acc[12] = {0};
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          double wj = wvol[((size_t)k * g->ny + j) * g->nx + i];
          if (wj == 0.0) continue;
          double rp[3], r[3], h[3];
          voxel_world(g, R, t, i, j, k, rp, r);
          apply_P(P, r, h);
          if (!(h[2] > 0.0)) continue;
          double u = h[0] / h[2], v = h[1] / h[2];
          double dl[2];
          det_gradient_at(img, g, u, v, mode, dl);
          double J[2][3];
          for (int c = 0; c < 3; ++c) {
            J[0][c] = (P[c] * h[2] - P[8 + c] * h[0]) / (h[2] * h[2]);
            J[1][c] = (P[4 + c] * h[2] - P[8 + c] * h[1]) / (h[2] * h[2]);
          }
          double W = distance_weight(P, h[2], weight);
          double gW[3] = {0, 0, 0};
          if (weight == OR_W_FDK)
            for (int c = 0; c < 3; ++c) gW[c] = -2.0 * W / h[2] * P[8 + c];
          double lv = (weight == OR_W_FDK) ? bilinear(img, g, u, v) : 0.0;
          double rt[4] = {rp[0], rp[1], rp[2], 1.0};
          for (int a = 0; a < 3; ++a) {
            double rho = W * (dl[0] * J[0][a] + dl[1] * J[1][a]) + lv * gW[a];
            for (int b = 0; b < 4; ++b) acc[4 * a + b] += wj * rho * rt[b];
          }
        }
      for (int q = 0; q < 12; ++q) slab[12 * k + q] = acc[q];
    }
    double *dst = gM + 12 * (size_t)inst_pose[n];
    for (int k = 0; k < g->nz; ++k)
      for (int q = 0; q < 12; ++q) dst[q] += slab[12 * k + q];
  }
  free(slab);
  for (int p = 0; p < n_pose; ++p) {
    double R[9], dR[27], t[3];
    pose_of(poses, p, R, dR, t);
    contract_pose(gM + 12 * p, dR, gth + 6 * p);
  }
}

/* ---------------------------------------------------------- sampled outputs */

/* Forward projections of selected pixels only: pix[m] = (instance, iu, iv);
 * out[m] = l of that ray (same definition as or_forward). */
void or_forward_pixels(const or_geom *g, const double *mu, const double *poses, const int *inst_view,
                       const int *inst_pose, int n_pix, const int *pix, double *out) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int m = 0; m < n_pix; ++m) {
    const int n = pix[3 * m], iu = pix[3 * m + 1], iv = pix[3 * m + 2];
    double R[9], t[3], s[3], e[3];
    pose_of(poses, inst_pose[n], R, NULL, t);
    pixel_ray(g, g->views + 12 * inst_view[n], iu, iv, s, e);
    long klo, khi;
    double acc = 0.0;
    if (sample_range(g, R, t, s, e, &klo, &khi)) {
      for (long k = klo; k <= khi; ++k) {
        double r[3], f[3];
        for (int a = 0; a < 3; ++a) r[a] = s[a] + (double)k * g->step * e[a];
        world_to_index(g, R, t, r, f);
        if (!inside_box(g, f)) continue;
        acc += trilinear(mu, g, f);
      }
    }
    out[m] = g->step * acc;
  }
}

/* Back-projection at selected voxels only: vox[m] = (i, j, k); out[m] =
 * sum over all instances (same definition as or_back). */
void or_back_voxels(const or_geom *g, const double *proj, const double *poses, int n_inst, const int *inst_view,
                    const int *inst_pose, int weight, int n_vox, const int *vox, double *out) {
  const long npix = (long)g->nu * g->nv;
#pragma omp parallel for schedule(dynamic, 16)
  for (int m = 0; m < n_vox; ++m) {
    double acc = 0.0;
    for (int n = 0; n < n_inst; ++n) {
      double R[9], t[3], P[12], rp[3], r[3], h[3];
      pose_of(poses, inst_pose[n], R, NULL, t);
      or_projection_matrix(g->views + 12 * inst_view[n], g->nu, g->nv, P);
      voxel_world(g, R, t, vox[3 * m], vox[3 * m + 1], vox[3 * m + 2], rp, r);
      apply_P(P, r, h);
      if (!(h[2] > 0.0)) continue;
      acc += distance_weight(P, h[2], weight) * bilinear(proj + (size_t)n * npix, g, h[0] / h[2], h[1] / h[2]);
    }
    out[m] = acc;
  }
}
