/*
 * proj.h - C ABI of the B300 (sm_103a) cone-beam projector library.
 *
 * Operations (paper: "Differentiable Forward and Back-Projector for Rigid
 * Motion Estimation in X-ray Imaging"):
 *   proj_set_volume         volume gradient grad mu by central differences
 *                           (Sec. II-C.1), cached in the workspace;
 *   proj_forward            ray-driven forward projection l = A(M) mu
 *                           (Eq. forward, Sec. II-C.1);
 *   proj_forward_pose_grad  dL/dtheta of a projection-domain loss, the
 *                           12 channels of G_f projected in the same march
 *                           (Eqs. for_grad, final_forward, for_int,
 *                           dis_forward), fused with the loss residual;
 *   proj_back               voxel-driven back-projection mu = A^T(M) l
 *                           (Eq. back, Sec. II-C.2);
 *   proj_back_pose_grad     dL/dtheta of an image-domain loss, the 12
 *                           channels of G_b back-projected (Eqs. back_derive,
 *                           final_back, back_int, dis_back);
 *   proj_forward_adjoint    exact transpose of proj_forward (the "A^T" of
 *                           Sec. II-C.2 for the ray-driven A).
 *
 * Conventions (the paper leaves them open; Table I fixes the symbols):
 *   - World frame in mm; pose theta = (tx, ty, tz, gx, gy, gz) in mm and
 *     rad; R = Rz(gz) Ry(gy) Rx(gx); a point r' of the object is seen at
 *     r = R r' + t (M = [R | t]), so r' = R^T (r - t).
 *   - Volume memory order [nz][ny][nx], FP32; voxel (i, j, k) centre in the
 *     object frame = vol_offset + ((i-(nx-1)/2) vx, (j-(ny-1)/2) vy,
 *     (k-(nz-1)/2) vz).  mu is zero outside the grid and the trilinear
 *     interpolant mu~ uses zero padding.
 *   - View v: source s, detector centre c, pixel-pitch vectors U (column
 *     direction, |U| = pixel width) and V (row direction); pixel (iu, iv)
 *     centre = c + (iu-(nu-1)/2) U + (iv-(nv-1)/2) V.  Images are
 *     [nv][nu], FP32.  The projection matrix P of Eq. projmatrix is built
 *     from these vectors in pixel-index units: P = [B^-1 | -B^-1 s],
 *     B = [U | V | q00 - s].
 *   - Ray of pixel i: r_k = s + k * step * e_i (e_i unit), k >= 0 integer;
 *     l_i = step * sum over k whose object index coordinate lies in the
 *     open box (-1, n)^3 of mu~(R^T (r_k - t)).
 *   - Back-projection: mu_j = sum over instances of W * l~(d_j), d_j the
 *     projection of R r'_j + t, l~ bilinear with zero padding, W = 1 or the
 *     FDK distance weight (w'(0) / w'(r_j))^2; voxels with w' <= 0 get 0.
 *   - Pose gradients are returned per pose: dL/dt in 1/mm, dL/dgamma in
 *     1/rad.
 *
 * Instances.  A plan has n_views physical views (geometry) and n_pose
 * poses.  An instance is one (view, pose) pair; every call processes all
 * n_inst instances of the plan.  Registration of 64 candidates seen by 2
 * views is n_views = 2, n_pose = 64, n_inst = 128; per-view motion
 * (motion-compensated reconstruction) is n_pose = n_inst = n_views.
 *
 * Memory and streams.  Every pointer whose name starts with d_ is device
 * memory owned by the caller; everything else is host memory read during
 * the call.  The plan owns only small device tables (views, instance map)
 * allocated at creation.  Calls never allocate: scratch space is the
 * caller's workspace d_ws of at least proj_workspace_size() bytes, which
 * must stay untouched between proj_set_volume and the calls that use the
 * volume.  Its first 256 bytes hold the device status word: zero them once
 * after allocating the workspace.  Every call is asynchronous on the caller's stream (NULL = legacy
 * default stream); outputs are overwritten, never accumulated.  Calls on
 * one plan and workspace must not overlap on the GPU.
 *
 * Errors.  Functions return PROJ_OK (0) or a negative code; the message of
 * the last failure in the calling thread is in proj_last_error().  Argument
 * checks run on the host before any launch and then nothing is launched.
 * Conditions only the device can see (a non-finite pose) make the affected
 * instances contribute zero and set a bit in a status word inside the
 * workspace; proj_check() reads and clears it (it synchronises the stream).
 */
#ifndef PROJ_H
#define PROJ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *proj_stream;

enum {
  PROJ_OK = 0,
  PROJ_E_ARG = -1,         /* invalid argument (null, size, index, value) */
  PROJ_E_CUDA = -2,        /* a CUDA runtime call or launch failed */
  PROJ_E_WORKSPACE = -3,   /* workspace missing, too small or misaligned */
  PROJ_E_UNSUPPORTED = -4, /* operation not enabled in the plan's flags */
  PROJ_E_DEVICE = -5       /* device-side status bit set (see proj_check) */
};

/* Loss modes of proj_forward_pose_grad. */
enum {
  PROJ_LOSS_RESIDUAL = 0, /* d_ref = dL/dl per instance [n_inst][nv][nu] */
  PROJ_LOSS_L2 = 1,       /* d_ref = target per view [n_views][nv][nu];
                             L_pose = sum over its instances of sum (l-b)^2
                             (Eq. forward_loss) */
  PROJ_LOSS_NCC = 2       /* d_ref = target per view; L_pose = -mean over its
                             instances of the Pearson NCC of l and b over
                             the whole image (Sec. II-D.3) */
};

/* Back-projection weights. */
enum {
  PROJ_W_NONE = 0,      /* W = 1 */
  PROJ_W_FDK = 1,       /* W = (w'(0)/w'(r))^2; gradients include l~ grad W */
  PROJ_W_FDK_CONST = 2  /* same W; gradients treat W as constant */
};

/* Operations a plan must support (sizes its workspace). */
enum {
  PROJ_OP_FORWARD = 1,
  PROJ_OP_FORWARD_GRAD = 2,
  PROJ_OP_BACK = 4,
  PROJ_OP_BACK_GRAD = 8,
  PROJ_OP_ADJOINT = 16,
  PROJ_OP_SHARPNESS = 32,
  PROJ_OP_ALL = 63
};

/* Option flags, ORed into the ops argument of proj_plan_create (a library
 * facility; the paper fixes no memory layout). */
enum {
  /* Keep one copy of the prepared volume (rows along x) instead of two
   * (rows along x and along y, each instance marching the copy whose rows
   * run closest to its detector u axis).  Halves the volume part of the
   * workspace (the float4 (mu, grad mu) volume is 16 B per voxel of the
   * padded grid, the cell records of the DRR march 16 B per voxel) at the
   * cost of slower gathers for instances whose u axis runs along y.
   * Results are identical to the two-copy plan's. */
  PROJ_FLAG_ONE_COPY = 256,
  /* Fused pose-gradient march over a bricked copy of the prepared volume:
   * bricks of 4^3 cells, each storing the 5^3 (mu, grad mu) elements at its
   * cells' corners (2 KB with padding), so a sample's 8 corners sit at fixed
   * offsets inside one brick, in place of the rows-along-y copy.  Every
   * instance marches the bricked copy with 4 x 8-pixel warps (the warp shape
   * setting is ignored); results are identical to the other layouts'.  About
   * 1.95x the volume memory of one row copy.  Kept as a measured
   * alternative layout (the rows-along-x / rows-along-y pair is faster on
   * the workloads measured). */
  PROJ_FLAG_BRICKS = 512
};

/* Device status bits (proj_check). */
enum {
  PROJ_STATUS_BAD_POSE = 1, /* a pose had a non-finite entry */
  PROJ_STATUS_BAD_INDEX = 2 /* a pose list held an index outside [-1, n_pose) */
};

typedef struct {
  int nx, ny, nz;        /* volume size in voxels, each >= 1 */
  double vx, vy, vz;     /* voxel pitch, mm, > 0 */
  double vol_offset[3];  /* object-frame position of the volume centre, mm */
  int nu, nv;            /* detector columns and rows, each >= 1 */
  int n_views;           /* >= 1 */
  const double *views;   /* host [n_views][12]: s, c, U, V (mm) */
  double step;           /* ray step along the world ray, mm, > 0 */
} proj_geometry;

typedef struct proj_plan_s *proj_plan;

/* Create a plan on the current CUDA device.
 *   geom       geometry, copied (views included); not referenced later.
 *   n_pose     number of poses, >= 1.
 *   n_inst     number of instances, >= 1.
 *   inst_view  host [n_inst], view of each instance in [0, n_views).
 *   inst_pose  host [n_inst], pose of each instance in [0, n_pose).
 *   ops        OR of PROJ_OP_* the plan must support (at least one), plus
 *              optional PROJ_FLAG_* options.
 *   out        receives the plan.
 * Limits: ny, nz, nv <= 65000; with PROJ_OP_BACK or PROJ_OP_BACK_GRAD at
 * most 65535 instances; padded volumes below 2^31 voxels.
 * Errors: PROJ_E_ARG (bad sizes, indices, non-finite or degenerate
 * geometry, singular detector basis, limits above), PROJ_E_CUDA (table
 * allocation). */
int proj_plan_create(const proj_geometry *geom, int n_pose, int n_inst, const int *inst_view,
                     const int *inst_pose, int ops, proj_plan *out);

/* Free a plan and its device tables (synchronous).  NULL is a no-op. */
int proj_plan_destroy(proj_plan plan);

/* Bytes of workspace the plan needs (multiple of 256; base must be
 * 256-byte aligned). */
int proj_workspace_size(proj_plan plan, size_t *bytes);

/* Prepare the volume for the ray-driven calls (Sec. II-C.1: grad mu by
 * central differences of the zero-padded volume): writes into the workspace,
 * when PROJ_OP_FORWARD is enabled, zero-bordered cell records of mu (the
 * four corners of each cell's xy face, two copies with rows along x and y)
 * and, when PROJ_OP_FORWARD_GRAD is enabled, a float4
 * (mu, d mu/dx', d mu/dy', d mu/dz') volume (per mm, object frame) on the
 * index grid [-1, n]^3 and its copy with rows along y; for either, the
 * occupancy bricks of the empty-space skipping (proj_set_skip_brick).
 *   d_mu  [nz][ny][nx] FP32.
 * Must run before proj_forward / proj_forward_pose_grad; stays valid until
 * the workspace is reused for another volume. */
int proj_set_volume(proj_plan plan, const float *d_mu, void *d_ws, size_t ws_bytes, proj_stream stream);

/* Forward projection of the volume last set (Eq. forward).
 *   d_pose  [n_pose][6] FP32.
 *   d_proj  out [n_inst][nv][nu] FP32. */
int proj_forward(proj_plan plan, const float *d_pose, float *d_proj, void *d_ws, size_t ws_bytes,
                 proj_stream stream);

/* Pose gradient of a projection-domain loss (Eqs. for_grad, final_forward,
 * dis_forward).  One march per ray accumulates l_i and the 12 sums of G_f
 * (grad mu interpolated from the central-difference grid at every sample);
 * the loss residual weights each ray at its end; nothing per channel is
 * written to memory.
 *   loss        PROJ_LOSS_*.
 *   d_ref       RESIDUAL: dL/dl [n_inst][nv][nu]; L2 / NCC: target images
 *               [n_views][nv][nu].
 *   d_grad      out [n_pose][6] FP32, dL/dtheta.
 *   d_loss      out [n_pose] FP32 or NULL (RESIDUAL writes 0).
 *   d_proj      out [n_inst][nv][nu] FP32 projections, or NULL. */
int proj_forward_pose_grad(proj_plan plan, const float *d_pose, int loss, const float *d_ref, float *d_grad,
                           float *d_loss, float *d_proj, void *d_ws, size_t ws_bytes, proj_stream stream);

/* proj_forward_pose_grad for a subset of the plan's poses, chosen per call
 * (a library facility for multi-start registration: starts that have
 * converged or failed leave the launch, new starts take their slots).
 *   d_pose_list  device [n_list] int32: pose indices in [0, n_pose), or -1
 *                for an empty slot.  The kernels read it when they run, so
 *                a caller may rewrite it on the stream between calls (also
 *                inside a captured CUDA graph).  An entry outside
 *                [-1, n_pose) is skipped and sets PROJ_STATUS_BAD_INDEX; a
 *                pose listed twice is evaluated twice with identical results.
 *   n_list       >= 1 (slots; the launch grid has n_list x the largest
 *                number of instances of one pose x ray tiles blocks, which
 *                must stay below 2^31).
 * Every instance of each listed pose is marched.  Rows of d_grad and d_loss
 * belong to the poses (as in proj_forward_pose_grad); only the rows of
 * listed poses are written, the others are left as they were.  d_proj rows
 * of the marched instances are written, the others left as they were.
 * Other arguments and errors as proj_forward_pose_grad. */
int proj_forward_pose_grad_list(proj_plan plan, const float *d_pose, const int *d_pose_list, int n_list, int loss,
                                const float *d_ref, float *d_grad, float *d_loss, float *d_proj, void *d_ws,
                                size_t ws_bytes, proj_stream stream);

/* Voxel-driven back-projection (Eq. back) of one image per instance.
 *   d_proj  [n_inst][nv][nu] FP32; copied first into zero-bordered cell
 *           records in the workspace (the 4 pixels of each bilinear cell).
 *   weight  PROJ_W_NONE or PROJ_W_FDK (FDK_CONST behaves as FDK here).
 *   d_vol   out [nz][ny][nx] FP32 (sum over all instances). */
int proj_back(proj_plan plan, const float *d_proj, const float *d_pose, int weight, float *d_vol, void *d_ws,
              size_t ws_bytes, proj_stream stream);

/* Exact transpose of proj_back (the projection-side gradient of a
 * back-projection, for autograd): each voxel value is spread, times W, over
 * the 4 bilinear corners of its projection in every instance.
 *   d_vol   [nz][ny][nx] FP32 (dL/dmu).
 *   weight  PROJ_W_NONE or PROJ_W_FDK (FDK_CONST behaves as FDK).
 *   d_proj  out [n_inst][nv][nu] FP32: the weights are accumulated with
 *           float vector reductions into detector cell records in the
 *           workspace, then the 4 records sharing each pixel are summed
 *           (the last bits depend on the order of the reductions). */
int proj_back_adjoint(proj_plan plan, const float *d_vol, const float *d_pose, int weight, float *d_proj, void *d_ws,
                      size_t ws_bytes, proj_stream stream);

/* Pose gradient of an image-domain loss through the back-projector
 * (Eqs. back_derive, final_back, back_int, dis_back): grad_d l by central
 * differences of each image interpolated at the projected voxel, the
 * projection Jacobian, and the FDK weight derivative for PROJ_W_FDK.
 *   d_proj      [n_inst][nv][nu] FP32 images that were back-projected.
 *   weight      PROJ_W_*.
 *   d_vol_resid dL/dmu [nz][ny][nx] FP32.
 *   d_grad      out [n_pose][6] FP32. */
int proj_back_pose_grad(proj_plan plan, const float *d_proj, const float *d_pose, int weight,
                        const float *d_vol_resid, float *d_grad, void *d_ws, size_t ws_bytes,
                        proj_stream stream);

/* Measurement aid, no counterpart in the paper: runs the pose set-up and a
 * kernel with the memory access pattern of the fused pose-gradient march
 * (same grid, rays, samples, volume copies and eight 16-byte corner loads
 * per sample) but none of its arithmetic, so its duration (with kernel
 * timing enabled, proj_kernel_time_ms) is the empirical ceiling of that
 * gather on this device.  The volume must be set.  Writes only the
 * workspace.  Errors as proj_forward_pose_grad. */
int proj_gather_probe(proj_plan plan, const float *d_pose, void *d_ws, size_t ws_bytes, proj_stream stream);

/* Ray-tile shape of the fused pose-gradient march.  Each CTA marches a
 * 16 x 16-pixel tile with 8 warps; warp_width is the number of pixels along
 * u covered by one warp (warp_width x 32/warp_width rays: 2 x 16, 4 x 8,
 * 8 x 4 or 16 x 2).  Which shape gathers (mu, grad mu) with the fewest L1
 * wavefronts depends on how the rays cross the volume, so it is a tuning
 * parameter of the plan (default 4).  Results of different shapes agree to
 * FP32 rounding (the per-tile sums are taken in a different order).
 * proj_set_warp_shape: PROJ_E_ARG unless warp_width is 2, 4, 8 or 16.
 * proj_autotune_forward_grad: sets up the poses, then times `reps` launches
 * of the march per shape on the caller's data (plan volume set, d_pose,
 * loss, d_ref as in proj_forward_pose_grad), stores the fastest shape in
 * the plan and returns it in *warp_width (may be NULL) with the mean
 * per-launch times in times_ms[4] (order 2, 4, 8, 16; may be NULL).
 * Writes only the workspace; synchronises the stream (not for capture). */
int proj_set_warp_shape(proj_plan plan, int warp_width);
int proj_get_warp_shape(proj_plan plan, int *warp_width);
int proj_autotune_forward_grad(proj_plan plan, const float *d_pose, int loss, const float *d_ref, void *d_ws,
                               size_t ws_bytes, proj_stream stream, int reps, float *times_ms, int *warp_width);

/* Empty-space skipping in proj_forward and the fused pose-gradient marches
 * (a library facility; the paper has none).  proj_set_volume also records,
 * for bricks of 8^3 and of 16^3 cells of the 2-voxel-bordered grid, whether
 * a brick holds, or lies within one cell of, a cell with a non-zero corner in
 * (mu, grad mu), and, one bit per cell, whether the cell itself has one (the
 * cell map).  Before marching, each ray walks the bricks it crosses and
 * keeps only its samples from two before the first to two after the last
 * occupied brick; inside that range the fused pose-gradient march (not the
 * DRR march) tests each sample's cell in the cell map and leaves out the
 * gathers and arithmetic of samples whose cell has none.  A sample left out
 * reads eight zero corners and adds exact zeros to every sum, and the kept
 * samples are summed in the same order, so results are bit-identical with
 * and without skipping; only the time changes (most for volumes with much
 * empty space around and inside the object; on dense volumes the tests cost
 * a little).  The exact transposes never skip (they do not read mu).
 * proj_set_skip_brick: edge 8 (default), 16, or 0 (off); PROJ_E_ARG
 * otherwise.  proj_set_skip_cells: the cell test of the fused march, which
 * works with or without bricks: 0 off, 1 on, 2 automatic (default): on when,
 * for the volume of the last proj_set_volume, at most 85 % of the cells in
 * the occupied 8^3 bricks have a non-zero corner (decided on the device, no
 * synchronisation; on a uniformly filled volume the tests cost about 12 %);
 * PROJ_E_ARG otherwise.
 * proj_autotune_march: like proj_autotune_forward_grad over the 3 x 2 x 4
 * combinations of brick edge (0, 8, 16), cell test (0 off, 1 on) and warp
 * shape (2, 4, 8, 16); keeps the fastest in the plan and returns it in
 * *warp_width, *brick_edge and *skip_cells (each may be NULL) with the times
 * in times_ms[24] (index 4 * (2 * edge position + cell test) + shape
 * position; may be NULL).  proj_count_marched_samples: like
 * proj_count_samples, but counts the samples the fused march gathers with
 * the plan's setting (the gradient grid's box (-2, n+1), clipped to the
 * occupied bricks, and of those the ones in cells with a non-zero corner when
 * the cell test is on); needs PROJ_OP_FORWARD_GRAD. */
int proj_set_skip_brick(proj_plan plan, int edge);
int proj_get_skip_brick(proj_plan plan, int *edge);
int proj_set_skip_cells(proj_plan plan, int mode);
int proj_get_skip_cells(proj_plan plan, int *mode);
int proj_autotune_march(proj_plan plan, const float *d_pose, int loss, const float *d_ref, void *d_ws,
                        size_t ws_bytes, proj_stream stream, int reps, float *times_ms, int *warp_width,
                        int *brick_edge, int *skip_cells);
int proj_count_marched_samples(proj_plan plan, const float *d_pose, long long *d_count, void *d_ws, size_t ws_bytes,
                               proj_stream stream);

/* Brick shape of the back-projection gradient (a library facility; the
 * paper fixes none): a block owns 32 x 8 voxel columns of gz voxels and a
 * chunk of instances.  Shapes: 0 = gz 16, 8 instances; 1 = gz 8, 8;
 * 2 = gz 16, 16; 3 = gz 8, 16 (default).  Results of different shapes
 * differ only in the order of the FP32 partial sums.
 * Errors: PROJ_E_ARG (NULL plan or pointer, shape out of range). */
int proj_set_brick_shape(proj_plan plan, int shape);
int proj_get_brick_shape(proj_plan plan, int *shape);

/* Times proj_back_pose_grad's voxel kernel under every brick shape on the
 * caller's data (CUDA events, one warm-up and `reps` launches each), keeps
 * the fastest in the plan and returns it in *shape (may be NULL) and the
 * times in times_ms[4] (ms per launch, may be NULL).  Arguments as
 * proj_back_pose_grad without d_grad: writes only the workspace.
 * Synchronises the stream (not for capture).  Needs PROJ_OP_BACK_GRAD;
 * reps in 1..1000.
 * Errors: PROJ_E_ARG, PROJ_E_UNSUPPORTED, PROJ_E_WORKSPACE, PROJ_E_CUDA. */
int proj_autotune_back_grad(proj_plan plan, const float *d_proj, const float *d_pose, int weight,
                            const float *d_vol_resid, void *d_ws, size_t ws_bytes, proj_stream stream, int reps,
                            float *times_ms, int *shape);

/* Batches: several independent forward pose-gradient problems (each a plan
 * with its own volume, detector, views, poses and workspace, e.g. registration
 * problems of uneven size) run by one persistent launch.  Resident blocks
 * take 16 x 16-pixel ray tiles of any problem from a single atomic work
 * counter (no waits); problems are ordered by estimated cost per tile,
 * longest first, so small problems fill the tail of large ones.  Results
 * are identical to proj_forward_pose_grad on each plan at the default warp
 * shape (the batched march always uses 4 x 8-pixel warps).
 *
 * proj_batch_create binds, for problem i: plans[i] (needs
 * PROJ_OP_FORWARD_GRAD; volume set with proj_set_volume before runs),
 * loss[i], d_pose[i] [n_pose_i][6], d_ref[i] (as in proj_forward_pose_grad),
 * d_grad[i] [n_pose_i][6], d_loss[i] (array may be NULL, entries may be
 * NULL), d_ws[i] / ws_bytes[i] (distinct workspaces).  All arrays are host
 * arrays of device pointers, read during the call; the device buffers must
 * outlive the batch.  The batch owns a small device descriptor table.
 * proj_batch_run launches the pose set-ups, the persistent march and the
 * per-problem reductions on the stream (no host-device copies).
 * Errors: PROJ_E_ARG, PROJ_E_UNSUPPORTED, PROJ_E_WORKSPACE, PROJ_E_CUDA. */
typedef struct proj_batch_s *proj_batch;
int proj_batch_create(int n, const proj_plan *plans, const int *loss, const float *const *d_pose,
                      const float *const *d_ref, float *const *d_grad, float *const *d_loss, void *const *d_ws,
                      const size_t *ws_bytes, proj_batch *out);
int proj_batch_run(proj_batch batch, proj_stream stream);
int proj_batch_destroy(proj_batch batch);

/* Exact transpose of proj_forward for the given poses: each sample spreads
 * step * y_i over its 8 trilinear corners.
 *   d_y    [n_inst][nv][nu] FP32.
 *   d_vol  out [nz][ny][nx] FP32: the weights are accumulated with float
 *          vector reductions into cell records in the workspace (the 4
 *          corners of each cell's xy face), then the 4 records sharing each
 *          voxel are summed (the last bits depend on the order of the
 *          reductions).  Needs PROJ_OP_ADJOINT. */
int proj_forward_adjoint(proj_plan plan, const float *d_y, const float *d_pose, float *d_vol, void *d_ws,
                         size_t ws_bytes, proj_stream stream);

/* FDK filtering of one image per instance (the "Ramp(l)" of the motion-
 * compensated reconstruction experiment, Sec. II-D.3): each pixel is
 * multiplied by the cosine weight SAD / sqrt(SAD^2 + a^2 + b^2) ((a, b): its
 * offset from the principal point on the isocentre plane, SAD: distance from
 * the source to that plane), then every row is convolved with the Ram-Lak
 * ramp kernel (h[0] = 1/4, h[k] = -1/(pi k)^2 for odd k, 0 for even k, in
 * units of 1/du^2, du the pixel pitch on the isocentre plane) with zero
 * padding, times du and times scale (e.g. pi / n_views for a full circular
 * scan, so that proj_back with PROJ_W_FDK then gives the FDK
 * reconstruction).  Assumes orthogonal pixel axes.
 *   d_proj  [n_inst][nv][nu] FP32; d_out  out, same shape, must not alias.
 * Uses no workspace. */
int proj_fdk_filter(proj_plan plan, const float *d_proj, float scale, float *d_out, proj_stream stream);

/* Image sharpness S = -Var(|grad mu|) over all voxels (|grad mu| from
 * central differences of the zero-padded volume, per mm; the variance uses
 * the population mean) and, when d_grad is not NULL, dS/dmu (exact
 * derivative of that expression; voxels with |grad mu| < 1e-12 contribute
 * no direction).  Needs PROJ_OP_SHARPNESS.
 *   d_vol  [nz][ny][nx] FP32; d_loss  out, 1 float; d_grad  out [nz][ny][nx]
 *          or NULL.  The moments are summed in FP64 in a fixed order. */
int proj_sharpness(proj_plan plan, const float *d_vol, float *d_loss, float *d_grad, void *d_ws, size_t ws_bytes,
                   proj_stream stream);

/* One Adam step on n poses (the optimiser of the registration and
 * motion-compensation loops, Sec. II-D.3), in one launch, no plan needed.
 * For each pose i with d_active[i] != 0 (every pose when d_active is NULL):
 * t_i += 1; per parameter j: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * pose -= lr[j] (m / (1 - b1^t_i)) / (sqrt(v / (1 - b2^t_i)) + eps).
 * Inactive poses keep pose, m, v and t_i, so a pose's bias correction counts
 * only its own updates.
 *   d_pose, d_grad, d_m, d_v  [n][6] FP32 (device); d_t  [n] FP32 step
 *   counts (device, start at 0); d_active  [n] bytes (device) or NULL;
 *   lr  6 step sizes (host memory, copied into the launch); b1, b2, eps
 *   FP32 (1 - b1 and 1 - b2 are formed from those FP32 values).
 * Asynchronous on stream, no allocation, capturable in a CUDA graph.
 * Errors: PROJ_E_ARG (NULL pointers, n < 0, b1 or b2 outside [0, 1),
 * eps < 0), PROJ_E_CUDA. */
int proj_pose_adam(float *d_pose, const float *d_grad, float *d_m, float *d_v, float *d_t,
                   const unsigned char *d_active, int n, const float *lr, float b1, float b2, float eps,
                   proj_stream stream);

/* Parameters of proj_registration_step. */
typedef struct {
  float lr[6];           /* Adam step sizes per pose parameter (mm, rad) */
  float b1, b2, eps;     /* Adam moments and epsilon (FP32 values) */
  float ncc_stop;        /* a start stops when -loss >= ncc_stop (loss = -NCC) ... */
  float dloss_stop;      /* ... or |loss - previous loss| < dloss_stop ... */
  long long max_iter;    /* ... or after max_iter updates */
  float tol_mm, tol_deg; /* hit tolerance against the truth: every |translation error| <= tol_mm and
                            every |rotation error| <= tol_deg */
} proj_reg_params;

/* The bookkeeping of one iteration of a multi-start registration (Sec.
 * II-D.3), after proj_forward_pose_grad(_list) has written the loss and
 * gradient of the listed starts, in one launch (one block):
 *   1. the starts in d_slots (n_slots entries, -1 = empty) are "listed";
 *   2. for each listed start i: if d_truth is given and pose i is within
 *      the tolerance of truth row i (or of row 0 when n_truth = 1),
 *      *d_hit_any = 1; the start stops (d_alive[i] = 0) when its loss meets
 *      a stopping rule; a start still alive counts the update in
 *      d_iters[i] and takes one Adam step (as proj_pose_adam); its loss is
 *      kept in d_last[i] for the next loss-change test;
 *   3. every slot that is empty or holds a stopped start takes the next
 *      start in order (*d_next, then *d_next + 1, ...) while starts remain,
 *      else becomes -1; *d_next advances by the starts taken.
 * Running every start at once: n_slots = n, d_slots = 0 .. n - 1, *d_next =
 * n (slots of stopped starts just empty).
 *   d_pose, d_grad [n][6], d_loss, d_last, d_t [n] FP32; d_m, d_v [n][6]
 *   FP32 (Adam state, zero at the start); d_alive [n] bytes (1 at the
 *   start); d_iters [n] int64; d_slots [n_slots] int32; d_next 1 int64;
 *   d_truth [n_truth][6] or NULL; d_hit_any 1 byte (needed with a truth);
 *   d_listed [n] bytes of scratch; prm host memory (copied into the launch).
 * Asynchronous, no allocation, capturable.  Errors: PROJ_E_ARG (NULL
 * pointers, negative sizes, n_truth not 1 or n, b1 or b2 outside [0, 1),
 * eps < 0), PROJ_E_CUDA. */
int proj_registration_step(int n, int n_slots, float *d_pose, const float *d_grad, const float *d_loss, float *d_last,
                           float *d_m, float *d_v, float *d_t, unsigned char *d_alive, long long *d_iters,
                           int *d_slots, long long *d_next, const float *d_truth, int n_truth,
                           unsigned char *d_hit_any, unsigned char *d_listed, const proj_reg_params *prm,
                           proj_stream stream);

/* Synchronise the stream, read and clear the workspace status word.
 * *status receives the PROJ_STATUS_* bits (may be NULL).  Returns PROJ_OK,
 * PROJ_E_DEVICE when a bit was set, or PROJ_E_CUDA. */
int proj_check(proj_plan plan, void *d_ws, size_t ws_bytes, proj_stream stream, int *status);

/* Ray samples |K_i| per instance for the given poses, counted on the
 * device by the same clipping and sample test the march kernels use (for
 * reporting samples/s).
 *   d_count  out [n_inst] int64. */
int proj_count_samples(proj_plan plan, const float *d_pose, long long *d_count, void *d_ws, size_t ws_bytes,
                       proj_stream stream);

/* Kernel timing for benchmarks.  While enabled, every call records two
 * CUDA events on its stream, immediately before and after its main kernels
 * (the march of proj_forward / proj_forward_pose_grad, the record pass and
 * voxel kernel of proj_back, the voxel kernel of proj_back_pose_grad, the
 * clearing, scatter and record-summing passes of the two transposes);
 * proj_kernel_time_ms waits for the second event and returns the elapsed
 * time of the last call's main kernels.  The events are created by the
 * first enable (not on the compute path). */
int proj_enable_kernel_timing(proj_plan plan, int enable);
int proj_kernel_time_ms(proj_plan plan, float *ms);

/* Forward pose gradient that allocates nothing (the paper has no
 * counterpart; this is a library facility).
 *
 * For callers that cannot allocate device memory - a plug-in whose host
 * application owns every allocation, a real-time loop whose memory is frozen
 * after start-up, code whose allocator is not CUDA's - and so can create
 * neither a plan nor a workspace.  The caller passes only inputs and outputs;
 * the geometry and instance maps are host data as in proj_plan_create.  All
 * scratch (tables, the prepared (mu, grad mu) volume, reduction records) is
 * one static device array of 6.2 MiB inside the library, which every GPU that
 * loads the library keeps until the process exits.
 *   Limits: pitched (mu, grad mu) volume of at most 74 x 70 x 68 (a 64^3 volume), n_inst, n_pose and
 *   n_views <= 64 each, n_inst x ceil(nu/16) x ceil(nv/16) <= 4096;
 *   larger sizes return PROJ_E_ARG with a message saying which limit.
 *   d_mu   [nz][ny][nx] FP32; d_pose, loss, d_ref, d_grad, d_loss as in
 *          proj_forward_pose_grad (d_loss may be NULL).
 * The result equals proj_forward_pose_grad's for the same inputs.  The first
 * call on a device looks up the array's device address (once per device,
 * with that device current) and caches it; make that first call before any
 * stream capture, and do not reset the device (cudaDeviceReset) after it.
 * Every call copies the host tables (views, instance maps) into the array
 * with cudaMemcpyAsync from pageable memory that lives only for the call, so
 * a call on a stream that is capturing a CUDA graph is refused with
 * PROJ_E_ARG before anything is enqueued.
 * Every call on a device shares the one array and overwrites it, so calls
 * that overlap on the GPU (other streams or threads) race: serialise them.
 * Non-finite poses give zero gradients (no status word is kept). */
int proj_forward_pose_grad_static(const proj_geometry *geom, int n_pose, int n_inst, const int *inst_view,
                                  const int *inst_pose, const float *d_mu, const float *d_pose, int loss,
                                  const float *d_ref, float *d_grad, float *d_loss, proj_stream stream);

/* Message of the last error in this thread ("" if none). */
const char *proj_last_error(void);

/* Library version string. */
const char *proj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PROJ_H */
