// Internal declarations of the sm_103a projector library (not part of the
// C ABI).  Device tables are rebuilt from the poses by the set-up kernel at
// the start of every call, in FP64, and stored in FP32 for the march and
// back-projection kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/proj.h"

namespace projk {

// Per-instance table (one (view, pose) pair), written by k_setup.
//   Ray-driven kernels: object-frame centred index coordinates of sample k
//   of pixel (iu, iv) are  f~_k = A + k * D,  D = (step / |d|) * d / vox,
//   d = C0 + iu * Uo + iv * Vo  (object-frame mm, R^T applied).
//   Voxel-driven kernels: (u', v', w') = Q[0:3] f~x + Q[3:6] f~y + Q[6:9] f~z
//   + Q[9:12] for a voxel at centred index f~ (Q = P [R | t] T_obj, stored
//   column by column), P3 = left 3x3 of P (row major) for the projection
//   Jacobian, w0 = w' of the world origin (FDK weight).
struct InstTable {
  float A[3];
  float C0[3];
  float Uo[3];
  float Vo[3];
  float Q[12];
  float P3[9];
  float w0;
  int view;
  int pose;
  int valid;
  int yfast;  // march the copy of the (mu, grad mu) volume whose rows run along y (detector u closer to y than x)
  int pad[2];
};
static_assert(sizeof(InstTable) == 40 * 4, "InstTable layout");

// Per-pose table in FP64: R (row major), t, dR/dg_j (j = x, y, z).
struct PoseTable {
  double R[9];
  double t[3];
  double dR[27];
  int valid;
  int pad;
};
static_assert(sizeof(PoseTable) % 8 == 0, "PoseTable layout");

// Static geometry shared by all kernels of a plan (passed by value).
struct Geo {
  int nx, ny, nz;       // voxels
  int px, py, pz;       // sizes with a 1-voxel border (n + 2): the cell records of mu (z rounded up to even)
  int qx, qy, qz;       // pitches of the (mu, grad mu) volume (2-voxel border, >= n + 4; qz even): element
                        // (x, y, z) at (((z >> 1) * qy + y) * qx + x) * 2 + (z & 1), i.e. x fastest with
                        // the two slices of a z pair interleaved element by element
  int rqx, rqy;         // pitches of its copy with y fastest: (((z >> 1) * rqx + x) * rqy + y) * 2 + (z & 1)
  float vx, vy, vz;     // voxel pitch, mm
  float hx, hy, hz;     // half extent of the open box (-1, n) in centred index units: (n+1)/2
  float gx, gy, gz;     // half extent of the gradient box (-2, n+1): (n+3)/2
  float cx, cy, cz;     // (n-1)/2
  float offx, offy, offz;
  int nu, nv;
  float step;
};

// Per-instance constants of FDK filtering: distance from the source to the
// plane through the isocentre parallel to the detector (sad), pixel pitches
// on that plane (du, dv) and the principal point in pixel indices (pu, pv).
struct FdkView {
  float sad, du, dv, pu, pv;
  float pad[3];
};

// Occupancy bricks for empty-space skipping in the marches.  Cells are
// those of the 2-voxel-bordered (mu, grad mu) grid (lower corner 0 .. n + 2
// per axis); a brick is 2^shift cells on a side.  Byte b of map is non-zero
// when brick b holds, or lies within one cell of, a cell with a non-zero
// corner in (mu, grad mu).  A sample whose cell has only zero corners adds
// exact zeros to every sum of the marches, so a ray's samples before the
// first and after the last occupied brick it crosses can be left out without
// changing any result.
//
// Inside that range the fused march tests each sample's own cell in the cell
// map (cells): bit (x & 31) of word (z * ch + y) * cw + (x >> 5) is set when
// cell (x, y, z) has a non-zero corner.  The test uses the march's own FP32
// position and cell of the sample, so the samples whose gathers it leaves out
// are exactly those that read eight zero corners.
struct Occ {
  const unsigned char* map;  // nullptr: no skipping
  int shift;                 // 3 (8-cell bricks) or 4 (16-cell bricks)
  int nb[3];                 // bricks per axis
  const unsigned* cells;     // cell map, or nullptr (brick ranges only)
  int cw, ch;                // words per row (x), rows per slice (y)
  const int* cells_flag;     // with cells: nullptr = always test; else test only when *cells_flag != 0
};
__host__ __device__ constexpr int occ_bricks(int n, int shift) { return (n + 3 + (1 << shift) - 1) >> shift; }
// Non-zero map of the (mu, grad mu) elements, one bit per element of the pitched grid, rows of
// nbits_words(qx) words, qy rows per slice, qz slices; and the cell map's words per row.
__host__ __device__ constexpr int nbits_words(int qx) { return (qx + 31) >> 5; }
__host__ __device__ constexpr int cell_words(int nx) { return (nx + 3 + 31) >> 5; }

// One problem of a persistent multi-problem fused march (proj_batch_*).
struct BatchProblem {
  Geo geo;
  const InstTable* inst;
  const float4* vol4;
  const float4* vol4y;  // y-fast copy, or null
  const float* ref;
  float* part;
  Occ occ;
  int n_tiles, tiles_u, loss, n_inst;
  long long item_begin;  // first global work item of this problem
};

// Optional per-call subset of a plan's poses for the fused march and its
// reduction (proj_forward_pose_grad_list).  With list == nullptr every
// instance of the plan is marched and every pose reduced.
struct PoseList {
  const int* list;      // device [n_list]: pose indices, or -1 for an empty slot
  int n_list;
  int ipp;              // most instances of any one pose (grid slots per listed pose)
  int n_pose;
  const int* pose_ptr;  // the plan's instances per pose (CSR)
  const int* pose_idx;
  int* status;          // PROJ_STATUS_BAD_INDEX for entries outside [-1, n_pose)
};

// Record of one K3 block (ray tile) partial: see kRec* offsets.
constexpr int kRec = 48;
constexpr int kRecG = 0;      // 12: sum of w * G   (RESIDUAL, L2)  or sum G (NCC)
constexpr int kRecLoss = 12;  // L2 loss partial
constexpr int kRecAG = 12;    // NCC: 12 sums l * G
constexpr int kRecBG = 24;    // NCC: 12 sums b * G
constexpr int kRecMom = 36;   // NCC: sum l, l^2, l b, b, b^2

// Ray tile of the march kernels: 16 x 16 pixels, 8 warps of 4 x 8.
constexpr int kTileU = 16;
constexpr int kTileV = 16;
constexpr int kMarchThreads = 256;

// Voxel-driven kernels: 32 x 8 columns per block, kZChunk voxels along z.
constexpr int kBpX = 32;
constexpr int kBpY = 8;
constexpr int kZChunk = 8;
constexpr int kBpThreads = kBpX * kBpY;
// Back-projection gradient: bricks of 32 x 8 x gz voxels (one thread per
// column of gz voxels), `views` instances per block; the shape is chosen per
// plan (proj_set_brick_shape, proj_autotune_back_grad):
//   0: gz 16, 8 views             1: gz 8, 8 views
//   2: gz 16, 16 views            3: gz 8, 16 views (default: fastest on the
//   motion-compensation workload, 24.9 vs 25.5 / 26.1 / 26.8 ms for 1 / 2 / 0)
constexpr int kGbX = 32;
constexpr int kGbY = 8;
constexpr int kBrickShapes = 4;
__host__ __device__ constexpr int brick_gz(int shape) { return (shape & 1) ? 8 : 16; }
__host__ __device__ constexpr int brick_views(int shape) { return shape >= 2 ? 16 : 8; }

// Launchers (defined in the .cu files; return cudaError_t of the launch).
cudaError_t launch_setup(const float* d_pose, int n_pose, const double* d_views, const int* d_inst_view,
                         const int* d_inst_pose, int n_inst, Geo geo, InstTable* d_inst, PoseTable* d_ptab,
                         int* d_status, cudaStream_t s);
// d_nbits (optional): the non-zero bits of (mu, grad mu), [qz][qy][nbits_words(qx)] words;
// d_vol4y (optional): the copy of (mu, grad mu) with rows along y (pitches rqx, rqy)
cudaError_t launch_volume_prep(const float* d_mu, Geo geo, float4* d_volq, float4* d_vol4, cudaStream_t s,
                               unsigned* d_nbits = nullptr, float4* d_vol4y = nullptr);
// the cell map, [nz + 3][ny + 3][cell_words(nx)] words, from the non-zero bits, then from it the
// occupancy bricks of both edges (8 and 16 cells; either map may be null); d_stat (2 counters and
// the flag, kCellStatBytes) receives the decision of the automatic cell test (see k_cell_decide)
constexpr int kCellStatBytes = 32;
cudaError_t launch_cell_bits(const unsigned* d_nbits, Geo geo, unsigned* d_cells, unsigned char* d_occ8,
                             unsigned char* d_occ16, void* d_stat, cudaStream_t s);
__host__ __device__ inline const int* cell_flag_of(const void* d_stat) {
  return reinterpret_cast<const int*>(static_cast<const char*>(d_stat) + 16);
}
// d_volqy: the copy of the cell records with rows along y (instances with yfast
// set march it), or null (all march d_volq)
cudaError_t launch_forward(const InstTable* d_inst, int n_inst, Geo geo, const float4* d_volq, const float4* d_volqy,
                           float* d_proj, cudaStream_t s, Occ occ = Occ{});
// grad_box 0: samples in the box (-1, n) of mu~ (the projector's sum); 1: samples the fused march gathers,
// those in the gradient grid's box (-2, n+1), clipped to the occupied bricks of occ when occ.map is set
cudaError_t launch_count(const InstTable* d_inst, int n_inst, Geo geo, long long* d_count, cudaStream_t s,
                         Occ occ = Occ{}, int grad_box = 0);
// warp_width: rays per warp row of the 16x16 tile (2, 4, 8 or 16; other values use 4)
// d_vol4y: the y-fast copy (instances with yfast set march it), or null (all march d_vol4)
// pl: optional pose subset (nullptr or pl->list == nullptr: all n_inst instances)
// d_volb: the bricked copy (PROJ_FLAG_BRICKS); when given, every instance marches it with 4 x 8 warps
cudaError_t launch_forward_grad(const InstTable* d_inst, int n_inst, Geo geo, const float4* d_vol4,
                                const float4* d_vol4y, int loss, const float* d_ref, float* d_proj, float* d_part,
                                cudaStream_t s, int warp_width = 4, const PoseList* pl = nullptr, Occ occ = Occ{},
                                const float4* d_volb = nullptr);
// the fused march's gathers without its arithmetic (empirical gather ceiling)
cudaError_t launch_gather_probe(const InstTable* d_inst, int n_inst, Geo geo, const float4* d_vol4,
                                const float4* d_vol4y, float* d_sink, cudaStream_t s, Occ occ = Occ{},
                                const float4* d_volb = nullptr);
// Bricked (mu, grad mu) volume (PROJ_FLAG_BRICKS): bricks of 4^3 cells of the 2-voxel-bordered grid, each
// holding the 5^3 elements at its cells' corners (a one-element apron on the upper faces, so the 8 corners
// of any cell sit at fixed offsets +1, +5, +25 from its lower corner), padded to 128 float4 (2 KB); brick
// (bx, by, bz) starts at element ((bz * vb_n(ny) + by) * vb_n(nx) + bx) * 128 and holds element (i, j, k)
// (0..4 each) at k * 25 + j * 5 + i.
__host__ __device__ constexpr int vb_n(int n) { return (n + 6) >> 2; }  // ceil((n + 3) / 4) bricks per axis
constexpr int kVbElems = 128;
cudaError_t launch_volume_bricks(const float4* d_vol4, Geo geo, float4* d_volb, cudaStream_t s);
// copy of the DRR march's cell records with rows along y (tiled transpose of every z slice)
cudaError_t launch_records_yfast(const float4* d_volq, Geo geo, float4* d_volqy, cudaStream_t s);
// d_pose_list: optional [n_list] poses to reduce (-1 = skip); nullptr = all n_pose
cudaError_t launch_forward_grad_reduce(const InstTable* d_inst, const PoseTable* d_ptab, int n_pose,
                                       const int* d_pose_ptr, const int* d_pose_idx, int n_tiles, Geo geo,
                                       int loss, const float* d_part, float* d_grad, float* d_loss,
                                       cudaStream_t s, const int* d_pose_list = nullptr, int n_list = 0);
// loss_all: the loss shared by every problem, or -1 for a batch of mixed losses
cudaError_t launch_forward_grad_batch(const BatchProblem* d_probs, int n_probs, long long n_items,
                                      unsigned long long* d_counter, int n_blocks, int loss_all, cudaStream_t s);
int forward_grad_batch_blocks_per_sm(int loss_all);
cudaError_t launch_forward_adjoint(const InstTable* d_inst, int n_inst, Geo geo, const float* d_y,
                                   float4* d_acc, float* d_vol, cudaStream_t s);
cudaError_t launch_detector_prep(const float* d_proj, int n_inst, Geo geo, float4* d_det4, cudaStream_t s);
// d_detq: detector cell records, [n_inst][nv+1][nu+1] float4 scratch
cudaError_t launch_back(const InstTable* d_inst, int n_inst, Geo geo, int weight, const float* d_proj,
                        float4* d_detq, float* d_vol, cudaStream_t s);
cudaError_t launch_back_adjoint(const InstTable* d_inst, int n_inst, Geo geo, int weight, const float* d_y,
                                float4* d_detq, float* d_proj, cudaStream_t s);
// shape: brick shape 0..3 (see brick_gz / brick_views); records per instance = back_grad_blocks(geo, shape)
cudaError_t launch_back_grad(const InstTable* d_inst, int n_inst, Geo geo, int weight, const float4* d_det4,
                             const float* d_wvol, float* d_part, int shape, cudaStream_t s);
cudaError_t launch_back_grad_reduce(const PoseTable* d_ptab, int n_pose, const int* d_pose_ptr,
                                    const int* d_pose_idx, int n_inst, int n_blocks, Geo geo, const float* d_part,
                                    float* d_grad, cudaStream_t s);

// Row and slice pitches (in float4 elements) of the (mu, grad mu) volume:
// at least n + 4 (2-voxel border), with qx = 2 (mod 8) and qx * qy = 4
// (mod 8), so the four (y, z) rows of a trilinear cell start 0, 32, 64 and
// 96 bytes into their 128-byte lines and a warp's corner gathers spread over
// all L1 data banks.  (Pitches that are whole lines cost up to 1.9x.)
inline void volume_pitches(int nx, int ny, int nz, int* qx, int* qy, int* qz) {
  int x = nx + 4;
  while (x % 8 != 2) ++x;
  int y = ny + 4;
  while ((x * y) % 8 != 4) ++y;
  *qx = x;
  *qy = y;
  *qz = (nz + 5) & ~1;  // even: z slices are stored in interleaved pairs
}

// z slices of the DRR march's cell records: n + 2, rounded up to even (pairs).
__host__ __device__ constexpr int record_slices(int nz) { return (nz + 3) & ~1; }

// The same rule for the copy whose rows run along y: row pitch (y) = 2 mod 8,
// slice pitch = 4 mod 8 (float4 units).
inline void volume_pitches_yfast(int nx, int ny, int* rqx, int* rqy) {
  int y = ny + 4;
  while (y % 8 != 2) ++y;
  int x = nx + 4;
  while ((x * y) % 8 != 4) ++x;
  *rqx = x;
  *rqy = y;
}

cudaError_t launch_fdk_filter(const FdkView* d_fv, int n_inst, Geo geo, float scale, const float* d_proj,
                              float* d_out, cudaStream_t s);
int sharpness_blocks(Geo geo);
cudaError_t launch_sharpness(const float* d_mu, Geo geo, float* d_m, double* d_part, double* d_stats, float* d_loss,
                             float* d_grad, cudaStream_t s);

// Sets the calling thread's message returned by proj_last_error().
void record_error(const char* msg);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Bricks (records per instance) of the back-projection gradient for a brick shape.
inline int back_grad_blocks(const Geo& g, int shape) {
  return ceil_div(g.nx, kGbX) * ceil_div(g.ny, kGbY) * ceil_div(g.nz, brick_gz(shape));
}

#ifdef __CUDACC__
// Two-wide FP32 arithmetic: sm_100 and later issue the same operation on a
// pair of 32-bit values as one instruction (PTX .f32x2).  The interpolating
// kernels apply it to pairs of channels that one 16-byte load leaves in
// adjacent registers.  Element by element the results are those of the
// scalar forms: lerp2(a, b, t).x == fmaf(t.x, b.x - a.x, a.x), add2 and
// mul2 are rounded adds and products, fma2 fused multiply-adds.
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 t) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rt, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rt, {%6, %7};\n\t"
      "sub.rn.f32x2 rd, rb, ra;\n\tfma.rn.f32x2 rd, rt, rd, ra;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(t.x), "f"(t.y));
  return r;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dup2(float s) { return make_float2(s, s); }

// Error-free FP32 accumulation (Knuth's two-sum): the running sum is hi + lo,
// lo collecting the exact rounding error of every add, so a fixed-order sum
// of FP32 values keeps about 48 significant bits.  The reductions use it in
// place of FP64 adds, which run at a small fraction of the FP32 rate here.
__device__ __forceinline__ void sum2_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}
#endif

}  // namespace projk
