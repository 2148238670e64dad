// Voxel-driven kernels: back-projection (Eq. back, Sec. II-C.2), the
// detector-gradient stencil (grad_d l by central differences) and the
// back-projection pose gradient (Eqs. back_derive, final_back, back_int,
// dis_back) with a deterministic two-stage reduction.
//
// Layout: a 256-thread block covers 32 (x) x 8 (y) voxel columns and
// kZChunk voxels along z; each warp covers 4 (x) x 8 (y) columns, so the 8
// lanes that the L1 data pipe serves together for 16-byte loads (a
// quarter-warp) form a 4 x 2 patch.  Whichever of x and y runs along the
// detector u axis in a view, that patch projects into a few neighbouring
// pixels; a row of 8 x-adjacent columns would spread over 16 pixels (two
// lines at the same bank slots) in the views where x runs along u.  Each
// thread projects its voxels with the instance's 3x4 matrix Q (centred voxel
// index -> (u',v',w')), one FMA chain per voxel.
#include <cstddef>

#include "proj_internal.cuh"

namespace projk {

namespace {

__device__ __forceinline__ float lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// Voxel column (x, y offsets in the block's 32 x 8 tile) of this thread:
// warp w takes x in [4w, 4w + 4), lane l takes x offset l & 3 and y = l >> 2.
__device__ __forceinline__ int col_x() { return ((threadIdx.x >> 5) << 2) + (threadIdx.x & 3); }
__device__ __forceinline__ int col_y() { return (threadIdx.x & 31) >> 2; }
static_assert(kBpX == 32 && kBpY == 8 && kGbX == 32 && kGbY == 8 && kBpThreads == 256,
              "col_x / col_y map 8 warps of 4 x 8 columns onto a 32 x 8 tile");

__device__ __forceinline__ float pix(const float* __restrict__ img, int nu, int nv, int iu, int iv) {
  return (iu >= 0 && iu < nu && iv >= 0 && iv < nv) ? __ldg(img + (size_t)iv * nu + iu) : 0.f;
}

// ---------------------------------------------------------------- K4
// (l, d_u l, d_v l, 0) with a 2-pixel border, [n_inst][nv+4][nu+4]: the
// central differences of the zero-padded image are non-zero up to one pixel
// outside the image and zero on the outer border.
// One thread per element of a row of the bordered float4 stack (x along u,
// row y = blockIdx.y, instance blockIdx.z; no integer division).
__global__ void k_detector_prep(const float* __restrict__ proj, int n_inst, Geo g, float4* __restrict__ det4) {
  const int qu = g.nu + 4, qv = g.nv + 4;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, in = blockIdx.z;
  if (x >= qu) return;
  const int iu = x - 2, iv = y - 2;
  const float* img = proj + (size_t)in * g.nu * g.nv;
  const float l = pix(img, g.nu, g.nv, iu, iv);
  const float du = 0.5f * (pix(img, g.nu, g.nv, iu + 1, iv) - pix(img, g.nu, g.nv, iu - 1, iv));
  const float dv = 0.5f * (pix(img, g.nu, g.nv, iu, iv + 1) - pix(img, g.nu, g.nv, iu, iv - 1));
  det4[((size_t)in * qv + y) * qu + x] = make_float4(l, du, dv, 0.f);
}

// Detector cell records, [n_inst][nv+1][nu+1] float4: record (x, y) holds
// the four pixels of the bilinear cell whose lower corner is pixel
// (x-1, y-1), (l(x-1, y-1), l(x, y-1), l(x-1, y), l(x, y)), zero outside the
// image, so a bilinear sample anywhere in (-1, nu) x (-1, nv) reads its 4
// corners with one 128-bit load and no edge tests.  With the FDK weight the
// records carry the instance's factor w0^2 of W = (w0 / w')^2 (k_back applies
// the per-voxel 1 / w'^2).
__global__ void k_detector_records(const float* __restrict__ proj, Geo g, const InstTable* __restrict__ inst,
                                   int weight, float4* __restrict__ detq) {
  const int ru = g.nu + 1, rv = g.nv + 1;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, in = blockIdx.z;
  if (x >= ru) return;
  const int iu = x - 1, iv = y - 1;
  const float* img = proj + (size_t)in * g.nu * g.nv;
  const float w0 = inst[in].w0, f = weight != PROJ_W_NONE ? w0 * w0 : 1.f;
  detq[((size_t)in * rv + y) * ru + x] =
      make_float4(f * pix(img, g.nu, g.nv, iu, iv), f * pix(img, g.nu, g.nv, iu + 1, iv),
                  f * pix(img, g.nu, g.nv, iu, iv + 1), f * pix(img, g.nu, g.nv, iu + 1, iv + 1));
}

// Pixel (i, j) = lane 0 of record (i+1, j+1), lane 1 of (i, j+1), lane 2 of
// (i+1, j) and lane 3 of (i, j): the transpose of k_detector_records, which
// gathers the back-projector transpose's record sums into [n_inst][nv][nu].
__global__ void k_detector_unrecord(const float4* __restrict__ detq, Geo g, float* __restrict__ proj) {
  const int ru = g.nu + 1, rv = g.nv + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, in = blockIdx.z;
  if (i >= g.nu) return;
  const float4* r = detq + ((size_t)in * rv + j) * ru + i;
  proj[((size_t)in * g.nv + j) * g.nu + i] = (__ldg(r + ru + 1).x + __ldg(r + ru).y) + (__ldg(r + 1).z + __ldg(r).w);
}

// Vector reduction (no return value): four FP32 adds to one 16-byte record.
__device__ __forceinline__ void red_add4(float4* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// Projection of the voxel-driven back-projection pair (k_back and its exact
// transpose k_back_adjoint share it): per instance and voxel column, the
// homogeneous pixel coordinates with 2 added to u and v (up = u + 2, vp = v +
// 2, folded into the instance's matrix), so that a voxel inside the image's
// bilinear support (u in (-1, nu), v in (-1, nv)) has up, vp in (1, n + 2).
// Q is read as three 16-byte loads (the tables are 256-byte aligned arrays of 160-byte entries).
static_assert(offsetof(InstTable, Q) % 16 == 0 && sizeof(InstTable) % 16 == 0, "InstTable::Q as float4");
// The column's values are taken at the chunk's first voxel, centred index
// fz0, so that voxel z of the chunk is (bu, bv, bw) + z (qz0, qz1, qz2).
__device__ __forceinline__ void bp_shifted(const InstTable& T, float fx, float fy, float fz0, float& bu, float& bv,
                                           float& bw, float& qz0, float& qz1, float& qz2) {
  const float4* q = reinterpret_cast<const float4*>(T.Q);
  const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);  // Q[0..3], Q[4..7], Q[8..11]
  qz2 = c.x;
  qz0 = fmaf(2.f, qz2, b.z);
  qz1 = fmaf(2.f, qz2, b.w);
  const float w = fmaf(b.y, fy, fmaf(a.z, fx, c.w));
  bu = fmaf(qz0, fz0, fmaf(2.f, w, fmaf(a.w, fy, fmaf(a.x, fx, c.y))));
  bv = fmaf(qz1, fz0, fmaf(2.f, w, fmaf(b.x, fy, fmaf(a.y, fx, c.z))));
  bw = fmaf(qz2, fz0, w);
}

// Detector cell record of (up, vp) in (1, n + 2): (floor(u) + 1, floor(v) + 1)
// and the bilinear fractions, without float-int conversions: for 1 <= x <
// 2^22 the sum x + (2^23 - 1/2) lies in [2^23, 2^24), where FP32 spacing is 1,
// so it rounds to 2^23 + RN(x - 1/2), whose low mantissa bits are floor(x)
// (floor(x) - 1 with fraction 1 at integers: the same bilinear value).  The
// record index is then (bits(tv) - 2^23's bits - 1) * ru + (bits(tu) - ... -
// 1), folded into koff.  __fadd_rn keeps the sum from being contracted with
// the product that formed up.
__device__ __forceinline__ unsigned bp_record(float up, float vp, unsigned ru, unsigned koff, float& au, float& av) {
  const float tu = __fadd_rn(up, 8388607.5f), tv = __fadd_rn(vp, 8388607.5f);
  au = up - (tu - 8388608.f);
  av = vp - (tv - 8388608.f);
  return __float_as_uint(tv) * ru + __float_as_uint(tu) - koff;
}

// ---------------------------------------------------------------- K5

__global__ void __launch_bounds__(kBpThreads) k_back(const InstTable* __restrict__ inst, int n_inst, Geo g,
                                                     int weight, const float4* __restrict__ detq,
                                                     float* __restrict__ vol) {
  const int ix = blockIdx.x * kBpX + col_x();
  const int iy = blockIdx.y * kBpY + col_y();
  const int iz0 = blockIdx.z * kZChunk;
  if (ix >= g.nx || iy >= g.ny) return;
  const float fx = (float)ix - g.cx, fy = (float)iy - g.cy, fz0 = (float)iz0 - g.cz;
  float acc[kZChunk];
#pragma unroll
  for (int z = 0; z < kZChunk; ++z) acc[z] = 0.f;
  const unsigned ru = (unsigned)g.nu + 1u, nu = (unsigned)g.nu, nv = (unsigned)g.nv;
  const bool fdk = weight != PROJ_W_NONE;
  for (int n = 0; n < n_inst; ++n) {
    const InstTable& T = inst[n];
    if (!T.valid) continue;
    float bu, bv, bw, qz0, qz1, qz2;
    bp_shifted(T, fx, fy, fz0, bu, bv, bw, qz0, qz1, qz2);
    const float4* rec = detq + (size_t)n * (g.nu + 1) * (g.nv + 1);
#pragma unroll
    for (int z = 0; z < kZChunk; ++z) {
      const float fz = (float)z;
      const float hw = fmaf(qz2, fz, bw);
      if (!(hw > 0.f)) continue;
      const float rw = __fdividef(1.0f, hw);  // fast reciprocal (about 2 ulp), the same in k_back and k_back_adjoint
      const float up = fmaf(qz0, fz, bu) * rw, vp = fmaf(qz1, fz, bv) * rw;
      // record (i, j) = (floor(u) + 1, floor(v) + 1) of u = up - 2, v = vp - 2 as in bp_record, and the
      // support test on it: i <= nu and j <= nv (unsigned) hold exactly when 1 < up < nu + 2 and
      // 1 < vp < nv + 2, but for up = nu + 2 (or vp = nv + 2) when the sum rounds to even below, where
      // the sample is the zero border pixel with weight 1 and adds +0; every up outside [1, 2^22),
      // negative, infinite or NaN gives an index far above nu
      const float tu = __fadd_rn(up, 8388607.5f), tv = __fadd_rn(vp, 8388607.5f);
      const unsigned i = __float_as_uint(tu) - 0x4B000001u, j = __float_as_uint(tv) - 0x4B000001u;
      if (i > nu || j > nv) continue;
      const float au = up - (tu - 8388608.f), av = vp - (tv - 8388608.f);
      const float4 q = __ldg(rec + j * ru + i);
      // the cell's two detector columns as a pair: lerp along v, then along u
      const float2 e = lerp2(lo2(q), hi2(q), dup2(av));
      const float val = lerp(e.x, e.y, au);
      // FDK: the record holds w0^2 l, times 1 / w'^2 here
      acc[z] = fdk ? fmaf(val, rw * rw, acc[z]) : acc[z] + val;
    }
  }
#pragma unroll
  for (int z = 0; z < kZChunk; ++z)
    if (iz0 + z < g.nz) vol[((size_t)(iz0 + z) * g.ny + iy) * g.nx + ix] = acc[z];
}

// ---------------------------------------------------------------- K6
//
// Per voxel j and instance n: rho = W rw (D_u P0 + D_v P1 - s P2) with rw =
// 1/w', s = D_u u + D_v v (+ 2 l~ for the FDK weight derivative), P0..P2 the
// rows of P's left 3x3: this is W (grad_d l) J_p + l~ grad W, the per-mm
// derivative of mu_j with respect to the moved voxel position.  With wj =
// dL/dmu_j the 12 sums wj rho and wj rho f~^T (f~ = centred voxel index)
// give dL/dM of the instance.
//
// Work decomposition: a block owns one brick of kGbX x kGbY x GZ voxels
// (one thread per (x, y) column holding its GZ residual weights in
// registers) and a chunk of VIEWS consecutive instances; blocks of the same
// chunk run together, so that chunk's detector stacks stay in L2.  The inner
// loop over z is branch-free - a voxel that projects outside the image or
// lies behind the source gets weight 0 and gathers from a valid address - so
// the gathers of several voxels can be in flight at once.  Per (brick,
// instance) one block reduction (a warp reduce-scatter, then the 8 warps in a
// fixed order) writes a record part[instance][brick][12].
//
// Arithmetic per voxel-view, kept short because the kernel issues about as
// many instructions as its gathers allow:
//  * projection straight into shifted pixel coordinates (up, vp) = (u + 3,
//    v + 3), one more than the padded stack's: the chunk's instance
//    constants are staged in shared memory with the +3 folded into Q, and
//    into the rows P0, P1 so that s can be formed from (up, vp) (D_u P0 +
//    D_v P1 - s P2 is unchanged when s -> s + 3 D_u + 3 D_v and P0 -> P0 +
//    3 P2, P1 -> P1 + 3 P2);
//  * the corner index and fractions without float-int conversions: for
//    1 <= x < 2^22 the sum x + (2^23 - 1/2) lies in [2^23, 2^24), where FP32
//    spacing is 1, so it rounds to 2^23 + RN(x - 1/2), whose low mantissa
//    bits are floor(x) (floor(x) - 1 with fraction 1 when x is an integer: the
//    same bilinear value); three adds per axis;
//  * the FDK factor w0^2 of W = (w0 rw)^2 applied once per record;
//  * since f~x and f~y are fixed for a thread, only sum rho and sum rho f~z
//    are accumulated per voxel (6 sums); the 12 follow per instance.
constexpr int kBgTab = 24;   // staged per-instance constants (floats), see k_back_grad

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Sum over the warp of 12 values per lane, as a reduce-scatter: after the
// two halving rounds lane l holds 3 partial sums, of values 6 (l >> 4 & 1) +
// 3 (l >> 3 & 1) + {0, 1, 2}; three butterfly rounds complete them.  Lanes
// with (l & 7) == 0 write their 3 sums to dst.  Fixed order: deterministic.
__device__ __forceinline__ void warp_sum12(const float (&v)[12], float* dst) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  float b[6], c[3];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float send = h16 ? v[i] : v[i + 6], keep = h16 ? v[i + 6] : v[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float send = h8 ? b[i] : b[i + 3], keep = h8 ? b[i + 3] : b[i];
    c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] += __shfl_xor_sync(0xffffffffu, c[i], o);
  if ((lane & 7) == 0) {
    const int base = (h16 ? 6 : 0) + (h8 ? 3 : 0);
    dst[base] = c[0];
    dst[base + 1] = c[1];
    dst[base + 2] = c[2];
  }
}

template <int GZ, int VIEWS>
__global__ void __launch_bounds__(kBpThreads, GZ <= 8 ? 4 : 3)
    k_back_grad(const InstTable* __restrict__ inst, int n_inst, Geo g, int weight, const float4* __restrict__ det4,
                const float* __restrict__ wvol, float* __restrict__ part, int bricks_x, int bricks_y) {
  // per instance of the chunk: Q with the +3 pixel shift folded in (columns x, y, z, constant; u, v, w each),
  // P0 + 3 P2, P1 + 3 P2, P2, the record factor (w0^2 or 1) and the valid flag
  __shared__ __align__(16) float tab[VIEWS][kBgTab];
  __shared__ float sred[2][kBpThreads / 32][12];
  const int warp = threadIdx.x >> 5;
  const int n_bricks = gridDim.x;
  const int brick = blockIdx.x;
  const int n0 = blockIdx.y * VIEWS, n1 = min(n_inst, n0 + VIEWS);
  if (threadIdx.x < n1 - n0) {
    const InstTable& T = inst[n0 + threadIdx.x];
    float* t = tab[threadIdx.x];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      t[3 * c + 0] = fmaf(3.f, T.Q[3 * c + 2], T.Q[3 * c + 0]);
      t[3 * c + 1] = fmaf(3.f, T.Q[3 * c + 2], T.Q[3 * c + 1]);
      t[3 * c + 2] = T.Q[3 * c + 2];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      t[12 + a] = fmaf(3.f, T.P3[6 + a], T.P3[a]);
      t[15 + a] = fmaf(3.f, T.P3[6 + a], T.P3[3 + a]);
      t[18 + a] = T.P3[6 + a];
    }
    t[21] = weight != PROJ_W_NONE ? T.w0 * T.w0 : 1.f;
    t[22] = T.valid ? 1.f : 0.f;
    t[23] = 0.f;
  }
  const int bx = brick % bricks_x, by = (brick / bricks_x) % bricks_y, bz = brick / (bricks_x * bricks_y);
  const int ix = bx * kGbX + col_x(), iy = by * kGbY + col_y(), iz0 = bz * GZ;
  const bool col = ix < g.nx && iy < g.ny;
  float wj[GZ];
#pragma unroll
  for (int z = 0; z < GZ; ++z)
    wj[z] = (col && iz0 + z < g.nz) ? __ldg(wvol + ((size_t)(iz0 + z) * g.ny + iy) * g.nx + ix) : 0.f;
  const float fx = (float)ix - g.cx, fy = (float)iy - g.cy, fz0 = (float)iz0 - g.cz;
  const unsigned qu = (unsigned)g.nu + 4u;
  // the float bits of 2^23 + i are 0x4B000000 + i; stack column = i - 1 (likewise rows)
  const unsigned koff = (0x4B000000u + 1u) * (qu + 1u);
  const size_t det_stride = (size_t)(g.nu + 4) * (g.nv + 4);
  const float ulim = (float)g.nu + 4.f, vlim = (float)g.nv + 4.f;
  __syncthreads();
  for (int n = n0; n < n1; ++n) {
    const float* t = tab[n - n0];
    float S0 = 0.f, S1 = 0.f, S2 = 0.f, T0 = 0.f, T1 = 0.f, T2 = 0.f;
    if (t[22] != 0.f && col) {
      const float4* img = det4 + (size_t)n * det_stride;
      const float bu = fmaf(t[3], fy, fmaf(t[0], fx, t[9]));
      const float bv = fmaf(t[4], fy, fmaf(t[1], fx, t[10]));
      const float bw = fmaf(t[5], fy, fmaf(t[2], fx, t[11]));
      const float qzu = t[6], qzv = t[7], qzw = t[8];
      const float P0x = t[12], P0y = t[13], P0z = t[14];
      const float P1x = t[15], P1y = t[16], P1z = t[17];
      const float P2x = t[18], P2y = t[19], P2z = t[20];
#pragma unroll
      for (int z = 0; z < GZ; ++z) {
        const float fz = fz0 + (float)z;
        const float hw = fmaf(qzw, fz, bw);
        const float rw = rcp_approx(hw);
        const float up0 = fmaf(qzu, fz, bu) * rw, vp0 = fmaf(qzv, fz, bv) * rw;
        // support of the interpolated gradient images: (-2, nu+1) x (-2, nv+1), i.e. 1 < up < nu + 4
        const bool ok = hw > 0.f && up0 > 1.f && up0 < ulim && vp0 > 1.f && vp0 < vlim;
        const float up = ok ? up0 : 3.5f, vp = ok ? vp0 : 3.5f;
        // __fadd_rn: never contracted with the product above, so the sum rounds the tested value of up
        const float tu = __fadd_rn(up, 8388607.5f), tv = __fadd_rn(vp, 8388607.5f);
        const float au = up - (tu - 8388608.f), av = vp - (tv - 8388608.f);
        const unsigned idx = __float_as_uint(tv) * qu + __float_as_uint(tu) - koff;
        const float4* p0 = img + idx;
        const float4 c00 = __ldg(p0), c10 = __ldg(p0 + 1), c01 = __ldg(p0 + qu), c11 = __ldg(p0 + qu + 1);
        const float L = lerp(lerp(c00.x, c10.x, au), lerp(c01.x, c11.x, au), av);
        const float Du = lerp(lerp(c00.y, c10.y, au), lerp(c01.y, c11.y, au), av);
        const float Dv = lerp(lerp(c00.z, c10.z, au), lerp(c01.z, c11.z, au), av);
        float sv = fmaf(Du, up, Dv * vp);
        if (weight == PROJ_W_FDK) sv = fmaf(2.f, L, sv);
        const float fw = weight != PROJ_W_NONE ? rw * rw * rw : rw;
        const float f = ok ? fw * wj[z] : 0.f;
        const float Duf = f * Du, Dvf = f * Dv, svf = f * sv;
        const float r0 = fmaf(Duf, P0x, fmaf(Dvf, P1x, -svf * P2x));
        const float r1 = fmaf(Duf, P0y, fmaf(Dvf, P1y, -svf * P2y));
        const float r2 = fmaf(Duf, P0z, fmaf(Dvf, P1z, -svf * P2z));
        S0 += r0;
        S1 += r1;
        S2 += r2;
        T0 = fmaf(r0, fz, T0);
        T1 = fmaf(r1, fz, T1);
        T2 = fmaf(r2, fz, T2);
      }
    }
    // a[0..2] = sum rho_a, a[3 + 3a + b] = sum rho_a f~_b
    const float a[12] = {S0, S1, S2, S0 * fx, S0 * fy, T0, S1 * fx, S1 * fy, T1, S2 * fx, S2 * fy, T2};
    float(*red)[12] = sred[(n - n0) & 1];
    warp_sum12(a, red[warp]);
    __syncthreads();
    if (threadIdx.x < 12) {
      float sq = 0.f;
      for (int w = 0; w < kBpThreads / 32; ++w) sq += red[w][threadIdx.x];
      part[((size_t)n * n_bricks + brick) * 12 + threadIdx.x] = sq * t[21];
    }
    // no second barrier: the next instance reduces into the other buffer, and the one after it
    // only after the next instance's barrier, which every reader of this buffer has passed
  }
}

// Per pose: fixed-order sum over bricks of its instances' records (each of
// 20 groups of bricks with the two-sum FP32 accumulation, the groups in FP64),
// conversion to dL/dM and contraction with dM/dtheta.
__global__ void k_back_grad_reduce(const PoseTable* __restrict__ ptab, const int* __restrict__ pose_ptr,
                                   const int* __restrict__ pose_idx, int n_inst, int n_blocks, Geo g,
                                   const float* __restrict__ part, float* __restrict__ grad) {
  constexpr int kGroups = 20;
  __shared__ double sp[kGroups][12];
  __shared__ double acc[12];
  const int p = blockIdx.x, t = threadIdx.x;
  if (t < 12) acc[t] = 0.0;
  __syncthreads();
  for (int e = pose_ptr[p]; e < pose_ptr[p + 1]; ++e) {
    const int n = pose_idx[e];
    if (t < kGroups * 12) {
      const int q = t % 12, grp = t / 12;
      float hi = 0.f, lo = 0.f;
#pragma unroll 4
      for (int b = grp; b < n_blocks; b += kGroups) sum2_add(hi, lo, part[((size_t)n * n_blocks + b) * 12 + q]);
      sp[grp][q] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (t < 12) {
      double s = 0.0;
      for (int grp = 0; grp < kGroups; ++grp) s += sp[grp][t];
      acc[t] += s;
    }
    __syncthreads();
  }
  if (t != 0) return;
  const PoseTable& P = ptab[p];
  float* out = grad + 6 * p;
  if (!P.valid) {
    for (int q = 0; q < 6; ++q) out[q] = 0.f;
    return;
  }
  // acc[0..2] = A0_a = sum w rho_a ; acc[3 + 3a + b] = sum w rho_a f~_b.
  const double off[3] = {g.offx, g.offy, g.offz};
  const double vox[3] = {g.vx, g.vy, g.vz};
  double gM[12];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) gM[4 * a + b] = off[b] * acc[a] + vox[b] * acc[3 + 3 * a + b];
    gM[4 * a + 3] = acc[a];
  }
  for (int a = 0; a < 3; ++a) out[a] = (float)gM[4 * a + 3];
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s += gM[4 * a + b] * P.dR[9 * j + 3 * a + b];
    out[3 + j] = (float)s;
  }
}

// ---------------------------------------------------------------- K8
// Exact transpose of k_back: each voxel spreads W * y_j over the 4 bilinear
// corners (inside the image) of its projection in every instance.  Output
// zeroed by the launcher; float atomics (order-dependent in the last bits).
__global__ void __launch_bounds__(kBpThreads) k_back_adjoint(const InstTable* __restrict__ inst, int n_inst, Geo g,
                                                             int weight, const float* __restrict__ y,
                                                             float4* __restrict__ detq) {
  const int ix = blockIdx.x * kBpX + (threadIdx.x & 31);
  const int iy = blockIdx.y * kBpY + (threadIdx.x >> 5);
  const int iz0 = blockIdx.z * kZChunk;
  if (ix >= g.nx || iy >= g.ny) return;
  const float fx = (float)ix - g.cx, fy = (float)iy - g.cy, fz0 = (float)iz0 - g.cz;
  float yv[kZChunk];
#pragma unroll
  for (int z = 0; z < kZChunk; ++z)
    yv[z] = (iz0 + z < g.nz) ? __ldg(y + ((size_t)(iz0 + z) * g.ny + iy) * g.nx + ix) : 0.f;
  const float ulim = (float)g.nu + 2.f, vlim = (float)g.nv + 2.f;
  const unsigned ru = (unsigned)g.nu + 1u, koff = (0x4B000000u + 1u) * (ru + 1u);
  for (int n = 0; n < n_inst; ++n) {
    const InstTable& T = inst[n];
    if (!T.valid) continue;
    float bu, bv, bw, qz0, qz1, qz2;
    bp_shifted(T, fx, fy, fz0, bu, bv, bw, qz0, qz1, qz2);
    float4* rec = detq + (size_t)n * (g.nu + 1) * (g.nv + 1);
#pragma unroll
    for (int z = 0; z < kZChunk; ++z) {
      if (yv[z] == 0.f) continue;
      const float fz = (float)z;
      const float hw = fmaf(qz2, fz, bw);
      if (!(hw > 0.f)) continue;
      const float rw = __fdividef(1.0f, hw);  // fast reciprocal (about 2 ulp), the same in k_back and k_back_adjoint
      const float up = fmaf(qz0, fz, bu) * rw, vp = fmaf(qz1, fz, bv) * rw;
      if (!(up > 1.f && up < ulim && vp > 1.f && vp < vlim)) continue;
      float au, av;
      const unsigned r = bp_record(up, vp, ru, koff, au, av);
      float val = yv[z];
      if (weight != PROJ_W_NONE) {
        const float r = T.w0 * rw;
        val *= r * r;
      }
      // the 4 corner weights go to record (i0 + 1, j0 + 1) in one vector
      // reduction; weights of corners outside the image land in border lanes
      // that k_detector_unrecord never reads
      red_add4(rec + r, val * (1.f - au) * (1.f - av), val * au * (1.f - av), val * (1.f - au) * av, val * au * av);
    }
  }
}


}  // namespace

cudaError_t launch_detector_prep(const float* d_proj, int n_inst, Geo geo, float4* d_det4, cudaStream_t s) {
  dim3 grid(ceil_div(geo.nu + 4, 128), geo.nv + 4, n_inst);
  k_detector_prep<<<grid, 128, 0, s>>>(d_proj, n_inst, geo, d_det4);
  return cudaGetLastError();
}

cudaError_t launch_back(const InstTable* d_inst, int n_inst, Geo geo, int weight, const float* d_proj,
                        float4* d_detq, float* d_vol, cudaStream_t s) {
  k_detector_records<<<dim3(ceil_div(geo.nu + 1, 128), geo.nv + 1, n_inst), 128, 0, s>>>(d_proj, geo, d_inst, weight,
                                                                                          d_detq);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(geo.nx, kBpX), ceil_div(geo.ny, kBpY), ceil_div(geo.nz, kZChunk));
  k_back<<<grid, kBpThreads, 0, s>>>(d_inst, n_inst, geo, weight, d_detq, d_vol);
  return cudaGetLastError();
}

cudaError_t launch_back_adjoint(const InstTable* d_inst, int n_inst, Geo geo, int weight, const float* d_y,
                                float4* d_detq, float* d_proj, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_detq, 0, sizeof(float4) * (size_t)n_inst * (geo.nu + 1) * (geo.nv + 1), s);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(geo.nx, kBpX), ceil_div(geo.ny, kBpY), ceil_div(geo.nz, kZChunk));
  k_back_adjoint<<<grid, kBpThreads, 0, s>>>(d_inst, n_inst, geo, weight, d_y, d_detq);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_detector_unrecord<<<dim3(ceil_div(geo.nu, 128), geo.nv, n_inst), 128, 0, s>>>(d_detq, geo, d_proj);
  return cudaGetLastError();
}

cudaError_t launch_back_grad(const InstTable* d_inst, int n_inst, Geo geo, int weight, const float4* d_det4,
                             const float* d_wvol, float* d_part, int shape, cudaStream_t s) {
  const int gz = brick_gz(shape), views = brick_views(shape);
  const int bx = ceil_div(geo.nx, kGbX), by = ceil_div(geo.ny, kGbY), bz = ceil_div(geo.nz, gz);
  dim3 grid(bx * by * bz, ceil_div(n_inst, views));  // = back_grad_blocks(geo, shape) records per instance
  switch (shape) {
    case 1: k_back_grad<8, 8><<<grid, kBpThreads, 0, s>>>(d_inst, n_inst, geo, weight, d_det4, d_wvol, d_part, bx, by); break;
    case 2: k_back_grad<16, 16><<<grid, kBpThreads, 0, s>>>(d_inst, n_inst, geo, weight, d_det4, d_wvol, d_part, bx, by); break;
    case 3: k_back_grad<8, 16><<<grid, kBpThreads, 0, s>>>(d_inst, n_inst, geo, weight, d_det4, d_wvol, d_part, bx, by); break;
    default: k_back_grad<16, 8><<<grid, kBpThreads, 0, s>>>(d_inst, n_inst, geo, weight, d_det4, d_wvol, d_part, bx, by); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_back_grad_reduce(const PoseTable* d_ptab, int n_pose, const int* d_pose_ptr,
                                    const int* d_pose_idx, int n_inst, int n_blocks, Geo geo, const float* d_part,
                                    float* d_grad, cudaStream_t s) {
  k_back_grad_reduce<<<n_pose, 256, 0, s>>>(d_ptab, d_pose_ptr, d_pose_idx, n_inst, n_blocks, geo, d_part, d_grad);
  return cudaGetLastError();
}

}  // namespace projk
