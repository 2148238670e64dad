// Ray-driven kernels: volume preparation (grad mu by central differences,
// Sec. II-C.1), forward projection (Eq. forward), the fused forward pose
// gradient (Eqs. for_grad, final_forward, for_int, dis_forward) with its
// deterministic reduction, the exact transpose of the forward projector and
// a sample counter.
//
// March layout: one thread per detector ray; a 256-thread block owns a
// 16 x 16 pixel tile of one instance and each warp a 4 x 8 sub-tile, so
// the 32 rays of a warp stay within a few voxels of each other at equal
// sample index k and their 8-corner gathers share cache lines.  Samples are
// anchored at world arc length k * step from the source (k integer), so a
// projection is a continuous function of the pose.
#include <algorithm>

#include "proj_internal.cuh"

namespace projk {

namespace {

__device__ __forceinline__ float lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// Warp sum of N values per lane (N a multiple of 8) as a reduce-scatter:
// three halving rounds (xor 16, 8, 4; each lane keeps the half its lane bit
// selects and adds its partner's copy of that half) leave each lane N / 8
// partial sums of values base + i, base = (lane & 16 ? N/2 : 0) +
// (lane & 8 ? N/4 : 0) + (lane & 4 ? N/8 : 0); butterflies over xor 2 and 1
// complete them, and lanes with (lane & 3) == 0 store them to dst[base + i].
// About 4N instead of 10N instructions for N separate warp sums; the fixed
// pattern keeps the result deterministic.
template <int N>
__device__ __forceinline__ void warp_sum_scatter(float (&v)[N], float* dst) {
  static_assert(N % 8 == 0, "N must be a multiple of 8");
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, m = N; o >= 4; o >>= 1, m >>= 1) {
    const bool hi = lane & o;
#pragma unroll
    for (int i = 0; i < m / 2; ++i) {
      const float send = hi ? v[i] : v[i + m / 2], keep = hi ? v[i + m / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 2; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < N / 8; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if ((lane & 3) == 0) {
    const int base = ((lane & 16) ? N / 2 : 0) + ((lane & 8) ? N / 4 : 0) + ((lane & 4) ? N / 8 : 0);
#pragma unroll
    for (int i = 0; i < N / 8; ++i) dst[base + i] = v[i];
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pixel of this thread inside the block's tile; false when outside the
// detector (ragged tiles).  Each warp takes a 4 x 8 pixel sub-tile, so each
// quarter-warp (the 8 lanes served together by the L1 data pipe for 16-byte
// loads) is a compact 4 x 2 patch of rays whose gathers share cache lines.
// WU is the warp's width in pixels (WU x 32/WU rays); 4 is the default, the
// other widths (2, 8, 16) serve the fused march's shape autotuner.
template <int WU = 4>
__device__ __forceinline__ bool tile_pixel(int tile, int tiles_u, const Geo& g, int& iu, int& iv) {
  static_assert(WU == 2 || WU == 4 || WU == 8 || WU == 16, "warp width");
  constexpr int WV = 32 / WU, kPerRow = kTileU / WU;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tu = tile % tiles_u, tv = tile / tiles_u;
  iu = tu * kTileU + (w % kPerRow) * WU + (lane % WU);
  iv = tv * kTileV + (w / kPerRow) * WV + (lane / WU);
  return iu < g.nu && iv < g.nv;
}

// Band-major block order for the marches and the forward transpose: the grid
// runs through every instance's tiles of one row of tiles before the next
// row.  Detector v runs along the orbit axis z, so the blocks resident at any
// time touch one slab of the volume's cell records, which stays in L2.
__device__ __forceinline__ void band_major_tile(int n_tiles, int tiles_u, int& n, int& tile) {
  const int n_inst = gridDim.x / n_tiles;
  const int b = blockIdx.x, tu = b % tiles_u, rest = b / tiles_u;
  n = rest % n_inst;
  tile = (rest / n_inst) * tiles_u + tu;
}

struct Ray {
  float ax, ay, az;  // padded index coordinates of the source (sample k = 0)
  float dx, dy, dz;  // index units per step
  int k0, k1;        // inclusive sample range inside the open box
};

// Ray through the centre of pixel (iu, iv) of instance T, clipped to the
// open index box (-m, n - 1 + m)^3 (centred: |f~| < (n - 1)/2 + m) with
// m = 1 (support of mu~) or m = 2 (support of the interpolated gradient
// grid); the returned sample origin is in index coordinates shifted by m
// (the border width of the array marched).  Returns false on a miss.
template <int M>
__device__ __forceinline__ bool ray_setup_m(const InstTable& T, const Geo& g, int iu, int iv, Ray& r) {
  const float fu = (float)iu, fv = (float)iv;
  const float dx = fmaf(fv, T.Vo[0], fmaf(fu, T.Uo[0], T.C0[0]));
  const float dy = fmaf(fv, T.Vo[1], fmaf(fu, T.Uo[1], T.C0[1]));
  const float dz = fmaf(fv, T.Vo[2], fmaf(fu, T.Uo[2], T.C0[2]));
  const float sc = g.step * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  r.dx = dx * sc / g.vx;
  r.dy = dy * sc / g.vy;
  r.dz = dz * sc / g.vz;
  float lo = 0.f, hi = 3.0e8f;
  const float A[3] = {T.A[0], T.A[1], T.A[2]};
  const float D[3] = {r.dx, r.dy, r.dz};
  const float H[3] = {M == 1 ? g.hx : g.gx, M == 1 ? g.hy : g.gy, M == 1 ? g.hz : g.gz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (fabsf(D[a]) > 1e-20f) {
      const float inv = 1.0f / D[a];
      const float t1 = (-H[a] - A[a]) * inv, t2 = (H[a] - A[a]) * inv;
      lo = fmaxf(lo, fminf(t1, t2));
      hi = fminf(hi, fmaxf(t1, t2));
    } else if (!(fabsf(A[a]) < H[a])) {
      return false;
    }
  }
  if (!(hi >= lo)) return false;
  r.k0 = (int)ceilf(lo);
  r.k1 = (int)floorf(hi);
  r.ax = A[0] + g.cx + (float)M;
  r.ay = A[1] + g.cy + (float)M;
  r.az = A[2] + g.cz + (float)M;
  return r.k1 >= r.k0;
}

__device__ __forceinline__ bool ray_setup(const InstTable& T, const Geo& g, int iu, int iv, Ray& r) {
  return ray_setup_m<1>(T, g, iu, iv, r);
}

// Empty-space skipping, first stage.  Narrows the inclusive sample range
// [k0, k1] of a ray to the samples between the first and the last occupied
// brick (Occ) that the ray crosses, widened by two samples at each end.
// Sample k sits at (ax, ay, az) + k (dx, dy, dz) in cell coordinates of the
// 2-voxel-bordered grid (cell c covers [c, c + 1)); (gx, gy, gz) = n + 2 is
// the largest cell index.  The walk steps from brick face to brick face in
// the sample parameter (a 3-D DDA) from sample k0 until it passes sample k1;
// no step waits on the occupancy byte it loads, so the loads of successive
// steps overlap.  Samples left out lie in bricks that hold no cell with a
// non-zero corner within one cell, so even with the rounding of their FP32
// positions they read eight zero corners and add exact zeros.  Returns false
// when no occupied brick is crossed.
__device__ __forceinline__ bool occ_bricks_clip(const Occ& o, float ax, float ay, float az, float dx, float dy,
                                                float dz, int gx, int gy, int gz, int& k0, int& k1) {
  const int sh = o.shift;
  const float edge = (float)(1 << sh), big = 3.0e30f;
  const float t0 = (float)k0, t1 = (float)k1;
  int bx = min(max(__float2int_rd(fmaf(t0, dx, ax)), 0), gx) >> sh;
  int by = min(max(__float2int_rd(fmaf(t0, dy, ay)), 0), gy) >> sh;
  int bz = min(max(__float2int_rd(fmaf(t0, dz, az)), 0), gz) >> sh;
  const int stx = dx > 0.f ? 1 : -1, sty = dy > 0.f ? 1 : -1, stz = dz > 0.f ? 1 : -1;
  // parameter of the next brick face along each axis, and the parameter span of one brick
  float tx = dx != 0.f ? ((float)((bx + (dx > 0.f ? 1 : 0)) << sh) - ax) / dx : big;
  float ty = dy != 0.f ? ((float)((by + (dy > 0.f ? 1 : 0)) << sh) - ay) / dy : big;
  float tz = dz != 0.f ? ((float)((bz + (dz > 0.f ? 1 : 0)) << sh) - az) / dz : big;
  const float ix = dx != 0.f ? edge / fabsf(dx) : big;
  const float iy = dy != 0.f ? edge / fabsf(dy) : big;
  const float iz = dz != 0.f ? edge / fabsf(dz) : big;
  float t_in = t0, t_first = 0.f, t_last = 0.f;
  bool found = false;
  const int max_steps = o.nb[0] + o.nb[1] + o.nb[2] + 3;
  for (int step = 0; step < max_steps; ++step) {
    const float t_out = fminf(tx, fminf(ty, tz));
    if (__ldg(o.map + (bz * o.nb[1] + by) * o.nb[0] + bx)) {
      if (!found) t_first = t_in;
      found = true;
      t_last = t_out;
    }
    if (t_out > t1) break;
    // step along the axis whose face comes first (x on ties, then y), without branches, so the
    // lanes of a warp stepping along different axes run the same instructions
    const bool ax_x = tx <= ty && tx <= tz, ax_y = !ax_x && ty <= tz, ax_z = !ax_x && !ax_y;
    bx += ax_x ? stx : 0;
    by += ax_y ? sty : 0;
    bz += ax_z ? stz : 0;
    tx += ax_x ? ix : 0.f;
    ty += ax_y ? iy : 0.f;
    tz += ax_z ? iz : 0.f;
    if ((unsigned)bx >= (unsigned)o.nb[0] || (unsigned)by >= (unsigned)o.nb[1] || (unsigned)bz >= (unsigned)o.nb[2])
      break;
    t_in = t_out;
  }
  if (!found) return false;
  k0 = max(k0, __float2int_rd(t_first) - 2);
  k1 = min(k1, __float2int_ru(fminf(t_last, t1)) + 2);
  return k0 <= k1;
}

// Brick stage of empty-space skipping for a march whose own sample origin is
// (ax, ay, az) in its own cell coordinates, with its cell clamp (lx, ly, lz):
// n + 2 for the (mu, grad mu) grid (rs = 0), n for the DRR march's
// 1-voxel-bordered records (rs = 1, its cells are one less than the bricks').
__device__ __forceinline__ bool occ_clip(const Occ& o, float ax, float ay, float az, float dx, float dy, float dz,
                                         int rs, int lx, int ly, int lz, int& k0, int& k1) {
  const float sr = (float)rs;
  // the bricks' grid is the 2-voxel-bordered one, largest cell n + 2 (= l + 2 rs for either march)
  return occ_bricks_clip(o, ax + sr, ay + sr, az + sr, dx, dy, dz, lx + 2 * rs, ly + 2 * rs, lz + 2 * rs, k0, k1);
}

// Cell stage, inside the marches: true when cell (cx, cy, cz) of the cell map
// (the march's cell plus rs) has a non-zero corner.  A sample in a cell
// without one reads eight zero corners and adds exact zeros, so the march
// leaves out its gathers and arithmetic and every sum is unchanged.
__device__ __forceinline__ bool cell_live(const Occ& o, int cx, int cy, int cz) {
  return (__ldg(o.cells + ((size_t)cz * o.ch + cy) * o.cw + (cx >> 5)) >> (cx & 31)) & 1u;
}

// Cell of padded index point (fx, fy, fz): lower corner clamped to
// [0, n] (1-voxel border) or [0, n + 2] (2-voxel border) so the 8 corners
// stay inside the padded array; fractions are taken from the clamped corner
// so that a point marginally outside the box (rounding) interpolates
// towards the zero border.  The lower clamp comes with the conversion: a
// float-to-unsigned conversion saturates, so a negative coordinate gives 0.
struct Cell {
  int idx;
  float ax, ay, az;
  int cx, cy, cz;  // the cell (lower corner after the clamp)
};

__device__ __forceinline__ Cell locate(float fx, float fy, float fz, const Geo& g) {
  const int ix = (int)min(__float2uint_rd(fx), (unsigned)(g.nx));
  const int iy = (int)min(__float2uint_rd(fy), (unsigned)(g.ny));
  const int iz = (int)min(__float2uint_rd(fz), (unsigned)(g.nz));
  Cell c;
  c.ax = fx - (float)ix;
  c.ay = fy - (float)iy;
  c.az = fz - (float)iz;
  c.idx = (iz * g.py + iy) * g.px + ix;
  c.cx = ix;
  c.cy = iy;
  c.cz = iz;
  return c;
}

// Cell records of the DRR march (YF = 0: rows along x; 1: the copy with rows
// along y), z slices interleaved in pairs as in the (mu, grad mu) volumes.
template <int YF>
__device__ __forceinline__ Cell locate_q(float fx, float fy, float fz, const Geo& g) {
  const int ix = (int)min(__float2uint_rd(fx), (unsigned)(g.nx));
  const int iy = (int)min(__float2uint_rd(fy), (unsigned)(g.ny));
  const int iz = (int)min(__float2uint_rd(fz), (unsigned)(g.nz));
  Cell c;
  c.ax = fx - (float)ix;
  c.ay = fy - (float)iy;
  c.az = fz - (float)iz;
  c.idx = YF ? ((((iz >> 1) * g.px + ix) * g.py + iy) << 1) + (iz & 1)
             : ((((iz >> 1) * g.py + iy) * g.px + ix) << 1) + (iz & 1);
  c.cx = ix;
  c.cy = iy;
  c.cz = iz;
  return c;
}

// YF = 0: the pitched (mu, grad mu) volume with x fastest; YF = 1: its copy
// with y fastest.  In both, the two slices of a z pair are interleaved element
// by element, so the two detector rows of a quarter-warp's 4 x 2 ray patch
// (v runs along z in a circular orbit) gather from neighbouring 16-byte slots;
// the +z corner is the neighbouring slot for an even slice and the next pair's
// slot for an odd one.
// YF = 2: either copy, chosen at run time through the element strides sx, sy
// (+1 voxel along x, y) and szp (+1 slice pair); the index equals that of
// YF = 0 or 1 for the same copy.  YF = 3: the bricked copy (vb_n).
template <int YF = 0>
__device__ __forceinline__ Cell locate2(float fx, float fy, float fz, const Geo& g, int sx = 0, int sy = 0,
                                        int szp = 0) {
  const int ix = (int)min(__float2uint_rd(fx), (unsigned)(g.nx + 2));
  const int iy = (int)min(__float2uint_rd(fy), (unsigned)(g.ny + 2));
  const int iz = (int)min(__float2uint_rd(fz), (unsigned)(g.nz + 2));
  Cell c;
  c.ax = fx - (float)ix;
  c.ay = fy - (float)iy;
  c.az = fz - (float)iz;
  if (YF == 3)
    c.idx = ((((iz >> 2) * vb_n(g.ny) + (iy >> 2)) * vb_n(g.nx) + (ix >> 2)) << 7) + (iz & 3) * 25 + (iy & 3) * 5 +
            (ix & 3);
  else if (YF == 2)
    c.idx = (iz >> 1) * szp + ix * sx + iy * sy + (iz & 1);
  else
    c.idx = YF ? ((((iz >> 1) * g.rqx + ix) * g.rqy + iy) << 1) + (iz & 1)
               : ((((iz >> 1) * g.qy + iy) * g.qx + ix) << 1) + (iz & 1);
  c.cx = ix;
  c.cy = iy;
  c.cz = iz;
  return c;
}

// ---------------------------------------------------------------- K1

// volq: mu with a 1-voxel zero border, (n+2)^3 cells, each cell holding the
// 2 x 2 corners of its xy face, (mu(x, y), mu(x+1, y), mu(x, y+1),
// mu(x+1, y+1)) at its own z, z slices interleaved in pairs: a trilinear
// sample reads its 8 corners as two 16-byte loads (this cell and the one
// above); launch_records_yfast then writes its copy with rows along y.
// vol4: (mu, grad mu) with a
// 2-voxel border, (n+4)^3; grad mu = central differences of the zero-padded
// volume, non-zero up to one voxel outside the grid and zero on the outer
// border layer.
// A block owns a 32 x 8 tile of (x, y) columns of the pitched (mu, grad mu)
// volume and walks a chunk of z slices, carrying mu at z - 1, z and z + 1 in
// registers: every voxel of mu is read once from DRAM (the x and y
// neighbours come from the slice the block just loaded, through L1).  The
// same thread writes the volq cell whose base corner is its element, where
// that falls inside volq's extent.  With vol4y the block also writes its tile
// of the copy with rows along y: each z pair of the tile is staged in shared
// memory and written as 32 runs of 16 elements (8 y x 2 slices, contiguous in
// that copy), so the copy costs its writes only.
constexpr int kPrepZChunk = 32;

__global__ void __launch_bounds__(256) k_volume_prep(const float* __restrict__ mu, Geo g, float4* __restrict__ volq,
                                                     float4* __restrict__ vol4, float4* __restrict__ vol4y,
                                                     unsigned* __restrict__ nbits) {
  // [y][slice of the pair][x]: the strides (66 and 33 float4) put the 8 elements that a quarter-warp
  // reads in the write-out (4 y x 2 slices of one x) on distinct bank groups
  __shared__ float4 stage[8][2][33];
  auto at = [&](int a, int b, int c) -> float {
    return (a >= 0 && a < g.nx && b >= 0 && b < g.ny && c >= 0 && c < g.nz)
               ? __ldg(mu + ((size_t)c * g.ny + b) * g.nx + a)
               : 0.0f;
  };
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x = blockIdx.x * 32 + tx, y = blockIdx.y * 8 + ty;
  const int z0 = blockIdx.z * kPrepZChunk, z1 = min(g.qz, z0 + kPrepZChunk);
  const int i = x - 2, j = y - 2;  // voxel column of this element
  const bool inq = x < g.qx && y < g.qy, in4 = vol4 && inq;
  const bool iny = x < g.rqx && y < g.rqy;
  // nbits: each warp (32 consecutive x of one row y) stores one word per z: bit = element non-zero
  const bool row_bits = nbits && y < g.qy && (int)blockIdx.x < nbits_words(g.qx);  // uniform per warp
  const int x1 = x - 1, y1 = y - 1;
  const bool in1xy = volq && x1 >= 0 && x1 < g.px && y1 >= 0 && y1 < g.py;
  float m_prev = at(i, j, z0 - 3), m = at(i, j, z0 - 2);
  const float sx = 0.5f / g.vx, sy = 0.5f / g.vy, sz = 0.5f / g.vz;
  for (int z = z0; z < z1; ++z) {
    const int k = z - 2;
    const float m_next = at(i, j, k + 1);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((inq && (vol4 || nbits)) || (vol4y && iny)) {
      v.x = m;
      v.y = (at(i + 1, j, k) - at(i - 1, j, k)) * sx;
      v.z = (at(i, j + 1, k) - at(i, j - 1, k)) * sy;
      v.w = (m_next - m_prev) * sz;
      if (in4) vol4[((((size_t)(z >> 1) * g.qy + y) * g.qx + x) << 1) + (z & 1)] = v;
    }
    if (row_bits) {
      const unsigned b = __ballot_sync(0xffffffffu, v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f);
      if (tx == 0) nbits[((size_t)z * g.qy + y) * nbits_words(g.qx) + blockIdx.x] = b;
    }
    if (vol4y) {  // uniform per block; z0 and z1 are even, so every pair is complete
      stage[ty][z & 1][tx] = v;
      if (z & 1) {
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = threadIdx.x + 256 * h, xl = e >> 4, yl = (e >> 1) & 7, zz = e & 1;
          const int xo = blockIdx.x * 32 + xl, yo = blockIdx.y * 8 + yl;
          if (xo < g.rqx && yo < g.rqy)
            vol4y[((((size_t)(z >> 1) * g.rqx + xo) * g.rqy + yo) << 1) + zz] = stage[yl][zz][xl];
        }
        __syncthreads();  // the next pair overwrites the stage
      }
    }
    const int zz1 = z - 1;
    if (in1xy && zz1 >= 0 && zz1 < g.pz)
      volq[((((size_t)(zz1 >> 1) * g.py + y1) * g.px + x1) << 1) + (zz1 & 1)] =
          make_float4(m, at(i + 1, j, k), at(i, j + 1, k), at(i + 1, j + 1, k));
    m_prev = m;
    m = m_next;
  }
}

// Cell map (Occ::cells): cell (x, y, z) of the 2-voxel-bordered grid has
// corners x..x+1, y..y+1, z..z+1, so its bit is the OR of the non-zero bits
// of those 8 elements: the OR of 4 rows (y, z pairs), then of bits x and x+1.
// One thread per word of the map.
// live counts the set bits (cells with a non-zero corner).
__global__ void k_cell_bits(const unsigned* __restrict__ nb, Geo g, unsigned* __restrict__ cells,
                            unsigned long long* __restrict__ live) {
  const int nw = nbits_words(g.qx), cw = cell_words(g.nx), ch = g.ny + 3;
  const long long n = (long long)cw * ch * (g.nz + 3);
  unsigned cnt = 0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(p % cw), y = (int)((p / cw) % ch), z = (int)(p / ((long long)cw * ch));
    // y + 1 <= ny + 3 < qy and z + 1 <= nz + 3 < qz: every row read exists
    auto rows = [&](int ww) -> unsigned {
      if (ww >= nw) return 0u;
      const unsigned* r = nb + ((size_t)z * g.qy + y) * nw + ww;
      const size_t slice = (size_t)g.qy * nw;
      return __ldg(r) | __ldg(r + nw) | __ldg(r + slice) | __ldg(r + slice + nw);
    };
    const unsigned r0 = rows(w), r1 = rows(w + 1);
    const unsigned word = r0 | (r0 >> 1) | (r1 << 31);
    cells[p] = word;
    cnt += __popc(word);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(live, (unsigned long long)cnt);
}

// Occupancy bricks (Occ) from the cell map: a brick of 8^3 cells is marked
// when a cell within one cell of it, i.e. in [8 b - 1, 8 b + 8] per axis
// (clipped to the grid), has a non-zero corner.  One warp per brick: its
// lanes take the (y, z) rows of that range (at most 100), each ORs the one or
// two map words the x range touches, and the warp votes.  For the automatic
// cell test the warps also add up the grid cells of the marked bricks
// (bricks on the far faces hold fewer than 512) into cell_stat[1].
__global__ void k_brick_maps8(const unsigned* __restrict__ cells, Geo g, unsigned char* __restrict__ occ8,
                              unsigned long long* __restrict__ cell_stat) {
  const int cw = cell_words(g.nx), ch = g.ny + 3;
  const int ex = g.nx + 3, ey = g.ny + 3, ez = g.nz + 3;  // cells per axis
  const int nb0 = occ_bricks(g.nx, 3), nb1 = occ_bricks(g.ny, 3);
  const int n8 = nb0 * nb1 * occ_bricks(g.nz, 3);
  const int lane = threadIdx.x & 31;
  unsigned long long counted = 0;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < n8; b += (gridDim.x * blockDim.x) >> 5) {
    const int bx = b % nb0, by = (b / nb0) % nb1, bz = b / (nb0 * nb1);
    const int x0 = max(8 * bx - 1, 0), x1 = min(8 * bx + 8, ex - 1);
    const int y0 = max(8 * by - 1, 0), y1 = min(8 * by + 8, ey - 1);
    const int z0 = max(8 * bz - 1, 0), z1 = min(8 * bz + 8, ez - 1);
    const int w0 = x0 >> 5, w1 = x1 >> 5;
    // bits x0 .. x1 of the words w0 .. w1 (at most two words: the range spans <= 10 cells)
    const unsigned m0 = (~0u << (x0 & 31)) & (w0 == w1 ? (~0u >> (31 - (x1 & 31))) : ~0u);
    const unsigned m1 = w0 == w1 ? 0u : (~0u >> (31 - (x1 & 31)));
    const int ny = y1 - y0 + 1, nrows = ny * (z1 - z0 + 1);
    unsigned any = 0;
    for (int r = lane; r < nrows; r += 32) {
      const unsigned* row = cells + ((size_t)(z0 + r / ny) * ch + (y0 + r % ny)) * cw;
      any |= (__ldg(row + w0) & m0) | (m1 ? (__ldg(row + w1) & m1) : 0u);
    }
    const bool marked = __any_sync(0xffffffffu, any != 0);
    if (lane == 0) {
      occ8[b] = marked ? 1 : 0;
      if (marked) counted += (unsigned long long)min(8, ex - 8 * bx) * min(8, ey - 8 * by) * min(8, ez - 8 * bz);
    }
  }
  if (lane == 0 && counted && cell_stat) atomicAdd(cell_stat + 1, counted);
}

// The 16^3 map from the 8^3 one: a 16^3 brick's cells within one cell,
// [16 B - 1, 16 B + 16], are exactly those of its eight 8^3 sub-bricks' ranges
// ([8 b - 1, 8 b + 8] for b = 2 B, 2 B + 1 per axis), so it is marked when
// one of them is (sub-bricks past the grid do not exist and count as empty).
__global__ void k_brick_maps16(const unsigned char* __restrict__ occ8, Geo g, unsigned char* __restrict__ occ16) {
  const int a0 = occ_bricks(g.nx, 3), a1 = occ_bricks(g.ny, 3), a2 = occ_bricks(g.nz, 3);
  const int nb0 = occ_bricks(g.nx, 4), nb1 = occ_bricks(g.ny, 4);
  const int n16 = nb0 * nb1 * occ_bricks(g.nz, 4);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n16; b += gridDim.x * blockDim.x) {
    const int bx = b % nb0, by = (b / nb0) % nb1, bz = b / (nb0 * nb1);
    unsigned char m = 0;
    for (int k = 2 * bz; k <= min(2 * bz + 1, a2 - 1); ++k)
      for (int j = 2 * by; j <= min(2 * by + 1, a1 - 1); ++j)
        for (int i = 2 * bx; i <= min(2 * bx + 1, a0 - 1); ++i) m |= occ8[(k * a1 + j) * a0 + i];
    occ16[b] = m ? 1 : 0;
  }
}

// Automatic cell test: the cell map pays off when a fair share of the cells
// inside the occupied 8^3 bricks has no non-zero corner (samples there are
// left out); on a dense volume every test is spent for nothing (measured: a
// uniformly filled volume marches about 12 % slower with the test).  The
// flag is set when the live cells (cell_stat[0], k_cell_bits) are at most
// 85 % of the grid cells of the occupied bricks (cell_stat[1], k_brick_maps).
__global__ void k_cell_decide(const unsigned long long* __restrict__ cell_stat, int* __restrict__ flag) {
  if (threadIdx.x == 0) *flag = (double)cell_stat[0] <= 0.85 * (double)cell_stat[1] ? 1 : 0;
}

// ---------------------------------------------------------------- K2

// Corners of a sample's cell: the xy face at z in one 16-byte cell record,
// the face at z + 1 in the record of the slice above (the neighbouring slot
// for an even slice, the next pair's slot for an odd one).  The DRR march
// skips by bricks only: with two gathers per sample, testing each sample's
// cell in the cell map costs more than it saves (measured on the
// registration phantom: 4.35 ms with bricks, 5.36 ms with the cell test).
template <int YF>
__device__ __forceinline__ float drr_ray(const InstTable& T, const Geo& g, int iu, int iv,
                                         const float4* __restrict__ volq, const Occ& occ) {
  float acc = 0.f;
  Ray r;
  if (!ray_setup(T, g, iu, iv, r)) return acc;
  // the records' 1-voxel border: cell coordinates of the 2-voxel-bordered grid are one more
  if (occ.map && !occ_clip(occ, r.ax, r.ay, r.az, r.dx, r.dy, r.dz, 1, g.nx, g.ny, g.nz, r.k0, r.k1))
    return acc;
  const int szp = 2 * g.px * g.py;
  // the sample index as a float pair (exact: |k| < 2^24): x and y of the position in one paired FMA
  const float2 one = dup2(1.f), d01 = make_float2(r.dx, r.dy), a01 = make_float2(r.ax, r.ay);
  float2 kk = dup2((float)r.k0);
  for (int k = r.k0; k <= r.k1; ++k, kk = add2(kk, one)) {
    const float2 f01 = fma2(kk, d01, a01);
    const Cell c = locate_q<YF>(f01.x, f01.y, fmaf(kk.x, r.dz, r.az), g);
    const float4 f0 = __ldg(volq + c.idx), f1 = __ldg(volq + c.idx + ((c.idx & 1) ? szp - 1 : 1));
    // the two x columns of the cell as a pair: lerp along y in each face, then along z, then along x
    const float2 ty = dup2(c.ay);
    const float2 e = lerp2(lerp2(lo2(f0), hi2(f0), ty), lerp2(lo2(f1), hi2(f1), ty), dup2(c.az));
    acc += lerp(e.x, e.y, c.ax);
  }
  return acc;
}

__global__ void __launch_bounds__(kMarchThreads) k_forward(const InstTable* __restrict__ inst, int n_tiles,
                                                           int tiles_u, Geo g, const float4* __restrict__ volq,
                                                           const float4* __restrict__ volqy, float* __restrict__ proj,
                                                           Occ occ) {
  int n, tile;
  band_major_tile(n_tiles, tiles_u, n, tile);
  int iu, iv;
  if (!tile_pixel(tile, tiles_u, g, iu, iv)) return;
  const InstTable& T = inst[n];
  float acc = 0.f;
  if (T.valid)
    acc = (volqy && T.yfast) ? drr_ray<1>(T, g, iu, iv, volqy, occ) : drr_ray<0>(T, g, iu, iv, volq, occ);
  proj[((size_t)n * g.nv + iv) * g.nu + iu] = g.step * acc;
}

// ---------------------------------------------------------------- count

// Samples per instance: grad_box 0, those in the open box (-1, n) of mu~
// (the sum of Eq. forward); grad_box 1, those the fused march gathers: the
// gradient grid's box (-2, n+1), clipped to the occupied bricks when occ.map
// is set, and of those only the samples whose cell has a non-zero corner when
// the cell test is on (occ.cells, and *occ.cells_flag if given).
__global__ void k_count(const InstTable* __restrict__ inst, int n_tiles, int tiles_u, Geo g,
                        unsigned long long* __restrict__ count, Occ occ, int grad_box) {
  const int n = blockIdx.x / n_tiles, tile = blockIdx.x % n_tiles;
  int iu, iv;
  unsigned long long c = 0;
  Ray r;
  if (tile_pixel(tile, tiles_u, g, iu, iv) && inst[n].valid) {
    if (!grad_box) {
      if (ray_setup(inst[n], g, iu, iv, r)) c = (unsigned long long)(r.k1 - r.k0 + 1);
    } else if (ray_setup_m<2>(inst[n], g, iu, iv, r) &&
               (!occ.map ||
                occ_clip(occ, r.ax, r.ay, r.az, r.dx, r.dy, r.dz, 0, g.nx + 2, g.ny + 2, g.nz + 2, r.k0, r.k1))) {
      if (occ.cells && (!occ.cells_flag || __ldg(occ.cells_flag))) {
        for (int k = r.k0; k <= r.k1; ++k) {
          const float kf = (float)k;
          const Cell cl = locate2(fmaf(kf, r.dx, r.ax), fmaf(kf, r.dy, r.ay), fmaf(kf, r.dz, r.az), g);
          c += cell_live(occ, cl.cx, cl.cy, cl.cz) ? 1 : 0;
        }
      } else {
        c = (unsigned long long)(r.k1 - r.k0 + 1);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count + n, c);
}

// ---------------------------------------------------------------- K3
//
// Per ray: a = sum_k mu~, S0 = sum_k g, S1[b][c] = sum_k g_b f~_c with
// g = interpolated central-difference gradient (per mm) and f~ the centred
// index coordinate of the sample, over the samples in the gradient grid's
// support (-2, n+1)^3 (mu~ is zero in the outer band, so a is unchanged).  Since r - t = R r' and r' = off + f~ vox,
// step * (S0, S1) determine the ray's dl/dM exactly (contraction in the
// reduction kernel).  At the end of the ray the loss residual weights the
// 12 sums; a warp/block reduction writes one record per tile.

// One 16 x 16 ray tile (instance n, tile index) of the fused march, block-
// wide: writes the tile's record part[(n * n_tiles + tile) * kRec ...].
// Shared by the per-problem kernel and the persistent multi-problem kernel.
// YF: 0 or 1, the copy marched (rows along x or y); 2, the copy named at run
// time by yf_rt, one code path for both (the persistent batch kernel, whose
// register budget does not hold two inlined marches).
template <int LOSS, int WU = 4, int YF = 0>
__device__ __forceinline__ void march_tile(const InstTable* __restrict__ inst, int n, int tile, int n_tiles,
                                           int tiles_u, const Geo& g, const float4* __restrict__ vol,
                                           const float* __restrict__ ref, float* __restrict__ proj,
                                           float* __restrict__ part, float (*red)[kRec], const Occ& occ,
                                           bool yf_rt = false) {
  int iu, iv;
  const bool on_det = tile_pixel<WU>(tile, tiles_u, g, iu, iv);
  const InstTable& T = inst[n];
  float a = 0.f;
  float s0[3] = {0.f, 0.f, 0.f};
  float s1[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  Ray r;
  bool live = on_det && T.valid && ray_setup_m<2>(T, g, iu, iv, r);
  // samples are numbered from the box entry kb whatever the skipping, so every kept sample's terms are
  // the same with skipping on or off
  const int kb = live ? r.k0 : 0;
  if (live && occ.map)
    live = occ_clip(occ, r.ax, r.ay, r.az, r.dx, r.dy, r.dz, 0, g.nx + 2, g.ny + 2, g.nz + 2, r.k0, r.k1);
  if (live) {
    // element strides of +1 voxel along x, y, z in the marched copy
    const bool yf = YF == 2 ? yf_rt : YF == 1;
    const bool cell_test = occ.cells && (!occ.cells_flag || __ldg(occ.cells_flag));
    // bricked copy: the corners sit at +1, +5, +25 inside the cell's brick
    const int sx = YF == 3 ? 1 : (yf ? 2 * g.rqy : 2), sy = YF == 3 ? 5 : (yf ? 2 : 2 * g.qx);
    const int szp = yf ? 2 * g.rqx * g.rqy : 2 * g.qx * g.qy;
    const float kbf = (float)kb;
    // sum_k g f~_k with f~_k = f~_kb + (k - kb) D: accumulate sum g and sum (k - kb) g, combine at the end.
    // The four channels run as two pairs, (mu, g_x) and (g_y, g_z): sums (a, s0x), (s0y, s0z), and
    // (-, tx), (ty, tz) (the first lane of the third pair accumulates mu (k - kb), unused).
    float2 A01 = make_float2(0.f, 0.f), A23 = A01, T01 = A01, T23 = A01;
    // the sample index as a float pair (exact: |k| < 2^24), so that x and y of the position and k - kb
    // come from paired instructions
    const float2 one = dup2(1.f), d01 = make_float2(r.dx, r.dy), a01 = make_float2(r.ax, r.ay), nkb = dup2(-kbf);
    float2 kk = dup2((float)r.k0);
    for (int k = r.k0; k <= r.k1; ++k, kk = add2(kk, one)) {
      const float2 f01 = fma2(kk, d01, a01);
      const Cell c = locate2<YF>(f01.x, f01.y, fmaf(kk.x, r.dz, r.az), g, sx, sy, szp);
      if (cell_test && !cell_live(occ, c.cx, c.cy, c.cz)) continue;
      const float4* p0 = vol + c.idx;
      const int sz = YF == 3 ? 25 : ((c.idx & 1) ? szp - 1 : 1);
      const float4 v000 = __ldg(p0), v100 = __ldg(p0 + sx);
      const float4 v010 = __ldg(p0 + sy), v110 = __ldg(p0 + sy + sx);
      const float4 v001 = __ldg(p0 + sz), v101 = __ldg(p0 + sz + sx);
      const float4 v011 = __ldg(p0 + sz + sy), v111 = __ldg(p0 + sz + sy + sx);
      // trilinear weights once per sample, then 8 two-wide FMAs per channel pair
      const float bx = 1.f - c.ax, by = 1.f - c.ay, bz = 1.f - c.az;
      const float w00 = bx * by, w10 = c.ax * by, w01 = bx * c.ay, w11 = c.ax * c.ay;
      const float q000 = w00 * bz, q100 = w10 * bz, q010 = w01 * bz, q110 = w11 * bz;
      const float q001 = w00 * c.az, q101 = w10 * c.az, q011 = w01 * c.az, q111 = w11 * c.az;
      float2 pa = mul2(dup2(q000), lo2(v000)), pb = mul2(dup2(q000), hi2(v000));  // (mu, g_x), (g_y, g_z)
      auto corner = [&](float q, const float4& v) {
        pa = fma2(dup2(q), lo2(v), pa);
        pb = fma2(dup2(q), hi2(v), pb);
      };
      corner(q100, v100);
      corner(q010, v010);
      corner(q110, v110);
      corner(q001, v001);
      corner(q101, v101);
      corner(q011, v011);
      corner(q111, v111);
      const float2 j = add2(kk, nkb);
      A01 = add2(A01, pa);
      A23 = add2(A23, pb);
      T01 = fma2(pa, j, T01);
      T23 = fma2(pb, j, T23);
    }
    a = A01.x;
    s0[0] = A01.y;
    s0[1] = A23.x;
    s0[2] = A23.y;
    const float t[3] = {T01.y, T23.x, T23.y};
    // centred index coordinates of sample kb
    const float fbx = fmaf(kbf, r.dx, r.ax) - (g.cx + 2.0f), fby = fmaf(kbf, r.dy, r.ay) - (g.cy + 2.0f),
                fbz = fmaf(kbf, r.dz, r.az) - (g.cz + 2.0f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      s1[3 * b + 0] = fmaf(r.dx, t[b], fbx * s0[b]);
      s1[3 * b + 1] = fmaf(r.dy, t[b], fby * s0[b]);
      s1[3 * b + 2] = fmaf(r.dz, t[b], fbz * s0[b]);
    }
  }
  const float l = g.step * a;
  const size_t pix = (size_t)iv * g.nu + iu;
  if (on_det && proj) proj[(size_t)n * g.nu * g.nv + pix] = l;

  float G[12];
  G[0] = g.step * s0[0];
  G[1] = g.step * s0[1];
  G[2] = g.step * s0[2];
#pragma unroll
  for (int q = 0; q < 9; ++q) G[3 + q] = g.step * s1[q];

  const int w = threadIdx.x >> 5;
  // the warp's part of the tile record, in record order (kRec* offsets), in one reduce-scatter
  if (LOSS == PROJ_LOSS_NCC) {
    const float b = on_det ? __ldg(ref + (size_t)T.view * g.nu * g.nv + pix) : 0.f;
    float v[kRec];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      v[kRecG + q] = G[q];
      v[kRecAG + q] = l * G[q];
      v[kRecBG + q] = b * G[q];
    }
    v[kRecMom + 0] = on_det ? l : 0.f;
    v[kRecMom + 1] = on_det ? l * l : 0.f;
    v[kRecMom + 2] = on_det ? l * b : 0.f;
    v[kRecMom + 3] = b;
    v[kRecMom + 4] = b * b;
#pragma unroll
    for (int q = kRecMom + 5; q < kRec; ++q) v[q] = 0.f;
    warp_sum_scatter<kRec>(v, red[w]);
  } else {
    float wt = 0.f, lossv = 0.f;
    if (on_det) {
      if (LOSS == PROJ_LOSS_RESIDUAL) {
        wt = __ldg(ref + (size_t)n * g.nu * g.nv + pix);
      } else {
        const float d = l - __ldg(ref + (size_t)T.view * g.nu * g.nv + pix);
        wt = 2.0f * d;
        lossv = d * d;
      }
    }
    float v[16];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[kRecG + q] = wt * G[q];
    v[kRecLoss] = lossv;
    v[13] = v[14] = v[15] = 0.f;
    warp_sum_scatter<16>(v, red[w]);
  }
  __syncthreads();
  const int nrec = (LOSS == PROJ_LOSS_NCC) ? (kRecMom + 5) : (kRecLoss + 1);
  if (threadIdx.x < kRec) {
    float s = 0.f;
    if ((int)threadIdx.x < nrec)
      for (int ww = 0; ww < kMarchThreads / 32; ++ww) s += red[ww][threadIdx.x];
    part[((size_t)n * n_tiles + tile) * kRec + threadIdx.x] = s;
  }
  __syncthreads();  // red is reused by the next tile of a persistent block
}

// Block -> (instance, tile) when a pose list selects the poses to march: the
// grid has n_list x ipp virtual instances (slot, j) per row of tiles, in the
// band-major order of band_major_tile; virtual instance (slot, j) is the j-th
// instance of pose list[slot].  Returns false for blocks with nothing to do.
__device__ __forceinline__ bool listed_tile(const PoseList& L, int n_tiles, int tiles_u, int& n, int& tile) {
  const int nv = L.n_list * L.ipp;
  const int b = blockIdx.x, tu = b % tiles_u, rest = b / tiles_u;
  const int q = rest % nv, slot = q / L.ipp, j = q % L.ipp;
  tile = (rest / nv) * tiles_u + tu;
  const int p = L.list[slot];
  if (p < 0) return false;
  if (p >= L.n_pose) {
    if (threadIdx.x == 0 && j == 0 && tile == 0) atomicOr(L.status, PROJ_STATUS_BAD_INDEX);
    return false;
  }
  const int e0 = L.pose_ptr[p];
  if (j >= L.pose_ptr[p + 1] - e0) return false;
  n = L.pose_idx[e0 + j];
  return true;
}

template <int LOSS, int WU>
__global__ void __launch_bounds__(kMarchThreads, 4)
    k_forward_grad(const InstTable* __restrict__ inst, int n_tiles, int tiles_u, Geo g,
                   const float4* __restrict__ vol, const float4* __restrict__ voly, const float* __restrict__ ref,
                   float* __restrict__ proj, float* __restrict__ part, PoseList L, Occ occ) {
  __shared__ float red[kMarchThreads / 32][kRec];
  int n, tile;
  if (L.list) {
    if (!listed_tile(L, n_tiles, tiles_u, n, tile)) return;  // uniform per block
  } else {
    band_major_tile(n_tiles, tiles_u, n, tile);
  }
  if (voly && inst[n].yfast)  // uniform per block
    march_tile<LOSS, WU, 1>(inst, n, tile, n_tiles, tiles_u, g, voly, ref, proj, part, red, occ);
  else
    march_tile<LOSS, WU, 0>(inst, n, tile, n_tiles, tiles_u, g, vol, ref, proj, part, red, occ);
}

// The fused march over the bricked copy (PROJ_FLAG_BRICKS), 4 x 8-pixel warps.
template <int LOSS>
__global__ void __launch_bounds__(kMarchThreads, 4)
    k_forward_grad_bricks(const InstTable* __restrict__ inst, int n_tiles, int tiles_u, Geo g,
                          const float4* __restrict__ volb, const float* __restrict__ ref, float* __restrict__ proj,
                          float* __restrict__ part, PoseList L, Occ occ) {
  __shared__ float red[kMarchThreads / 32][kRec];
  int n, tile;
  if (L.list) {
    if (!listed_tile(L, n_tiles, tiles_u, n, tile)) return;  // uniform per block
  } else {
    band_major_tile(n_tiles, tiles_u, n, tile);
  }
  march_tile<LOSS, 4, 3>(inst, n, tile, n_tiles, tiles_u, g, volb, ref, proj, part, red, occ);
}

// Bricked copy: one thread per element of a brick (128 per brick, 125 used);
// element (i, j, k) of brick (bx, by, bz) is element (4 bx + i, 4 by + j,
// 4 bz + k) of the pitched, pair-interleaved copy, zero outside it.
__global__ void k_volume_bricks(const float4* __restrict__ vol4, Geo g, float4* __restrict__ volb) {
  const int bnx = vb_n(g.nx), bny = vb_n(g.ny);
  const long long n = (long long)bnx * bny * vb_n(g.nz) * kVbElems;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(p & (kVbElems - 1));
    const long long b = p >> 7;
    const int bx = (int)(b % bnx), by = (int)((b / bnx) % bny), bz = (int)(b / ((long long)bnx * bny));
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < 125) {
      const int x = 4 * bx + e % 5, y = 4 * by + (e / 5) % 5, z = 4 * bz + e / 25;
      if (x < g.qx && y < g.qy && z < g.qz) v = __ldg(vol4 + ((((size_t)(z >> 1) * g.qy + y) * g.qx + x) << 1) + (z & 1));
    }
    volb[p] = v;
  }
}

// ---------------------------------------------------------------- gather probe
//
// The fused march's memory access pattern without its arithmetic: the same
// grid, pixel mapping, ray set-up, stepping, volume copy and the same eight
// 16-byte corner loads per sample (as volatile 128-bit loads, so none is
// dropped or narrowed), but only one add per load instead of the
// interpolation and accumulation.  Its duration is the empirical ceiling of
// the gather the fused march performs.

__device__ __forceinline__ float ld_probe(const float4* p) {
  float v[4];
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
  return v[0];
}

template <int YF>
__device__ __forceinline__ float probe_ray(const InstTable& T, const Geo& g, int iu, int iv, const float4* vol,
                                           const Occ& occ) {
  Ray r;
  float acc = 0.f;
  if (!(T.valid && ray_setup_m<2>(T, g, iu, iv, r))) return acc;
  if (occ.map && !occ_clip(occ, r.ax, r.ay, r.az, r.dx, r.dy, r.dz, 0, g.nx + 2, g.ny + 2, g.nz + 2, r.k0, r.k1))
    return acc;
  const int sx = YF == 3 ? 1 : (YF ? 2 * g.rqy : 2), sy = YF == 3 ? 5 : (YF ? 2 : 2 * g.qx);
  const int szp = YF ? 2 * g.rqx * g.rqy : 2 * g.qx * g.qy;
  const bool cell_test = occ.cells && (!occ.cells_flag || __ldg(occ.cells_flag));
  for (int k = r.k0; k <= r.k1; ++k) {
    const float kf = (float)k;
    const Cell c = locate2<YF>(fmaf(kf, r.dx, r.ax), fmaf(kf, r.dy, r.ay), fmaf(kf, r.dz, r.az), g);
    if (cell_test && !cell_live(occ, c.cx, c.cy, c.cz)) continue;
    const float4* p0 = vol + c.idx;
    const int sz = YF == 3 ? 25 : ((c.idx & 1) ? szp - 1 : 1);
    acc += ld_probe(p0) + ld_probe(p0 + sx) + ld_probe(p0 + sy) + ld_probe(p0 + sy + sx) + ld_probe(p0 + sz) +
           ld_probe(p0 + sz + sx) + ld_probe(p0 + sz + sy) + ld_probe(p0 + sz + sy + sx);
  }
  return acc;
}

__global__ void __launch_bounds__(kMarchThreads, 4)
    k_gather_probe(const InstTable* __restrict__ inst, int n_tiles, int tiles_u, Geo g, const float4* __restrict__ vol,
                   const float4* __restrict__ voly, float* __restrict__ sink, Occ occ,
                   const float4* __restrict__ volb) {
  int n, tile;
  band_major_tile(n_tiles, tiles_u, n, tile);  // the fused march's block order
  int iu, iv;
  const bool on = tile_pixel<4>(tile, tiles_u, g, iu, iv);
  float acc = 0.f;
  if (on)
    acc = volb ? probe_ray<3>(inst[n], g, iu, iv, volb, occ)
               : ((voly && inst[n].yfast) ? probe_ray<1>(inst[n], g, iu, iv, voly, occ)
                                          : probe_ray<0>(inst[n], g, iu, iv, vol, occ));
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0 && acc == 1.2345e-30f) sink[0] = acc;  // keeps the loads live; never taken in practice
}

// ---------------------------------------------------------------- batch
//
// Persistent multi-problem march: a grid of resident blocks takes work items
// (problem, instance, tile) from one atomic counter until the list is
// exhausted.  Items are numbered problem by problem in the order the host
// chose (longest tiles first), so small problems fill the tail of the large
// ones.  The counter is the only shared state; no block waits for another.

// LOSS >= 0: every problem of the batch has that loss (one march, either
// volume copy through run-time strides); LOSS < 0: each problem's own loss
// (3 variants, more registers).
template <int LOSS>
__global__ void __launch_bounds__(kMarchThreads, 4)
    k_forward_grad_batch(const BatchProblem* __restrict__ probs, int n_probs, long long n_items,
                         unsigned long long* __restrict__ counter) {
  __shared__ float red[kMarchThreads / 32][kRec];
  __shared__ long long item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(counter, 1ULL);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= n_items) return;
    int p = 0;
    while (p + 1 < n_probs && probs[p + 1].item_begin <= item) ++p;
    const BatchProblem& B = probs[p];
    // band-major within the problem, as in k_forward_grad
    const int local = (int)(item - B.item_begin), tu = local % B.tiles_u, rest = local / B.tiles_u;
    const int n = rest % B.n_inst, tile = (rest / B.n_inst) * B.tiles_u + tu;
    const bool yf = B.vol4y && B.inst[n].yfast;
    const float4* vol = yf ? B.vol4y : B.vol4;
    if constexpr (LOSS >= 0) {
      march_tile<LOSS, 4, 2>(B.inst, n, tile, B.n_tiles, B.tiles_u, B.geo, vol, B.ref, nullptr, B.part, red, B.occ, yf);
      continue;
    }
    switch (B.loss) {
      case PROJ_LOSS_RESIDUAL:
        march_tile<PROJ_LOSS_RESIDUAL, 4, 2>(B.inst, n, tile, B.n_tiles, B.tiles_u, B.geo, vol, B.ref, nullptr,
                                             B.part, red, B.occ, yf);
        break;
      case PROJ_LOSS_L2:
        march_tile<PROJ_LOSS_L2, 4, 2>(B.inst, n, tile, B.n_tiles, B.tiles_u, B.geo, vol, B.ref, nullptr, B.part,
                                       red, B.occ, yf);
        break;
      default:
        march_tile<PROJ_LOSS_NCC, 4, 2>(B.inst, n, tile, B.n_tiles, B.tiles_u, B.geo, vol, B.ref, nullptr, B.part,
                                        red, B.occ, yf);
        break;
    }
  }
}

// Per pose: sum the tile records of each of its instances in a fixed order
// (each of 21 groups of tiles with the two-sum FP32 accumulation, the groups
// and everything after in FP64), apply the loss (thread q < 12 keeps the sum
// of component q), convert the accumulator sums to dL/dM and contract with
// dM/dtheta.
constexpr int kReduceThreads = 1024;
__global__ void __launch_bounds__(kReduceThreads) k_forward_grad_reduce(const InstTable* __restrict__ inst, const PoseTable* __restrict__ ptab,
                                      const int* __restrict__ pose_ptr, const int* __restrict__ pose_idx,
                                      int n_tiles, Geo g, int loss, const float* __restrict__ part,
                                      float* __restrict__ grad, float* __restrict__ loss_out,
                                      const int* __restrict__ pose_list, int n_pose) {
  constexpr int kGroups = kReduceThreads / kRec;  // 21 groups of tiles summed side by side
  __shared__ double sp[kGroups][kRec];
  __shared__ double rec[kRec];
  __shared__ double accs[12];
  const int p = pose_list ? pose_list[blockIdx.x] : (int)blockIdx.x;
  if (p < 0 || p >= n_pose) return;  // empty slot (or an index the march reported)
  const int t = threadIdx.x;
  double acc = 0.0;  // component t of the 12 (threads 0..11)
  double L = 0.0;    // thread 0
  const int e0 = pose_ptr[p], e1 = pose_ptr[p + 1];
  const double np = (double)(e1 - e0);
  for (int e = e0; e < e1; ++e) {
    const int n = pose_idx[e];
    if (t < kGroups * kRec) {
      const int q = t % kRec, grp = t / kRec;
      float hi = 0.f, lo = 0.f;
#pragma unroll 4
      for (int tile = grp; tile < n_tiles; tile += kGroups) sum2_add(hi, lo, part[((size_t)n * n_tiles + tile) * kRec + q]);
      sp[grp][q] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (t < kRec) {
      double s = 0.0;
      for (int grp = 0; grp < kGroups; ++grp) s += sp[grp][t];
      rec[t] = s;
    }
    __syncthreads();
    // no barrier after this: the next instance writes sp, and rec only after its first barrier
    if (t < 12 && inst[n].valid) {
      if (loss == PROJ_LOSS_NCC) {
        const double N = (double)g.nu * g.nv;
        const double ma = rec[kRecMom] / N, mb = rec[kRecMom + 3] / N;
        const double A = rec[kRecMom + 2] - N * ma * mb;
        const double Va = rec[kRecMom + 1] - N * ma * ma;
        const double Vb = rec[kRecMom + 4] - N * mb * mb;
        if (Va > 0.0 && Vb > 0.0) {
          const double r = 1.0 / sqrt(Va * Vb);
          const double c2 = A * r / Va;
          const double gq = r * (rec[kRecBG + t] - mb * rec[kRecG + t]) - c2 * (rec[kRecAG + t] - ma * rec[kRecG + t]);
          acc -= gq / np;
          if (t == 0) L -= A * r / np;
        }
      } else {
        acc += rec[kRecG + t];
        if (t == 0 && loss == PROJ_LOSS_L2) L += rec[kRecLoss];
      }
    }
  }
  if (t < 12) accs[t] = acc;
  __syncthreads();
  if (t != 0) return;
  const PoseTable& P = ptab[p];
  float* out = grad + 6 * p;
  if (!P.valid) {
    for (int q = 0; q < 6; ++q) out[q] = 0.f;
    if (loss_out) loss_out[p] = 0.f;
    return;
  }
  // accs[0..2] = S0_b, accs[3 + 3b + c] = sum g_b f~_c.  T[b][c] = sum g_b r'_c.
  const double off[3] = {g.offx, g.offy, g.offz};
  const double vox[3] = {g.vx, g.vy, g.vz};
  double Tm[9];
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) Tm[3 * b + c] = off[c] * accs[b] + vox[c] * accs[3 + 3 * b + c];
  double gM[12];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) s += P.R[3 * a + c] * Tm[3 * b + c];
      gM[4 * a + b] = s;
    }
    gM[4 * a + 3] = -(P.R[3 * a] * accs[0] + P.R[3 * a + 1] * accs[1] + P.R[3 * a + 2] * accs[2]);
  }
  for (int a = 0; a < 3; ++a) out[a] = (float)gM[4 * a + 3];
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s += gM[4 * a + b] * P.dR[9 * j + 3 * a + b];
    out[3 + j] = (float)s;
  }
  if (loss_out) loss_out[p] = (float)L;
}

// ---------------------------------------------------------------- K7

// Vector reduction into global memory (no return value): four FP32 adds to
// one 16-byte-aligned record, one L2 operation.
__device__ __forceinline__ void red_add4(float4* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// The transpose scatters into cell records laid out like the forward march's
// (x fastest, no pair interleave): record (x, y, z) accumulates the weights of
// the four corners of cell (x, y, z)'s xy face, so a sample adds its 8
// corner weights with two vector reductions (its record and the record one
// slice up); k_unrecord then sums the four records that share each voxel.
__global__ void __launch_bounds__(kMarchThreads) k_forward_adjoint(const InstTable* __restrict__ inst, int n_tiles,
                                                                   int tiles_u, Geo g, const float* __restrict__ y,
                                                                   float4* __restrict__ acc) {
  int n, tile;
  band_major_tile(n_tiles, tiles_u, n, tile);
  int iu, iv;
  if (!tile_pixel(tile, tiles_u, g, iu, iv)) return;
  const InstTable& T = inst[n];
  const float yi = g.step * __ldg(y + ((size_t)n * g.nv + iv) * g.nu + iu);
  Ray r;
  if (yi == 0.f || !T.valid || !ray_setup(T, g, iu, iv, r)) return;
  const int pxy = g.px * g.py;
  // The 8 corner weights (corner q = offsets (q & 1, (q >> 1) & 1, q >> 2))
  // are summed in registers while the ray stays in one cell.  On a step to
  // the cell above or below, the shared face's record is the new cell's too,
  // so its 4 weights carry over and only the face left behind is reduced;
  // any other step reduces both faces.
  int cur = -1;
  float w[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto face = [&](int rec, int q) {
    red_add4(acc + rec, yi * w[q], yi * w[q + 1], yi * w[q + 2], yi * w[q + 3]);
  };
  for (int k = r.k0; k <= r.k1; ++k) {
    const float kf = (float)k;
    const Cell c = locate(fmaf(kf, r.dx, r.ax), fmaf(kf, r.dy, r.ay), fmaf(kf, r.dz, r.az), g);
    if (c.idx != cur) {
      const int d = c.idx - cur;
      if (cur < 0) {
      } else if (d == pxy) {
        face(cur, 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          w[q] = w[q + 4];
          w[q + 4] = 0.f;
        }
      } else if (d == -pxy) {
        face(cur + pxy, 4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          w[q + 4] = w[q];
          w[q] = 0.f;
        }
      } else {
        face(cur, 0);
        face(cur + pxy, 4);
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = 0.f;
      }
      cur = c.idx;
    }
    const float bx = 1.f - c.ax, by = 1.f - c.ay, bz = 1.f - c.az;
    w[0] += bx * by * bz;
    w[1] += c.ax * by * bz;
    w[2] += bx * c.ay * bz;
    w[3] += c.ax * c.ay * bz;
    w[4] += bx * by * c.az;
    w[5] += c.ax * by * c.az;
    w[6] += bx * c.ay * c.az;
    w[7] += c.ax * c.ay * c.az;
  }
  if (cur >= 0) {
    face(cur, 0);
    face(cur + pxy, 4);
  }
}

// Voxel (i, j, k) is padded point (i+1, j+1, k+1): corner 0 of record
// (i+1, j+1), corner 1 of record (i, j+1), corner 2 of record (i+1, j) and
// corner 3 of record (i, j), all in slice k+1.  Writes [nz][ny][nx].
__global__ void k_unrecord(const float4* __restrict__ acc, Geo g, float* __restrict__ vol) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((long long)g.nx * g.ny));
    const float4* a = acc + ((size_t)(k + 1) * g.py + j) * g.px + i;
    vol[p] = (__ldg(a + g.px + 1).x + __ldg(a + g.px).y) + (__ldg(a + 1).z + __ldg(a).w);
  }
}

int tiles_u_of(const Geo& g) { return ceil_div(g.nu, kTileU); }
int tiles_of(const Geo& g) { return ceil_div(g.nu, kTileU) * ceil_div(g.nv, kTileV); }

int elementwise_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 148LL * 64 ? (b < 1 ? 1 : b) : 148LL * 64);
}

}  // namespace

cudaError_t launch_volume_prep(const float* d_mu, Geo geo, float4* d_volq, float4* d_vol4, cudaStream_t s,
                               unsigned* d_nbits, float4* d_vol4y) {
  // the pitched extents (qx, qy, qz) exceed the 1-padded ones (n + 2) in every axis, and with the y-fast
  // copy the grid covers its pitches (rqx, rqy) too; blocks past nbits_words(qx) store no bits
  const int X = d_vol4y ? std::max(geo.qx, geo.rqx) : geo.qx, Y = d_vol4y ? std::max(geo.qy, geo.rqy) : geo.qy;
  dim3 grid(ceil_div(X, 32), ceil_div(Y, 8), ceil_div(geo.qz, kPrepZChunk));
  k_volume_prep<<<grid, 256, 0, s>>>(d_mu, geo, d_volq, d_vol4, d_vol4y, d_nbits);
  return cudaGetLastError();
}

cudaError_t launch_volume_bricks(const float4* d_vol4, Geo geo, float4* d_volb, cudaStream_t s) {
  k_volume_bricks<<<elementwise_grid((long long)vb_n(geo.nx) * vb_n(geo.ny) * vb_n(geo.nz) * kVbElems), 256, 0, s>>>(
      d_vol4, geo, d_volb);
  return cudaGetLastError();
}

cudaError_t launch_cell_bits(const unsigned* d_nbits, Geo geo, unsigned* d_cells, unsigned char* d_occ8,
                             unsigned char* d_occ16, void* d_stat, cudaStream_t s) {
  unsigned long long* stat = static_cast<unsigned long long*>(d_stat);
  cudaError_t e = cudaMemsetAsync(d_stat, 0, kCellStatBytes, s);
  if (e != cudaSuccess) return e;
  k_cell_bits<<<elementwise_grid((long long)cell_words(geo.nx) * (geo.ny + 3) * (geo.nz + 3)), 256, 0, s>>>(
      d_nbits, geo, d_cells, stat);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (d_occ8) {
    const long long n8 = (long long)occ_bricks(geo.nx, 3) * occ_bricks(geo.ny, 3) * occ_bricks(geo.nz, 3);
    k_brick_maps8<<<elementwise_grid(32 * n8), 256, 0, s>>>(d_cells, geo, d_occ8, stat);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (d_occ16) {
      const long long n16 = (long long)occ_bricks(geo.nx, 4) * occ_bricks(geo.ny, 4) * occ_bricks(geo.nz, 4);
      k_brick_maps16<<<elementwise_grid(n16), 256, 0, s>>>(d_occ8, geo, d_occ16);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  k_cell_decide<<<1, 32, 0, s>>>(stat, const_cast<int*>(cell_flag_of(d_stat)));
  return cudaGetLastError();
}

cudaError_t launch_forward(const InstTable* d_inst, int n_inst, Geo geo, const float4* d_volq, const float4* d_volqy,
                           float* d_proj, cudaStream_t s, Occ occ) {
  const int nt = tiles_of(geo);
  k_forward<<<n_inst * nt, kMarchThreads, 0, s>>>(d_inst, nt, tiles_u_of(geo), geo, d_volq, d_volqy, d_proj, occ);
  return cudaGetLastError();
}

cudaError_t launch_count(const InstTable* d_inst, int n_inst, Geo geo, long long* d_count, cudaStream_t s, Occ occ,
                         int grad_box) {
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(long long) * n_inst, s);
  if (e != cudaSuccess) return e;
  const int nt = tiles_of(geo);
  k_count<<<n_inst * nt, kMarchThreads, 0, s>>>(d_inst, nt, tiles_u_of(geo), geo,
                                                reinterpret_cast<unsigned long long*>(d_count), occ, grad_box);
  return cudaGetLastError();
}

namespace {
template <int WU>
void launch_forward_grad_w(const InstTable* d_inst, int grid, int nt, int tu, const Geo& geo, const float4* d_vol4,
                           const float4* d_vol4y, int loss, const float* d_ref, float* d_proj, float* d_part,
                           const PoseList& L, const Occ& occ, cudaStream_t s) {
  switch (loss) {
    case PROJ_LOSS_RESIDUAL:
      k_forward_grad<PROJ_LOSS_RESIDUAL, WU><<<grid, kMarchThreads, 0, s>>>(d_inst, nt, tu, geo, d_vol4, d_vol4y,
                                                                            d_ref, d_proj, d_part, L, occ);
      break;
    case PROJ_LOSS_L2:
      k_forward_grad<PROJ_LOSS_L2, WU><<<grid, kMarchThreads, 0, s>>>(d_inst, nt, tu, geo, d_vol4, d_vol4y, d_ref,
                                                                      d_proj, d_part, L, occ);
      break;
    default:
      k_forward_grad<PROJ_LOSS_NCC, WU><<<grid, kMarchThreads, 0, s>>>(d_inst, nt, tu, geo, d_vol4, d_vol4y, d_ref,
                                                                       d_proj, d_part, L, occ);
      break;
  }
}
}  // namespace

cudaError_t launch_forward_grad(const InstTable* d_inst, int n_inst, Geo geo, const float4* d_vol4,
                                const float4* d_vol4y, int loss, const float* d_ref, float* d_proj, float* d_part,
                                cudaStream_t s, int warp_width, const PoseList* pl, Occ occ, const float4* d_volb) {
  const int nt = tiles_of(geo), tu = tiles_u_of(geo);
  PoseList L{};
  if (pl && pl->list) L = *pl;
  const long long grid_ll = L.list ? (long long)L.n_list * L.ipp * nt : (long long)n_inst * nt;
  if (grid_ll < 1) return cudaSuccess;
  if (grid_ll > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const int grid = (int)grid_ll;
  if (d_volb) {
    if (loss == PROJ_LOSS_RESIDUAL)
      k_forward_grad_bricks<PROJ_LOSS_RESIDUAL><<<grid, kMarchThreads, 0, s>>>(d_inst, nt, tu, geo, d_volb, d_ref,
                                                                               d_proj, d_part, L, occ);
    else if (loss == PROJ_LOSS_L2)
      k_forward_grad_bricks<PROJ_LOSS_L2><<<grid, kMarchThreads, 0, s>>>(d_inst, nt, tu, geo, d_volb, d_ref, d_proj,
                                                                         d_part, L, occ);
    else
      k_forward_grad_bricks<PROJ_LOSS_NCC><<<grid, kMarchThreads, 0, s>>>(d_inst, nt, tu, geo, d_volb, d_ref, d_proj,
                                                                          d_part, L, occ);
    return cudaGetLastError();
  }
  switch (warp_width) {
    case 2: launch_forward_grad_w<2>(d_inst, grid, nt, tu, geo, d_vol4, d_vol4y, loss, d_ref, d_proj, d_part, L, occ, s); break;
    case 8: launch_forward_grad_w<8>(d_inst, grid, nt, tu, geo, d_vol4, d_vol4y, loss, d_ref, d_proj, d_part, L, occ, s); break;
    case 16:
      launch_forward_grad_w<16>(d_inst, grid, nt, tu, geo, d_vol4, d_vol4y, loss, d_ref, d_proj, d_part, L, occ, s);
      break;
    default: launch_forward_grad_w<4>(d_inst, grid, nt, tu, geo, d_vol4, d_vol4y, loss, d_ref, d_proj, d_part, L, occ, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_probe(const InstTable* d_inst, int n_inst, Geo geo, const float4* d_vol4,
                                const float4* d_vol4y, float* d_sink, cudaStream_t s, Occ occ, const float4* d_volb) {
  const int nt = tiles_of(geo);
  k_gather_probe<<<n_inst * nt, kMarchThreads, 0, s>>>(d_inst, nt, tiles_u_of(geo), geo, d_vol4, d_vol4y, d_sink,
                                                       occ, d_volb);
  return cudaGetLastError();
}

namespace {
constexpr int kTr = 32;

// One z slice tile of 32 x 32 (x, y) of a volume stored in interleaved z
// pairs: reads element (x, y, z) at (((z >> 1) * sqy + y) * sqx + x) * 2 + (z & 1)
// for x < X, y < Y (zero beyond), writes it at
// (((z >> 1) * dqx + x) * dqy + y) * 2 + (z & 1) for x < dqx, y < dqy: rows
// along x in, rows along y out.
__global__ void k_transpose_xy(const float4* __restrict__ v, int X, int Y, int sqx, int sqy, float4* __restrict__ vy,
                               int dqx, int dqy) {
  __shared__ float4 t[kTr][kTr + 1];
  const int x0 = blockIdx.x * kTr, y0 = blockIdx.y * kTr, z = blockIdx.z;
  for (int j = threadIdx.y; j < kTr; j += blockDim.y) {
    const int x = x0 + threadIdx.x, y = y0 + j;
    t[j][threadIdx.x] = (x < X && y < Y) ? v[((((size_t)(z >> 1) * sqy + y) * sqx + x) << 1) + (z & 1)]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < kTr; j += blockDim.y) {
    const int y = y0 + threadIdx.x, x = x0 + j;
    if (x < dqx && y < dqy) vy[((((size_t)(z >> 1) * dqx + x) * dqy + y) << 1) + (z & 1)] = t[threadIdx.x][j];
  }
}
}  // namespace

cudaError_t launch_records_yfast(const float4* d_volq, Geo geo, float4* d_volqy, cudaStream_t s) {
  dim3 grid(ceil_div(geo.px, kTr), ceil_div(geo.py, kTr), record_slices(geo.nz)), block(kTr, 8);
  k_transpose_xy<<<grid, block, 0, s>>>(d_volq, geo.px, geo.py, geo.px, geo.py, d_volqy, geo.px, geo.py);
  return cudaGetLastError();
}

cudaError_t launch_forward_grad_batch(const BatchProblem* d_probs, int n_probs, long long n_items,
                                      unsigned long long* d_counter, int n_blocks, int loss_all, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  switch (loss_all) {
    case PROJ_LOSS_RESIDUAL:
      k_forward_grad_batch<PROJ_LOSS_RESIDUAL><<<n_blocks, kMarchThreads, 0, s>>>(d_probs, n_probs, n_items, d_counter);
      break;
    case PROJ_LOSS_L2:
      k_forward_grad_batch<PROJ_LOSS_L2><<<n_blocks, kMarchThreads, 0, s>>>(d_probs, n_probs, n_items, d_counter);
      break;
    case PROJ_LOSS_NCC:
      k_forward_grad_batch<PROJ_LOSS_NCC><<<n_blocks, kMarchThreads, 0, s>>>(d_probs, n_probs, n_items, d_counter);
      break;
    default:
      k_forward_grad_batch<-1><<<n_blocks, kMarchThreads, 0, s>>>(d_probs, n_probs, n_items, d_counter);
      break;
  }
  return cudaGetLastError();
}

int forward_grad_batch_blocks_per_sm(int loss_all) {
  int b = 0;
  cudaError_t e;
  switch (loss_all) {
    case PROJ_LOSS_RESIDUAL:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_grad_batch<PROJ_LOSS_RESIDUAL>, kMarchThreads, 0);
      break;
    case PROJ_LOSS_L2:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_grad_batch<PROJ_LOSS_L2>, kMarchThreads, 0);
      break;
    case PROJ_LOSS_NCC:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_grad_batch<PROJ_LOSS_NCC>, kMarchThreads, 0);
      break;
    default:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_forward_grad_batch<-1>, kMarchThreads, 0);
      break;
  }
  if (e != cudaSuccess) b = 2;
  return b < 1 ? 1 : b;
}

cudaError_t launch_forward_grad_reduce(const InstTable* d_inst, const PoseTable* d_ptab, int n_pose,
                                       const int* d_pose_ptr, const int* d_pose_idx, int n_tiles, Geo geo,
                                       int loss, const float* d_part, float* d_grad, float* d_loss,
                                       cudaStream_t s, const int* d_pose_list, int n_list) {
  const int blocks = d_pose_list ? n_list : n_pose;
  if (blocks < 1) return cudaSuccess;
  k_forward_grad_reduce<<<blocks, kReduceThreads, 0, s>>>(d_inst, d_ptab, d_pose_ptr, d_pose_idx, n_tiles, geo, loss, d_part,
                                               d_grad, d_loss, d_pose_list, n_pose);
  return cudaGetLastError();
}

cudaError_t launch_forward_adjoint(const InstTable* d_inst, int n_inst, Geo geo, const float* d_y, float4* d_acc,
                                   float* d_vol, cudaStream_t s) {
  const long long npad = (long long)geo.px * geo.py * geo.pz;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, sizeof(float4) * npad, s);
  if (e != cudaSuccess) return e;
  const int nt = tiles_of(geo);
  k_forward_adjoint<<<n_inst * nt, kMarchThreads, 0, s>>>(d_inst, nt, tiles_u_of(geo), geo, d_y, d_acc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)geo.nx * geo.ny * geo.nz;
  k_unrecord<<<elementwise_grid(n), 256, 0, s>>>(d_acc, geo, d_vol);
  return cudaGetLastError();
}

}  // namespace projk
