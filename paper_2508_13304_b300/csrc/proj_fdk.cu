// Motion-compensated FDK pieces: projection filtering (cosine pre-weight and
// Ram-Lak ramp filter along detector rows, the "Ramp(l)" of the motion-
// compensated reconstruction experiment, Sec. II-D.3) and the image
// sharpness loss -Var(|grad mu|) with its gradient with respect to mu.
#include "proj_internal.cuh"

namespace projk {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kFiltThreads = 256;

// Ram-Lak taps in units of 1 / du^2: h[0] = 1/4, h[k] = -1/(pi k)^2 for odd k,
// 0 for even k != 0 (spatial form of the band-limited ramp).
__device__ __forceinline__ float ramlak(int k) {
  if (k == 0) return 0.25f;
  if ((k & 1) == 0) return 0.f;
  const float pk = (float)kPi * (float)k;
  return -1.0f / (pk * pk);
}

// One block per detector row: q(u) = scale * du * sum_k x(k) h(u - k) / du^2
// with x = l * cos weight, du the pixel pitch on the isocentre plane.
__global__ void __launch_bounds__(kFiltThreads) k_fdk_filter(const FdkView* __restrict__ fv, int nu, int nv,
                                                             float scale, const float* __restrict__ proj,
                                                             float* __restrict__ out) {
  extern __shared__ float row[];
  const int r = blockIdx.x;              // instance * nv + iv
  const int n = r / nv, iv = r % nv;
  const FdkView V = fv[n];
  const float* src = proj + (size_t)r * nu;
  const float b = ((float)iv - V.pv) * V.dv;            // isocentre-plane offsets, mm
  for (int u = threadIdx.x; u < nu; u += blockDim.x) {
    const float a = ((float)u - V.pu) * V.du;
    row[u] = __ldg(src + u) * V.sad * rsqrtf(V.sad * V.sad + a * a + b * b);
  }
  __syncthreads();
  const float f = scale / V.du;          // du * (1 / du^2)
  for (int u = threadIdx.x; u < nu; u += blockDim.x) {
    float acc = 0.25f * row[u];
    // odd offsets only (even taps are zero)
    for (int k = 1; k < nu; k += 2) {
      const float h = ramlak(k);
      float s = 0.f;
      if (u - k >= 0) s += row[u - k];
      if (u + k < nu) s += row[u + k];
      acc = fmaf(h, s, acc);
    }
    out[(size_t)r * nu + u] = f * acc;
  }
}

// ---------------------------------------------------------------- sharpness

__device__ __forceinline__ float vat(const float* __restrict__ mu, const Geo& g, int i, int j, int k) {
  return (i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz)
             ? __ldg(mu + ((size_t)k * g.ny + j) * g.nx + i)
             : 0.f;
}

// |grad mu| per voxel (central differences of the zero-padded volume, per
// mm) into m, and per-block FP64 sums of m and m^2.
__global__ void k_sharp_magnitude(const float* __restrict__ mu, Geo g, float* __restrict__ m,
                                  double* __restrict__ part) {
  __shared__ double sm[2][8];
  const long long n = (long long)g.nx * g.ny * g.nz;
  const float sx = 0.5f / g.vx, sy = 0.5f / g.vy, sz = 0.5f / g.vz;
  double s1 = 0.0, s2 = 0.0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((long long)g.nx * g.ny));
    const float gx = (vat(mu, g, i + 1, j, k) - vat(mu, g, i - 1, j, k)) * sx;
    const float gy = (vat(mu, g, i, j + 1, k) - vat(mu, g, i, j - 1, k)) * sy;
    const float gz = (vat(mu, g, i, j, k + 1) - vat(mu, g, i, j, k - 1)) * sz;
    const float v = sqrtf(fmaf(gx, gx, fmaf(gy, gy, gz * gz)));
    m[p] = v;
    s1 += v;
    s2 += (double)v * v;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sm[0][w] = s1;
    sm[1][w] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a += sm[0][q];
      b += sm[1][q];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// Fixed-order sum of the block partials: mean of m and S = -Var(m).
__global__ void k_sharp_stats(const double* __restrict__ part, int n_blocks, long long n, double* __restrict__ stats,
                              float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < n_blocks; ++q) {
    a += part[2 * q];
    b += part[2 * q + 1];
  }
  const double mean = a / (double)n;
  const double var = b / (double)n - mean * mean;
  stats[0] = mean;
  if (loss) *loss = (float)(-var);
}

// dS/dmu_j = -(2/N) sum_a [c_a(j - e_a) - c_a(j + e_a)] / (2 v_a), with
// c_a(i) = (m_i - mean) g_a(i) / m_i for voxels i of the grid (0 where
// m_i < 1e-12): the chain rule through m_i = |g(i)| and the central
// differences g_a(i) = (mu[i + e_a] - mu[i - e_a]) / (2 v_a).
__global__ void k_sharp_grad(const float* __restrict__ mu, const float* __restrict__ m, Geo g,
                             const double* __restrict__ stats, float* __restrict__ grad) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const float mean = (float)stats[0];
  const float coef = (float)(-2.0 / (double)n);
  const float inv2[3] = {0.5f / g.vx, 0.5f / g.vy, 0.5f / g.vz};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((long long)g.nx * g.ny));
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int dx = (a == 0), dy = (a == 1), dz = (a == 2);
#pragma unroll
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const int ii = i + sgn * dx, jj = j + sgn * dy, kk = k + sgn * dz;
        if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
        const float mi = __ldg(m + ((size_t)kk * g.ny + jj) * g.nx + ii);
        if (!(mi >= 1e-12f)) continue;
        const float ga = (vat(mu, g, ii + dx, jj + dy, kk + dz) - vat(mu, g, ii - dx, jj - dy, kk - dz)) * inv2[a];
        const float c = (mi - mean) * ga / mi;
        // the neighbour at j - e_a (sgn = -1) has j as its +e_a neighbour
        acc += (sgn < 0 ? c : -c) * inv2[a];
      }
    }
    grad[p] = coef * acc;
  }
}

int elementwise_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 148LL * 64 ? (b < 1 ? 1 : b) : 148LL * 64);
}

}  // namespace

cudaError_t launch_fdk_filter(const FdkView* d_fv, int n_inst, Geo geo, float scale, const float* d_proj,
                              float* d_out, cudaStream_t s) {
  const size_t smem = sizeof(float) * geo.nu;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fdk_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fdk_filter<<<n_inst * geo.nv, kFiltThreads, smem, s>>>(d_fv, geo.nu, geo.nv, scale, d_proj, d_out);
  return cudaGetLastError();
}

int sharpness_blocks(Geo geo) { return elementwise_grid((long long)geo.nx * geo.ny * geo.nz); }

cudaError_t launch_sharpness(const float* d_mu, Geo geo, float* d_m, double* d_part, double* d_stats, float* d_loss,
                             float* d_grad, cudaStream_t s) {
  const long long n = (long long)geo.nx * geo.ny * geo.nz;
  const int nb = elementwise_grid(n);
  k_sharp_magnitude<<<nb, 256, 0, s>>>(d_mu, geo, d_m, d_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sharp_stats<<<1, 32, 0, s>>>(d_part, nb, n, d_stats, d_loss);
  e = cudaGetLastError();
  if (e != cudaSuccess || !d_grad) return e;
  k_sharp_grad<<<nb, 256, 0, s>>>(d_mu, d_m, geo, d_stats, d_grad);
  return cudaGetLastError();
}

}  // namespace projk
