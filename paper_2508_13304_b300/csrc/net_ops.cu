// Data-movement kernels of the pose-proposal network: im2col / col2im of the
// 3x3 stride-2 pad-1 convolution (NHWC, BF16), BF16 transposes, column sums
// (bias gradients), DRR preparation (box downsampling and per-image
// standardisation) and the mean-squared pose loss with its gradient.
#include "net_internal.cuh"

namespace pnk {

namespace {

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 148LL * 32) b = 148LL * 32;
  return (int)(b < 1 ? 1 : b);
}

// col[m][k], m = (b, ho, wo), k = (kh * 3 + kw) * C + c for k < 9C, 0 above.
// Input pixel (hi, wi) = (2 ho - 1 + kh, 2 wo - 1 + kw); zero outside.
__global__ void k_im2col(const __nv_bfloat16* __restrict__ x, int B, int H, int W, int C, int kp,
                         __nv_bfloat16* __restrict__ col) {
  const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
  const long long groups = (long long)B * Ho * Wo * (kp / 8);
  const bool vec = (C % 8) == 0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
    const int k8 = (int)(g % (kp / 8));
    const long long m = g / (kp / 8);
    const int wo = (int)(m % Wo), ho = (int)((m / Wo) % Ho), b = (int)(m / ((long long)Wo * Ho));
    __nv_bfloat16* dst = col + m * kp + k8 * 8;
    if (vec) {
      const int k = k8 * 8, tap = k / C, c = k % C;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (tap < 9) {
        const int hi = 2 * ho - 1 + tap / 3, wi = 2 * wo - 1 + tap % 3;
        if (hi >= 0 && hi < H && wi >= 0 && wi < W)
          v = *reinterpret_cast<const uint4*>(x + (((size_t)b * H + hi) * W + wi) * C + c);
      }
      *reinterpret_cast<uint4*>(dst) = v;
    } else {
      for (int j = 0; j < 8; ++j) {
        const int k = k8 * 8 + j, tap = k / C, c = k % C;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (tap < 9) {
          const int hi = 2 * ho - 1 + tap / 3, wi = 2 * wo - 1 + tap % 3;
          if (hi >= 0 && hi < H && wi >= 0 && wi < W) v = x[(((size_t)b * H + hi) * W + wi) * C + c];
        }
        dst[j] = v;
      }
    }
  }
}

// dx[b][hi][wi][c] = sum over the taps that read (hi, wi) of dcol, times
// (mask > 0) when a mask (the post-ReLU input) is given.
__global__ void k_col2im(const float* __restrict__ dcol, int B, int H, int W, int C, int kp,
                         const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ dx16,
                         float* __restrict__ dx32) {
  const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
  const long long n = (long long)B * H * W * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int wi = (int)(p % W), hi = (int)((p / W) % H), b = (int)(p / ((long long)W * H));
    float s = 0.f;
    if (!mask || __bfloat162float(mask[i]) > 0.f) {
      for (int kh = 0; kh < 3; ++kh) {
        const int t = hi + 1 - kh;
        if (t < 0 || (t & 1) || (t >> 1) >= Ho) continue;
        const int ho = t >> 1;
        for (int kw = 0; kw < 3; ++kw) {
          const int u = wi + 1 - kw;
          if (u < 0 || (u & 1) || (u >> 1) >= Wo) continue;
          const int wo = u >> 1;
          s += dcol[(((size_t)b * Ho + ho) * Wo + wo) * kp + (kh * 3 + kw) * C + c];
        }
      }
    }
    if (dx16) dx16[i] = __float2bfloat16_rn(s);
    if (dx32) dx32[i] = s;
  }
}

constexpr int kTr = 32;

__global__ void k_transpose(const __nv_bfloat16* __restrict__ src, int R, int C, __nv_bfloat16* __restrict__ dst,
                            int ld) {
  __shared__ __nv_bfloat16 t[kTr][kTr + 2];
  const int c0 = blockIdx.x * kTr, r0 = blockIdx.y * kTr;
  for (int j = threadIdx.y; j < kTr; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    t[j][threadIdx.x] = (r < R && c < C) ? src[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < kTr; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;  // rows R..ld-1 of dst are zero padding
    if (r < ld && c < C) dst[(size_t)c * ld + r] = t[threadIdx.x][j];
  }
}

// Column sums, stage 1: block q sums rows [q * rows, (q + 1) * rows) of every
// column (one thread per column, columns strided by the block size).
__global__ void k_colsum_part(const __nv_bfloat16* __restrict__ y, int M, int N, int ld, int rows,
                              float* __restrict__ part) {
  const int q = blockIdx.x;
  const int r0 = q * rows, r1 = min(M, r0 + rows);
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += __bfloat162float(y[(size_t)r * ld + c]);
    part[(size_t)q * N + c] = s;
  }
}

// Column sums, stage 2: one block per column sums the n_part partials in a
// fixed order (thread t the partials t, t + 256, ..., then a shared-memory
// tree), in FP64; a column per thread made one long dependent chain of FP64
// adds, which run at a small fraction of the FP32 rate here.
constexpr int kColsumFinalThreads = 256;
__global__ void __launch_bounds__(kColsumFinalThreads) k_colsum_final(const float* __restrict__ part, int n_part, int N,
                                                                     float* __restrict__ out) {
  __shared__ double red[kColsumFinalThreads];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < n_part; q += kColsumFinalThreads) s += part[(size_t)q * N + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kColsumFinalThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = (float)red[0];
}

// One block per (image, view): box-average by `factor` into shared memory,
// then standardise (zero mean, unit variance over the downsampled image) and
// write NHWC with the views as channels.
__global__ void k_prepare(const float* __restrict__ proj, int n_views, int nu, int nv, int factor,
                          __nv_bfloat16* __restrict__ out) {
  extern __shared__ float img[];
  __shared__ double red[2][32];
  const int iv = blockIdx.x % n_views, im = blockIdx.x / n_views;
  const int wo = nu / factor, ho = nv / factor;
  const float* src = proj + (size_t)blockIdx.x * nu * nv;
  const float inv = 1.0f / (float)(factor * factor);
  double s1 = 0.0, s2 = 0.0;
  for (int p = threadIdx.x; p < wo * ho; p += blockDim.x) {
    const int x = p % wo, y = p / wo;
    float a = 0.f;
    for (int dy = 0; dy < factor; ++dy)
      for (int dx = 0; dx < factor; ++dx) a += src[(size_t)(y * factor + dy) * nu + x * factor + dx];
    a *= inv;
    img[p] = a;
    s1 += a;
    s2 += (double)a * a;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    red[0][0] = a;
    red[1][0] = b;
  }
  __syncthreads();
  const double n = (double)wo * ho;
  const double mean = red[0][0] / n;
  const double var = red[1][0] / n - mean * mean;
  const float scale = var > 1e-20 ? (float)(1.0 / sqrt(var)) : 0.f;
  const float m = (float)mean;
  for (int p = threadIdx.x; p < wo * ho; p += blockDim.x)
    out[((size_t)im * wo * ho + p) * n_views + iv] = __float2bfloat16_rn((img[p] - m) * scale);
}

// Single block: loss = mean over B x n_out of (y - t)^2; dy = 2 (y - t) / (B n_out)
// in BF16 with zero padding columns [n_out, lddy).
__global__ void k_mse(const float* __restrict__ y, int B, int n_out, int ldy, const float* __restrict__ t,
                      float* __restrict__ loss, __nv_bfloat16* __restrict__ dy, int lddy) {
  __shared__ double red[32];
  const double inv = 1.0 / ((double)B * n_out);
  double s = 0.0;
  for (int i = threadIdx.x; i < B * lddy; i += blockDim.x) {
    const int b = i / lddy, j = i % lddy;
    float g = 0.f;
    if (j < n_out) {
      const float d = y[(size_t)b * ldy + j] - t[(size_t)b * n_out + j];
      s += (double)d * d;
      g = (float)(2.0 * inv) * d;
    }
    if (dy) dy[i] = __float2bfloat16_rn(g);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    if (loss) *loss = (float)(a * inv);
  }
}

__global__ void k_to_bf16(const float* __restrict__ src, long long n, __nv_bfloat16* __restrict__ dst) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// Adam on flat FP32 arrays, and the BF16 copy of the updated weights.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float step, float b1, float a1, float b2, float a2, float eps, float decay,
                       __nv_bfloat16* __restrict__ p16) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + a1 * gi;
    const float vi = b2 * v[i] + a2 * gi * gi;
    const float pi = p[i] * decay - step * mi / (sqrtf(vi) + eps);
    m[i] = mi;
    v[i] = vi;
    p[i] = pi;
    if (p16) p16[i] = __float2bfloat16_rn(pi);
  }
}

// Weights of the input-gradient GEMM: wt[c][tap * cout + o] = w[o][tap * C + c], one thread per element.
__global__ void k_dgrad_weights(const __nv_bfloat16* __restrict__ w, int cout, int C, __nv_bfloat16* __restrict__ wt) {
  const long long n = 9LL * cout * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(i % cout);
    const long long r = i / cout;
    const int tap = (int)(r % 9), c = (int)(r / 9);
    wt[i] = w[((long long)o * 9 + tap) * C + c];
  }
}

}  // namespace

cudaError_t launch_im2col(const __nv_bfloat16* x, int B, int H, int W, int C, int kp, __nv_bfloat16* col,
                          cudaStream_t s) {
  const long long groups = (long long)B * ((H + 1) / 2) * ((W + 1) / 2) * (kp / 8);
  k_im2col<<<grid_for(groups, 256), 256, 0, s>>>(x, B, H, W, C, kp, col);
  return cudaGetLastError();
}

cudaError_t launch_col2im(const float* dcol, int B, int H, int W, int C, int kp, const __nv_bfloat16* mask,
                          __nv_bfloat16* dx16, float* dx32, cudaStream_t s) {
  k_col2im<<<grid_for((long long)B * H * W * C, 256), 256, 0, s>>>(dcol, B, H, W, C, kp, mask, dx16, dx32);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst, int ld, cudaStream_t s) {
  dim3 grid((C + kTr - 1) / kTr, (ld + kTr - 1) / kTr), block(kTr, 8);
  k_transpose<<<grid, block, 0, s>>>(src, R, C, dst, ld);
  return cudaGetLastError();
}

int colsum_parts(int M) {
  int n = (M + 255) / 256;
  return n > 1024 ? 1024 : (n < 1 ? 1 : n);
}

cudaError_t launch_colsum(const __nv_bfloat16* y, int M, int N, int ld, float* part, int n_part, float* out,
                          cudaStream_t s) {
  const int rows = (M + n_part - 1) / n_part;
  k_colsum_part<<<n_part, 256, 0, s>>>(y, M, N, ld, rows, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_colsum_final<<<N, kColsumFinalThreads, 0, s>>>(part, n_part, N, out);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const float* proj, int n_img, int n_views, int nu, int nv, int factor,
                           __nv_bfloat16* out, cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)(nu / factor) * (nv / factor);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_prepare, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_prepare<<<n_img * n_views, 256, smem, s>>>(proj, n_views, nu, nv, factor, out);
  return cudaGetLastError();
}

cudaError_t launch_mse(const float* y, int B, int n_out, int ldy, const float* target, float* loss,
                       __nv_bfloat16* dy, int lddy, cudaStream_t s) {
  k_mse<<<1, 1024, 0, s>>>(y, B, n_out, ldy, target, loss, dy, lddy);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, long long n, __nv_bfloat16* dst, cudaStream_t s) {
  k_to_bf16<<<grid_for(n, 256), 256, 0, s>>>(src, n, dst);
  return cudaGetLastError();
}

cudaError_t launch_conv_dgrad_weights(const __nv_bfloat16* w, int cout, int C, __nv_bfloat16* wt, cudaStream_t s) {
  k_dgrad_weights<<<grid_for(9LL * cout * C, 256), 256, 0, s>>>(w, cout, C, wt);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float step, float b1, float a1,
                        float b2, float a2, float eps, float decay, __nv_bfloat16* p16, cudaStream_t s) {
  k_adam<<<grid_for(n, 256), 256, 0, s>>>(p, g, m, v, n, step, b1, a1, b2, a2, eps, decay, p16);
  return cudaGetLastError();
}

}  // namespace pnk
