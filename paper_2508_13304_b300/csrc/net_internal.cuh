// Internal declarations of the pose-proposal network kernels (BF16 tensor-core
// GEMM on tcgen05/TMEM with TMA-staged operands, and the small data-movement
// kernels around it).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pnk {

// Status bits written by device code (read and cleared by pn_status).
constexpr int kStatusTimeoutTma = 1;   // a stage never filled
constexpr int kStatusTimeoutMma = 2;   // the accumulator never completed
constexpr int kStatusTimeoutFree = 4;  // a stage was never released

// GEMM tiling: 128 x BN output tile per CTA, K in blocks of 64 BF16 (one
// 128-byte swizzle atom row), kStages-deep TMA ring.
constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kStages = 4;
constexpr int kGemmThreads = 128;

struct GemmEpi {
  const float* bias;            // [N] or null
  const __nv_bfloat16* mask;    // [M][ldm]: output *= (mask > 0), or null
  int ldm;
  int relu;                     // max(0, .) after bias
  float* d32;                   // [M][ldd] FP32 output, or null
  __nv_bfloat16* d16;           // [M][ldd] BF16 output, or null
  int ldd;
  float* part;                  // split-K partials [split][M][N] (raw sums), or null
  unsigned long long wait_ns;   // limit of every mbarrier wait (global-timer ns)
  int stall_tma;                // test hook: the 1-SM kernel arms its stage barriers but issues no TMA
};

size_t gemm_smem_bytes(int bn);
// pair: 0 = 1-SM 128 x bn tiles; 1 = 2-SM 256 x 256 tiles, one per cluster; 2 = the same
// tiles on a persistent grid with two TMEM accumulators (pair != 0: bn 256, B box 128 rows)
cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int bn, int pair,
                        int split, int kb_per_split, const GemmEpi& epi, int* status, cudaStream_t s);
cudaError_t launch_split_reduce(const float* part, int split, int M, int N, const GemmEpi& epi, cudaStream_t s);
// implicit-GEMM 3x3 stride-2 pad-1 convolution: x NHWC [B][H][W][C] (C % 8 == 0), weights by the tensor map tw
// ([cout][9 C], boxes of bn rows), output through epi (rows = output pixels, columns = output channels)
cudaError_t launch_conv_implicit(const __nv_bfloat16* x, int B, int H, int W, int C, const CUtensorMap& tw, int cout,
                                 int bn, const GemmEpi& epi, int* status, cudaStream_t s);
// its input gradient as an implicit GEMM: dy [B][Ho][Wo][cout] (cout % 8 == 0), weights by the tensor map
// twt ([C][9 cout], k = tap * cout + o, boxes of bn rows), output through epi (rows = the B x H x W input
// pixels, columns = the C input channels)
cudaError_t launch_conv_dgrad_implicit(const __nv_bfloat16* dy, int B, int H, int W, int cout, const CUtensorMap& twt,
                                       int C, int bn, const GemmEpi& epi, int* status, cudaStream_t s);
// one Adam step on flat FP32 arrays (and the BF16 copy of p when p16 is not null)
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float step, float b1, float a1,
                        float b2, float a2, float eps, float decay, __nv_bfloat16* p16, cudaStream_t s);
// wt[c][tap * cout + o] = w[o][tap * C + c]: the weights of the input-gradient GEMM
cudaError_t launch_conv_dgrad_weights(const __nv_bfloat16* w, int cout, int C, __nv_bfloat16* wt, cudaStream_t s);

cudaError_t launch_im2col(const __nv_bfloat16* x, int B, int H, int W, int C, int kp, __nv_bfloat16* col,
                          cudaStream_t s);
cudaError_t launch_col2im(const float* dcol, int B, int H, int W, int C, int kp, const __nv_bfloat16* mask,
                          __nv_bfloat16* dx16, float* dx32, cudaStream_t s);
cudaError_t launch_transpose(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst, int ld, cudaStream_t s);
cudaError_t launch_colsum(const __nv_bfloat16* y, int M, int N, int ld, float* part, int n_part, float* out,
                          cudaStream_t s);
int colsum_parts(int M);
cudaError_t launch_prepare(const float* proj, int n_img, int n_views, int nu, int nv, int factor,
                           __nv_bfloat16* out, cudaStream_t s);
cudaError_t launch_mse(const float* y, int B, int n_out, int ldy, const float* target, float* loss,
                       __nv_bfloat16* dy, int lddy, cudaStream_t s);
cudaError_t launch_to_bf16(const float* src, long long n, __nv_bfloat16* dst, cudaStream_t s);

int* status_word();   // device address of the status word of the current device

}  // namespace pnk
