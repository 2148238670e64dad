/* C ABI of the pose-proposal network kernels of libproj.so (sm_103a).
 *
 * The paper closes with learned, coarse-to-fine pose initialisation as
 * future work (Sec. V); this library provides the building blocks of a
 * small convolutional pose regressor trained on digitally reconstructed
 * radiographs from proj_forward: a BF16 GEMM on the 5th-generation tensor
 * cores (tcgen05.mma with the accumulator in tensor memory, operands staged
 * by TMA) and the data-movement kernels that map 3x3 stride-2 convolutions
 * and their gradients onto it.  The paper has no counterpart of these calls.
 *
 * Conventions.  BF16 arrays are passed as void* (IEEE bfloat16, 2 bytes).
 * Matrices are row-major with an explicit leading dimension in elements.
 * Images and activations are NHWC: [batch][height][width][channels].
 * Every pointer is a device pointer on the current device unless stated;
 * every call only enqueues work on `stream` (no synchronisation, no
 * allocation) except pn_status.  Return codes are those of proj.h
 * (PROJ_OK, PROJ_E_ARG, PROJ_E_CUDA); the message of the last failure is
 * in proj_last_error().  Device-side wait timeouts set bits of a per-device
 * status word, read with pn_status. */
#ifndef PAPER_2508_13304_POSENET_H
#define PAPER_2508_13304_POSENET_H

#include <stddef.h>

#include "proj.h"

#ifdef __cplusplus
extern "C" {
#endif

/* D = epilogue(A . B^T): A [M][K] (leading dimension lda), B [N][K] (ldb),
 * both BF16, FP32 accumulation.  Epilogue per element, in this order: + bias[n]
 * (bias may be NULL), max(0, .) if relu, times (mask[m][n] > 0) if mask
 * (BF16 [M][ldm]) is not NULL.  Output to D32 (FP32) and/or D16 (BF16),
 * both [M][ldd]; at least one.  Requirements: M, N, K >= 1; lda, ldb
 * multiples of 8 and >= K; A and B 16-byte aligned (TMA); ldd >= N.
 * split_k >= 1 divides the K loop over that many CTAs per tile; with
 * split_k > 1, part must hold split_k * M * N floats (raw partial sums,
 * added in a fixed order by a second kernel, so results are deterministic).
 * Elements of A and B past M, N or K are read as zero. */
int pn_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, const float *bias,
                 const void *mask, int ldm, int relu, float *D32, void *D16, int ldd, int split_k, float *part,
                 proj_stream stream);

/* Tile choice of pn_gemm_bf16 for wide outputs (N tiles of 256, M > 128):
 * mode 2 (the default): 256 x 256 tiles on pairs of SMs (a cluster of two
 * CTAs, tcgen05.mma.cta_group::2, each SM staging half of the B tile), one
 * cluster per pair of SMs looping over tiles with two TMEM accumulators so
 * that one tile's epilogue overlaps the next tile's MMAs; mode 1: the same
 * tiles, one cluster per tile; mode 0: 128 x 256 tiles on single SMs.
 * Results are identical across modes (each element accumulates K in the
 * same order).  Process-wide; returns the previous mode. */
int pn_gemm_use_pair_tiles(int mode);

/* The split_k that pn_gemm_bf16 would use well for this shape (about two
 * waves of CTAs on the device's SMs, at least 4 K blocks of 64 per CTA). */
int pn_gemm_split_hint(int M, int N, int K);

/* im2col of a 3x3, stride-2, padding-1 convolution: x NHWC BF16
 * [B][H][W][C] -> col BF16 [B*Ho*Wo][kp] with Ho = (H+1)/2, Wo = (W+1)/2,
 * col[(b,ho,wo)][(kh*3+kw)*C + c] = x[b][2ho-1+kh][2wo-1+kw][c] (zero outside
 * the image) and zero for columns >= 9C.  kp: multiple of 8, >= 9C.  With C
 * a multiple of 8, x must be 16-byte aligned. */
int pn_im2col_3x3s2(const void *x, int B, int H, int W, int C, int kp, void *col, proj_stream stream);

/* Adjoint of pn_im2col_3x3s2 (input gradient of the convolution): dx[b][hi][wi][c]
 * = sum of dcol over the (output pixel, tap) pairs that read (hi, wi, c),
 * dcol FP32 [B*Ho*Wo][kp].  If mask (BF16 NHWC like dx) is not NULL the sum
 * is zeroed where mask <= 0 (ReLU backward of the layer that produced x).
 * Output BF16 (dx16) and/or FP32 (dx32). */
int pn_col2im_3x3s2(const float *dcol, int B, int H, int W, int C, int kp, const void *mask, void *dx16,
                    float *dx32, proj_stream stream);

/* dst [cols][ld_dst] = src [rows][cols]^T, BF16; columns rows..ld_dst-1 of
 * dst are written with zeros (so a GEMM operand can have a leading
 * dimension that is a multiple of 8).  ld_dst >= rows. */
int pn_transpose_bf16(const void *src, int rows, int cols, void *dst, int ld_dst, proj_stream stream);

/* out[n] = sum over m of y[m][n] (y BF16 [M][ld]) with FP32 partial sums per
 * row block and an FP64 fixed-order final sum (bias gradients).  scratch:
 * at least pn_colsum_scratch_floats(M, N) floats. */
size_t pn_colsum_scratch_floats(int M, int N);
int pn_colsum_bf16(const void *y, int M, int N, int ld, float *out, float *scratch, proj_stream stream);

/* Network input from DRRs: proj FP32 [n_img][n_views][nv][nu] (the views of
 * an image consecutive, as proj_forward writes instances) -> out BF16 NHWC
 * [n_img][nv/factor][nu/factor][n_views]: box average over factor x factor
 * pixels, then per (image, view) zero mean and unit variance (a constant
 * image maps to zeros).  nu and nv multiples of factor; (nu/factor)*(nv/factor)
 * floats must fit in 200 KB of shared memory. */
int pn_prepare_images(const float *proj, int n_img, int n_views, int nu, int nv, int factor, void *out,
                      proj_stream stream);

/* Mean squared error of y (FP32 [B][ldy], first n_out columns) against
 * target (FP32 [B][n_out]): *loss = mean (y - t)^2 over B*n_out (loss may be
 * NULL); dy (BF16 [B][lddy], may be NULL) = 2 (y - t) / (B n_out), zero in
 * columns n_out..lddy-1.  B * lddy <= 2^24. */
int pn_mse_loss(const float *y, int B, int n_out, int ldy, const float *target, float *loss, void *dy, int lddy,
                proj_stream stream);

/* dst = BF16(src), round to nearest even, n elements. */
int pn_to_bf16(const float *src, long long n, void *dst, proj_stream stream);

/* 3x3, stride-2, padding-1 convolution as an implicit GEMM on the tensor
 * cores: the same products and accumulation order as pn_im2col_3x3s2 (kp =
 * 9 C) followed by pn_gemm_bf16 on 1-SM tiles, hence the same results, but
 * the (pixel x tap x channel) matrix is never written: the kernel gathers
 * each 128 x 64 operand tile from x into shared memory itself.
 *   x      BF16 NHWC [B][H][W][C], C a multiple of 8, 16-byte aligned.
 *   w      BF16 [cout][9 C] (k = (kh * 3 + kw) * C + c), 16-byte aligned.
 *   bias   [cout] FP32 or NULL; relu: max(0, .) after the bias.
 *   y32, y16  outputs [B][Ho][Wo][cout] (FP32 / BF16; at least one),
 *          Ho = (H + 1) / 2, Wo = (W + 1) / 2.
 * Errors: PROJ_E_ARG (shapes, alignment, C not a multiple of 8),
 * PROJ_E_CUDA.  Waits are bounded as in pn_gemm_bf16 (pn_status). */
int pn_conv3x3s2_bf16(const void *x, int B, int H, int W, int C, const void *w, int cout, const float *bias,
                      int relu, float *y32, void *y16, proj_stream stream);

/* Input gradient of pn_conv3x3s2_bf16 as an implicit GEMM on the tensor
 * cores, the adjoint of the convolution's patch gather without a column
 * matrix: dx[b][iy][ix][c] = sum over taps (ky, kx) and output channels o of
 * dy[b][oy][ox][o] w[o][(ky * 3 + kx) C + c], over the (oy, ox) with
 * 2 oy - 1 + ky = iy and 2 ox - 1 + kx = ix inside the output grid.  The
 * kernel gathers each 128 x 64 tile of dy rows into shared memory; FP32
 * accumulation.  With cout a multiple of 64 the input pixels run in their
 * four parity classes (iy mod 2, ix mod 2), each over only the 1, 2 or 4
 * taps that reach an output pixel; else every pixel runs over all 9 taps
 * (zero rows for the taps with no output pixel).
 *   dy     BF16 NHWC [B][Ho][Wo][cout], Ho = (H + 1) / 2, Wo = (W + 1) / 2,
 *          cout a multiple of 8, 16-byte aligned.
 *   wt     BF16 [C][9 cout], k = (ky * 3 + kx) cout + o: the weights
 *          rearranged by pn_conv_dgrad_weights, 16-byte aligned.
 *   mask   BF16 NHWC [B][H][W][C] or NULL: dx is zeroed where mask <= 0
 *          (ReLU backward of the layer that produced the convolution's x).
 *   dx32, dx16  outputs [B][H][W][C] (FP32 / BF16; at least one).
 * Errors: PROJ_E_ARG (shapes, alignment, cout not a multiple of 8),
 * PROJ_E_CUDA.  Waits are bounded as in pn_gemm_bf16 (pn_status). */
int pn_conv3x3s2_dgrad_bf16(const void *dy, int B, int H, int W, int C, const void *wt, int cout, const void *mask,
                            float *dx32, void *dx16, proj_stream stream);

/* wt[c][(ky * 3 + kx) cout + o] = w[o][(ky * 3 + kx) C + c]: the weights of
 * pn_conv3x3s2_dgrad_bf16 from those of the convolution (BF16, no padding
 * columns: w is [cout][9 C]). */
int pn_conv_dgrad_weights(const void *w, int cout, int C, void *wt, proj_stream stream);

/* One Adam step on n FP32 elements (flat arrays, the whole network in one
 * launch): m = b1 m + a1 g; v = b2 v + a2 g^2; p = decay p - step m /
 * (sqrt(v) + eps), with a1 = 1 - b1 and a2 = 1 - b2 (passed separately so
 * that they carry full FP32 precision), step = lr sqrt(1 - b2^t) /
 * (1 - b1^t) and decay = 1 - lr wd from the caller; p16 (BF16, n elements)
 * or NULL receives the updated p rounded to BF16.  Errors: PROJ_E_ARG,
 * PROJ_E_CUDA. */
int pn_adam_step(float *p, const float *g, float *m, float *v, long long n, float step, float b1, float a1, float b2,
                 float a2, float eps, float decay, void *p16, proj_stream stream);

/* Synchronise the stream, return and clear the status word of the current
 * device: 0 = clean; bit 1: a TMA stage never filled, bit 2: an
 * accumulator never completed, bit 4: a stage was never released (each
 * after a bound on the wait, 2 s unless pn_gemm_test_hooks lowers it; the
 * CTA then released its tensor memory and returned, and the output of that
 * launch is undefined). */
int pn_status(proj_stream stream, int *status);

/* Test hook for the GEMM's failure path (no counterpart in the paper).
 * Every mbarrier wait of the GEMM kernels gives up after wait_ns of the
 * global timer (0 restores the default, 2 s), sets a pn_status bit and lets
 * the CTA skip its stores, free its tensor memory and return.  With
 * stall_tma non-zero, GEMMs run on 1-SM tiles and the TMA producer arms each
 * stage barrier for its bytes but issues no copy, so the waits on those
 * barriers run out: the call then returns normally, its output is left
 * unwritten, and pn_status reports bit 1 (a stage never filled) and, with
 * more K blocks than pipeline stages, bit 4 (a stage never released).  No
 * copy is left in flight.  Settings are process-wide and apply to GEMMs
 * launched afterwards; for tests of the failure path only.  Returns PROJ_OK. */
int pn_gemm_test_hooks(unsigned long long wait_ns, int stall_tma);

#ifdef __cplusplus
}
#endif

#endif
