// C ABI of the pose-proposal network kernels (include/posenet.h): argument
// checks, TMA tensor maps, tile and split choices, launches.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "net_internal.cuh"
#include "posenet.h"

namespace projk {
void record_error(const char* msg);
}

namespace pnk {

namespace {

__device__ int g_pn_status;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  projk::record_error(buf);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(PROJ_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
int g_use_pair = 2;
// limit of every mbarrier wait of the GEMM kernels, and the test hook that
// stalls the 1-SM kernel's TMA producer (pn_gemm_test_hooks)
constexpr unsigned long long kDefaultWaitNs = 2000000000ULL;  // 2 s
unsigned long long g_wait_ns = kDefaultWaitNs;
int g_stall_tma = 0;
int* g_status_addr[64] = {};
int g_n_sm[64] = {};

EncodeTiledFn encoder() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return g_encode;
}

int device_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_n_sm[dev]) {
    int n = 0;
    g_n_sm[dev] = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 148;
  }
  return g_n_sm[dev];
}

// Tensor map of a row-major BF16 matrix [rows][cols] (leading dimension ld)
// read in boxes of box_rows x 64 with the 128-byte swizzle; zero fill outside.
int make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows) {
  EncodeTiledFn enc = encoder();
  if (!enc) return fail(PROJ_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(PROJ_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return PROJ_OK;
}

// Widest N tile whose padding wastes at most 1/8 of the tile columns.
int bn_for(int N) {
  const int cands[4] = {256, 128, 64, 32};
  for (int c : cands) {
    const long long padded = (long long)((N + c - 1) / c) * c;
    if (padded * 8 <= (long long)N * 9) return c;
  }
  return 32;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

int* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pn_status) != cudaSuccess) return nullptr;
    g_status_addr[dev] = static_cast<int*>(p);
  }
  return g_status_addr[dev];
}

}  // namespace pnk

using namespace pnk;

extern "C" {

int pn_gemm_use_pair_tiles(int mode) {
  const int old = g_use_pair;
  g_use_pair = mode < 0 ? 0 : (mode > 2 ? 2 : mode);
  return old;
}

int pn_gemm_test_hooks(unsigned long long wait_ns, int stall_tma) {
  g_wait_ns = wait_ns ? wait_ns : kDefaultWaitNs;
  g_stall_tma = stall_tma ? 1 : 0;
  return PROJ_OK;
}

int pn_gemm_split_hint(int M, int N, int K) {
  if (M < 1 || N < 1 || K < 1) return 1;
  const int bn = bn_for(N);
  const long long tiles = (long long)((M + kBM - 1) / kBM) * ((N + bn - 1) / bn);
  const int nkb = (K + kBK - 1) / kBK;
  const long long want = (2LL * device_sms() + tiles - 1) / tiles;
  long long split = want < nkb / 4 ? want : nkb / 4;
  if (split > 64) split = 64;
  return split < 1 ? 1 : (int)split;
}

int pn_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, const float* bias,
                 const void* mask, int ldm, int relu, float* D32, void* D16, int ldd, int split_k, float* part,
                 proj_stream stream) {
  if (M < 1 || N < 1 || K < 1) return fail(PROJ_E_ARG, "pn_gemm_bf16: M, N, K must be >= 1 (%d, %d, %d)", M, N, K);
  if (!A || !B) return fail(PROJ_E_ARG, "pn_gemm_bf16: NULL operand");
  if (!D32 && !D16) return fail(PROJ_E_ARG, "pn_gemm_bf16: no output");
  if (lda < K || ldb < K || lda % 8 || ldb % 8)
    return fail(PROJ_E_ARG, "pn_gemm_bf16: lda and ldb must be multiples of 8 and >= K (%d, %d, K %d)", lda, ldb, K);
  if (!aligned16(A) || !aligned16(B)) return fail(PROJ_E_ARG, "pn_gemm_bf16: A and B must be 16-byte aligned");
  if (ldd < N) return fail(PROJ_E_ARG, "pn_gemm_bf16: ldd %d < N %d", ldd, N);
  if (mask && ldm < N) return fail(PROJ_E_ARG, "pn_gemm_bf16: ldm %d < N %d", ldm, N);
  if (split_k < 1) return fail(PROJ_E_ARG, "pn_gemm_bf16: split_k must be >= 1");
  if (split_k > 1 && !part) return fail(PROJ_E_ARG, "pn_gemm_bf16: split_k > 1 needs a partial-sum buffer");
  int* status = status_word();
  if (!status) return fail(PROJ_E_CUDA, "pn_gemm_bf16: no device status word");
  const int bn = bn_for(N);
  const int pair = (bn == 256 && M > kBM && !g_stall_tma) ? g_use_pair : 0;
  CUtensorMap ta, tb;
  int rc = make_map(&ta, A, M, K, lda, kBM);
  if (rc) return rc;
  if ((rc = make_map(&tb, B, N, K, ldb, pair ? 128 : bn))) return rc;
  const int nkb = (K + kBK - 1) / kBK;
  const int kbs = (nkb + split_k - 1) / split_k;
  const int split = (nkb + kbs - 1) / kbs;  // every CTA gets at least one K block
  GemmEpi epi;
  epi.bias = bias;
  epi.mask = static_cast<const __nv_bfloat16*>(mask);
  epi.ldm = ldm;
  epi.relu = relu;
  epi.d32 = D32;
  epi.d16 = static_cast<__nv_bfloat16*>(D16);
  epi.ldd = ldd;
  epi.part = split > 1 ? part : nullptr;
  epi.wait_ns = g_wait_ns;
  epi.stall_tma = g_stall_tma;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_gemm(ta, tb, M, N, K, bn, pair, split, kbs, epi, status, s);
  if (e != cudaSuccess) return cuda_fail(e, "GEMM launch");
  if (split > 1) {
    epi.part = nullptr;
    e = launch_split_reduce(part, split, M, N, epi, s);
    if (e != cudaSuccess) return cuda_fail(e, "split-K reduction launch");
  }
  return PROJ_OK;
}

int pn_conv3x3s2_bf16(const void* x, int B, int H, int W, int C, const void* w, int cout, const float* bias,
                      int relu, float* y32, void* y16, proj_stream stream) {
  if (!x || !w || (!y32 && !y16)) return fail(PROJ_E_ARG, "pn_conv3x3s2_bf16: NULL input, weights or output");
  if (B < 1 || H < 1 || W < 1 || cout < 1) return fail(PROJ_E_ARG, "pn_conv3x3s2_bf16: empty shape");
  if (C < 8 || C % 8) return fail(PROJ_E_ARG, "pn_conv3x3s2_bf16: C = %d must be a positive multiple of 8", C);
  if (!aligned16(x) || !aligned16(w)) return fail(PROJ_E_ARG, "pn_conv3x3s2_bf16: x and w must be 16-byte aligned");
  const long long M = (long long)B * ((H + 1) / 2) * ((W + 1) / 2);
  if (M > 0x7fffffffLL || (long long)B * H * W * C > (1LL << 40))
    return fail(PROJ_E_ARG, "pn_conv3x3s2_bf16: shape too large");
  int* status = status_word();
  if (!status) return fail(PROJ_E_CUDA, "pn_conv3x3s2_bf16: no device status word");
  const int bn = bn_for(cout);
  CUtensorMap tw;
  int rc = make_map(&tw, w, cout, 9 * C, 9 * C, bn);
  if (rc) return rc;
  GemmEpi epi;
  epi.bias = bias;
  epi.mask = nullptr;
  epi.ldm = 0;
  epi.relu = relu;
  epi.d32 = y32;
  epi.d16 = static_cast<__nv_bfloat16*>(y16);
  epi.ldd = cout;
  epi.part = nullptr;
  epi.wait_ns = g_wait_ns;
  epi.stall_tma = 0;
  cudaError_t e = launch_conv_implicit(static_cast<const __nv_bfloat16*>(x), B, H, W, C, tw, cout, bn, epi, status,
                                       (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "implicit convolution launch");
}

int pn_conv3x3s2_dgrad_bf16(const void* dy, int B, int H, int W, int C, const void* wt, int cout, const void* mask,
                            float* dx32, void* dx16, proj_stream stream) {
  if (!dy || !wt || (!dx32 && !dx16)) return fail(PROJ_E_ARG, "pn_conv3x3s2_dgrad_bf16: NULL input, weights or output");
  if (B < 1 || H < 1 || W < 1 || C < 1) return fail(PROJ_E_ARG, "pn_conv3x3s2_dgrad_bf16: empty shape");
  if (cout < 8 || cout % 8)
    return fail(PROJ_E_ARG, "pn_conv3x3s2_dgrad_bf16: cout = %d must be a positive multiple of 8", cout);
  if (!aligned16(dy) || !aligned16(wt)) return fail(PROJ_E_ARG, "pn_conv3x3s2_dgrad_bf16: dy and wt must be 16-byte aligned");
  const long long M = (long long)B * H * W;
  if (M > 0x7fffffffLL || M * C > (1LL << 40)) return fail(PROJ_E_ARG, "pn_conv3x3s2_dgrad_bf16: shape too large");
  int* status = status_word();
  if (!status) return fail(PROJ_E_CUDA, "pn_conv3x3s2_dgrad_bf16: no device status word");
  const int bn = bn_for(C);
  CUtensorMap tw;
  int rc = make_map(&tw, wt, C, 9 * cout, 9 * cout, bn);
  if (rc) return rc;
  GemmEpi epi;
  epi.bias = nullptr;
  epi.mask = static_cast<const __nv_bfloat16*>(mask);
  epi.ldm = C;
  epi.relu = 0;
  epi.d32 = dx32;
  epi.d16 = static_cast<__nv_bfloat16*>(dx16);
  epi.ldd = C;
  epi.part = nullptr;
  epi.wait_ns = g_wait_ns;
  epi.stall_tma = 0;
  cudaError_t e = launch_conv_dgrad_implicit(static_cast<const __nv_bfloat16*>(dy), B, H, W, cout, tw, C, bn, epi,
                                             status, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "implicit input-gradient launch");
}

int pn_conv_dgrad_weights(const void* w, int cout, int C, void* wt, proj_stream stream) {
  if (!w || !wt) return fail(PROJ_E_ARG, "pn_conv_dgrad_weights: NULL argument");
  if (cout < 1 || C < 1) return fail(PROJ_E_ARG, "pn_conv_dgrad_weights: empty shape");
  cudaError_t e = launch_conv_dgrad_weights(static_cast<const __nv_bfloat16*>(w), cout, C,
                                            static_cast<__nv_bfloat16*>(wt), (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "dgrad weights launch");
}

int pn_im2col_3x3s2(const void* x, int B, int H, int W, int C, int kp, void* col, proj_stream stream) {
  if (!x || !col) return fail(PROJ_E_ARG, "pn_im2col_3x3s2: NULL argument");
  if (B < 1 || H < 1 || W < 1 || C < 1) return fail(PROJ_E_ARG, "pn_im2col_3x3s2: empty shape");
  if (kp % 8 || kp < 9 * C) return fail(PROJ_E_ARG, "pn_im2col_3x3s2: kp %d must be a multiple of 8 and >= 9C", kp);
  if (C % 8 == 0 && !aligned16(x)) return fail(PROJ_E_ARG, "pn_im2col_3x3s2: x must be 16-byte aligned");
  if (!aligned16(col)) return fail(PROJ_E_ARG, "pn_im2col_3x3s2: col must be 16-byte aligned");
  cudaError_t e = launch_im2col(static_cast<const __nv_bfloat16*>(x), B, H, W, C, kp,
                                static_cast<__nv_bfloat16*>(col), (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "im2col launch");
}

int pn_col2im_3x3s2(const float* dcol, int B, int H, int W, int C, int kp, const void* mask, void* dx16, float* dx32,
                    proj_stream stream) {
  if (!dcol || (!dx16 && !dx32)) return fail(PROJ_E_ARG, "pn_col2im_3x3s2: NULL argument");
  if (B < 1 || H < 1 || W < 1 || C < 1 || kp < 9 * C) return fail(PROJ_E_ARG, "pn_col2im_3x3s2: bad shape");
  cudaError_t e = launch_col2im(dcol, B, H, W, C, kp, static_cast<const __nv_bfloat16*>(mask),
                                static_cast<__nv_bfloat16*>(dx16), dx32, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "col2im launch");
}

int pn_transpose_bf16(const void* src, int rows, int cols, void* dst, int ld_dst, proj_stream stream) {
  if (!src || !dst || src == dst) return fail(PROJ_E_ARG, "pn_transpose_bf16: NULL or aliased argument");
  if (rows < 1 || cols < 1 || ld_dst < rows) return fail(PROJ_E_ARG, "pn_transpose_bf16: bad shape");
  cudaError_t e = launch_transpose(static_cast<const __nv_bfloat16*>(src), rows, cols,
                                   static_cast<__nv_bfloat16*>(dst), ld_dst, (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "transpose launch");
}

size_t pn_colsum_scratch_floats(int M, int N) {
  if (M < 1 || N < 1) return 0;
  return (size_t)colsum_parts(M) * N;
}

int pn_colsum_bf16(const void* y, int M, int N, int ld, float* out, float* scratch, proj_stream stream) {
  if (!y || !out || !scratch) return fail(PROJ_E_ARG, "pn_colsum_bf16: NULL argument");
  if (M < 1 || N < 1 || ld < N) return fail(PROJ_E_ARG, "pn_colsum_bf16: bad shape");
  cudaError_t e = launch_colsum(static_cast<const __nv_bfloat16*>(y), M, N, ld, scratch, colsum_parts(M), out,
                                (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "column-sum launch");
}

int pn_prepare_images(const float* proj, int n_img, int n_views, int nu, int nv, int factor, void* out,
                      proj_stream stream) {
  if (!proj || !out) return fail(PROJ_E_ARG, "pn_prepare_images: NULL argument");
  if (n_img < 1 || n_views < 1 || factor < 1 || nu < factor || nv < factor || nu % factor || nv % factor)
    return fail(PROJ_E_ARG, "pn_prepare_images: sizes must be positive multiples of factor");
  if ((size_t)(nu / factor) * (nv / factor) * sizeof(float) > 200 * 1024)
    return fail(PROJ_E_ARG, "pn_prepare_images: downsampled image too large");
  cudaError_t e = launch_prepare(proj, n_img, n_views, nu, nv, factor, static_cast<__nv_bfloat16*>(out),
                                 (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "prepare launch");
}

int pn_mse_loss(const float* y, int B, int n_out, int ldy, const float* target, float* loss, void* dy, int lddy,
                proj_stream stream) {
  if (!y || !target) return fail(PROJ_E_ARG, "pn_mse_loss: NULL argument");
  if (B < 1 || n_out < 1 || ldy < n_out || lddy < n_out || (long long)B * lddy > (1LL << 24))
    return fail(PROJ_E_ARG, "pn_mse_loss: bad shape");
  cudaError_t e = launch_mse(y, B, n_out, ldy, target, loss, static_cast<__nv_bfloat16*>(dy), lddy,
                             (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "mse launch");
}

int pn_to_bf16(const float* src, long long n, void* dst, proj_stream stream) {
  if (!src || !dst || n < 1) return fail(PROJ_E_ARG, "pn_to_bf16: bad argument");
  cudaError_t e = launch_to_bf16(src, n, static_cast<__nv_bfloat16*>(dst), (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "conversion launch");
}

int pn_adam_step(float* p, const float* g, float* m, float* v, long long n, float step, float b1, float a1, float b2,
                 float a2, float eps, float decay, void* p16, proj_stream stream) {
  if (!p || !g || !m || !v || n < 1) return fail(PROJ_E_ARG, "pn_adam_step: bad argument");
  cudaError_t e = launch_adam(p, g, m, v, n, step, b1, a1, b2, a2, eps, decay, static_cast<__nv_bfloat16*>(p16),
                              (cudaStream_t)stream);
  return e == cudaSuccess ? PROJ_OK : cuda_fail(e, "adam launch");
}

int pn_status(proj_stream stream, int* status) {
  if (!status) return fail(PROJ_E_ARG, "pn_status: NULL argument");
  int* w = status_word();
  if (!w) return fail(PROJ_E_CUDA, "pn_status: no device status word");
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "pn_status");
  *status = h;
  return PROJ_OK;
}

}  // extern "C"
