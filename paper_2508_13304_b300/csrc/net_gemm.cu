// BF16 GEMM on the 5th-generation tensor cores (sm_103a):
//   D[M][N] = epilogue( A[M][K] . B[N][K]^T ),  FP32 accumulation in TMEM.
//
// One CTA computes a 128 x BN tile of D.  Warp 0 (one lane) streams 128 x 64
// tiles of A and BN x 64 tiles of B into a kStages-deep shared-memory ring
// with TMA (128-byte swizzle, zero fill past the matrix edges); warp 1 (one
// lane) issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
// K = 16 per instruction) into the TMEM accumulator and releases each stage
// with tcgen05.commit; then all four warps read their 32 TMEM lanes
// (tcgen05.ld 32x32b) and apply bias, ReLU and a ReLU mask before storing
// FP32 and/or BF16.  With split-K the CTA writes raw FP32 partial sums that
// a second kernel adds in a fixed order.  Every wait on an mbarrier is
// bounded by the global timer; a timeout sets a status bit and the CTA
// releases its TMEM and returns.
#include <algorithm>
#include <cstdio>

#include "net_internal.cuh"

namespace pnk {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the completion of the phase with the given parity, at most
// limit_ns of the global timer (GemmEpi::wait_ns: 2 s unless a test lowers it).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile stored as rows
// of 128 bytes (64 BF16 of K) with the 128-byte swizzle, 8-row groups 1024
// bytes apart: start address, leading offset (unused by swizzled K-major
// layouts), stride offset 1024 B, descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = bn, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(bn >> 3) << 17) |
         (static_cast<uint32_t>(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
__host__ __device__ constexpr int tmem_cols() {
  return BN < 32 ? 32 : BN;
}

__device__ __forceinline__ float epi_value(float acc, int row, int col, const GemmEpi& e) {
  float v = acc;
  if (e.bias) v += __ldg(e.bias + col);
  if (e.relu) v = fmaxf(v, 0.f);
  if (e.mask && !(__bfloat162float(e.mask[(size_t)row * e.ldm + col]) > 0.f)) v = 0.f;
  return v;
}

// Epilogue of one CTA: its 128 TMEM lanes are rows m0..m0+127 of D, its BN
// columns are n0..; each warp reads its 32 lanes 16 columns at a time.
// out_row >= 0 stores this lane's row as row out_row of D (and of the mask)
// instead, for GEMMs whose rows are a permutation of D's.
template <int BN>
__device__ __forceinline__ void epilogue(uint32_t tmem_d, int m0, int n0, int M, int N, int z, const GemmEpi& epi,
                                         int quarter, int out_row = -1) {
  const int lane = threadIdx.x & 31;
  const int lrow = m0 + quarter * 32 + lane;  // a warp reads TMEM lanes 32 * (warp id mod 4) ...
  const int row = out_row >= 0 ? out_row : lrow;
  const uint32_t lane_base = tmem_d + (static_cast<uint32_t>(quarter * 32) << 16);
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float v[16];
    __syncwarp();  // tcgen05.ld is warp-collective
    tmem_ld16(lane_base + c0, v);
    const int col0 = n0 + c0;
    if (lrow >= M || col0 >= N) continue;
    const int nval = min(16, N - col0);
    if (epi.part) {
      float* dst = epi.part + ((size_t)z * M + row) * N + col0;
      for (int j = 0; j < nval; ++j) dst[j] = v[j];
      continue;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < nval) v[j] = epi_value(v[j], row, col0 + j, epi);
    if (epi.d32) {
      float* dst = epi.d32 + (size_t)row * epi.ldd + col0;
      if (nval == 16 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else {
        for (int j = 0; j < nval; ++j) dst[j] = v[j];
      }
    }
    if (epi.d16) {
      __nv_bfloat16* dst = epi.d16 + (size_t)row * epi.ldd + col0;
      if (nval == 16 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        __nv_bfloat162 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
        reinterpret_cast<uint4*>(dst)[0] = *reinterpret_cast<uint4*>(&h[0]);
        reinterpret_cast<uint4*>(dst)[1] = *reinterpret_cast<uint4*>(&h[4]);
      } else {
        for (int j = 0; j < nval; ++j) dst[j] = __float2bfloat16_rn(v[j]);
      }
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N, int K,
                int kb_per_split, GemmEpi epi, int* status) {
  constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = BN * kBK * 2;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // swizzle atoms need 1024-byte alignment
  uint8_t* const gbase = smem_raw + (base - raw);
  const uint32_t sA = base, sB = base + kStages * kBytesA;
  const uint32_t bars = sB + kStages * kBytesB;  // full[kStages], empty[kStages], done
  uint64_t* const bar_ptr = reinterpret_cast<uint64_t*>(gbase + (bars - base));
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 2 * kStages + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (kStages + s); };
  const uint32_t done = bars + 8u * (2 * kStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int nkb_all = (K + kBK - 1) / kBK;
  const int kb0 = blockIdx.z * kb_per_split;
  const int nkb = min(nkb_all, kb0 + kb_per_split) - kb0;  // >= 1 by construction on the host

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols<BN>())
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;
  int fail = 0;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (i >= kStages && !mbar_wait(empty(s), ((i / kStages) - 1) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutFree;
        break;
      }
      mbar_expect_tx(full(s), kBytesA + kBytesB);
      if (epi.stall_tma) continue;  // test hook: the stage is armed but never filled
      tma_load_2d(sA + s * kBytesA, &ta, full(s), (kb0 + i) * kBK, m0);
      tma_load_2d(sB + s * kBytesB, &tb, full(s), (kb0 + i) * kBK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(full(s), (i / kStages) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutTma;
        break;
      }
      tc_fence_after();
      const uint64_t da = sw128_desc(sA + s * kBytesA), db = sw128_desc(sB + s * kBytesB);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)  // +32 bytes of K per instruction
        umma_bf16(tmem_d, da + 2 * kk, db + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit(empty(s));
    }
    umma_commit(done);
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0, epi.wait_ns);
  if (!ok && threadIdx.x == 0) fail |= kStatusTimeoutMma;
  if (fail) atomicOr(status, fail);
  // a producer or MMA timeout leaves the accumulator incomplete: no thread stores it
  const bool any_fail = __syncthreads_or(fail != 0 || !ok) != 0;
  tc_fence_after();

  if (!any_fail) epilogue<BN>(tmem_d, m0, n0, M, N, blockIdx.z, epi, warp);

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(tmem_cols<BN>())
                 : "memory");
  }
}

// ---------------------------------------------------------------- 2-SM tile
//
// A cluster of two CTAs on two SMs computes a 256 x 256 tile with
// tcgen05.mma.cta_group::2 (M = 256): CTA r of the pair stages rows
// [128 r, 128 r + 128) of the A tile and rows [128 r, 128 r + 128) of the B
// tile, so each SM moves half the B bytes of a 1-SM 128 x 256 tile and the
// ring can be 6 stages deep.  Both CTAs' TMA loads signal the even CTA's
// "full" barrier (which expects the bytes of both); the even CTA issues the
// MMAs and multicasts each commit to both CTAs' "empty" / "done" barriers.
// Each CTA's TMEM holds its 128 rows of the accumulator.

constexpr int kStagesPair = 6;

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t o;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(o) : "r"(addr), "r"(rank));
  return o;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster, int x,
                                                 int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  const uint16_t both = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(both)
      : "memory");
}

__host__ __device__ constexpr uint32_t idesc_bf16_pair() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(256 >> 3) << 17) |
         (static_cast<uint32_t>(256 >> 4) << 24);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16_pair(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
                     int K, int kb_per_split, GemmEpi epi, int* status) {
  constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = 128 * kBK * 2;
  constexpr uint32_t kCols = 256;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* const gbase = smem_raw + (base - raw);
  const uint32_t sA = base, sB = base + kStagesPair * kBytesA;
  const uint32_t bars = sB + kStagesPair * kBytesB;
  uint64_t* const bar_ptr = reinterpret_cast<uint64_t*>(gbase + (bars - base));
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 2 * kStagesPair + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (kStagesPair + s); };
  const uint32_t done = bars + 8u * (2 * kStagesPair);

  const uint32_t rank = cluster_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (blockIdx.x >> 1) * 256 + (int)rank * 128;  // this CTA's rows of A and D
  const int n0 = blockIdx.y * 256;                           // the pair's columns of D
  const int nb = n0 + (int)rank * 128;                       // this CTA's rows of B
  const int nkb_all = (K + kBK - 1) / kBK;
  const int kb0 = blockIdx.z * kb_per_split;
  const int nkb = min(nkb_all, kb0 + kb_per_split) - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesPair; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers initialised and TMEM allocated
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;
  int fail = 0;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStagesPair;
      if (i >= kStagesPair && !mbar_wait(empty(s), ((i / kStagesPair) - 1) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutFree;
        break;
      }
      if (rank == 0) mbar_expect_tx(full(s), 2 * (kBytesA + kBytesB));
      const uint32_t leader_full = map_to_rank(full(s), 0);
      tma_load_2d_pair(sA + s * kBytesA, &ta, leader_full, (kb0 + i) * kBK, m0);
      tma_load_2d_pair(sB + s * kBytesB, &tb, leader_full, (kb0 + i) * kBK, nb);
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    constexpr uint32_t idesc = idesc_bf16_pair();
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStagesPair;
      if (!mbar_wait(full(s), (i / kStagesPair) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutTma;
        break;
      }
      tc_fence_after();
      const uint64_t da = sw128_desc(sA + s * kBytesA), db = sw128_desc(sB + s * kBytesB);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        umma_bf16_pair(tmem_d, da + 2 * kk, db + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit_pair(empty(s));
    }
    umma_commit_pair(done);
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0, epi.wait_ns);
  if (!ok && threadIdx.x == 0) fail |= kStatusTimeoutMma;
  if (fail) atomicOr(status, fail);
  tc_fence_after();
  if (ok) epilogue<256>(tmem_d, m0, n0, M, N, blockIdx.z, epi, warp);

  tc_fence_before();
  cluster_sync();  // neither CTA frees TMEM or exits while its peer may still touch the pair's state
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kCols) : "memory");
  }
}

// ---------------------------------------------------------------- persistent 2-SM
//
// The same 256 x 256 pair tiles, with one cluster per pair of SMs looping
// over tiles and two TMEM accumulators (2 x 256 columns): warp 0 streams
// K blocks without pausing between tiles, warp 1 of the even CTA issues the
// MMAs of tile j into accumulator j % 2 once the epilogue has drained it,
// and warps 2..5 of both CTAs drain the other accumulator meanwhile (warp w
// reads TMEM lanes 32 (w mod 4) ...).  An epilogue releases an accumulator
// by arriving, once per CTA, on the even CTA's "tmem_empty" barrier.

constexpr int kPersistThreads = 192;

__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

constexpr int kGroupM = 8;

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPersistThreads, 1)
    k_gemm_bf16_pair_persistent(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                                int M, int N, int K, int kb_per_split, int m_pairs, int n_tiles, int n_work,
                                GemmEpi epi, int* status) {
  constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = 128 * kBK * 2;
  constexpr uint32_t kCols = 512;  // two accumulators of 256 columns
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* const gbase = smem_raw + (base - raw);
  const uint32_t sA = base, sB = base + kStagesPair * kBytesA;
  const uint32_t bars = sB + kStagesPair * kBytesB;
  // full[S], empty[S], tmem_full[2], tmem_empty[2]
  uint64_t* const bar_ptr = reinterpret_cast<uint64_t*>(gbase + (bars - base));
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 2 * kStagesPair + 4);
  volatile int* const epi_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (kStagesPair + s); };
  auto tmem_full = [&](int b) { return bars + 8u * (2 * kStagesPair + b); };
  auto tmem_empty = [&](int b) { return bars + 8u * (2 * kStagesPair + 2 + b); };

  const uint32_t rank = cluster_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;
  const int nkb_all = (K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesPair; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tmem_full(b), 1);
      mbar_init(tmem_empty(b), 2);  // one arrival per CTA of the pair (used in the even CTA)
    }
    *epi_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;
  int fail = 0;

  // work item w -> (split z, N tile, M pair): groups of kGroupM M pairs, M
  // fastest inside a group, then N, then the next group, so the tiles the
  // clusters hold at one time share a few A and B panels in L2
  auto decode = [&](int w, int& mp, int& nt, int& z) {
    const int per_z = m_pairs * n_tiles;
    z = w / per_z;
    const int local = w - z * per_z;
    const int grp = local / (kGroupM * n_tiles), in = local - grp * (kGroupM * n_tiles);
    const int gsize = min(kGroupM, m_pairs - grp * kGroupM);
    mp = grp * kGroupM + in % gsize;
    nt = in / gsize;
  };
  auto kb_range = [&](int z, int& kb0, int& nkb) {
    kb0 = z * kb_per_split;
    nkb = min(nkb_all, kb0 + kb_per_split) - kb0;
  };

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;  // K blocks issued so far (ring position)
      for (int w = cluster; w < n_work && !fail; w += n_clusters) {
        int mp, nt, z, kb0, nkb;
        decode(w, mp, nt, z);
        kb_range(z, kb0, nkb);
        const int m0 = mp * 256 + (int)rank * 128, nb = nt * 256 + (int)rank * 128;
        for (int i = 0; i < nkb; ++i, ++g) {
          const int s = (int)(g % kStagesPair);
          const long long u = g / kStagesPair;
          if (u > 0 && !mbar_wait(empty(s), (uint32_t)((u - 1) & 1), epi.wait_ns)) {
            fail = kStatusTimeoutFree;
            break;
          }
          if (rank == 0) mbar_expect_tx(full(s), 2 * (kBytesA + kBytesB));
          const uint32_t leader_full = map_to_rank(full(s), 0);
          tma_load_2d_pair(sA + s * kBytesA, &ta, leader_full, (kb0 + i) * kBK, m0);
          tma_load_2d_pair(sB + s * kBytesB, &tb, leader_full, (kb0 + i) * kBK, nb);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      constexpr uint32_t idesc = idesc_bf16_pair();
      long long g = 0;
      int j = 0;  // tiles of this cluster so far
      for (int w = cluster; w < n_work && !fail; w += n_clusters, ++j) {
        int mp, nt, z, kb0, nkb;
        decode(w, mp, nt, z);
        kb_range(z, kb0, nkb);
        const int b = j & 1, ub = j >> 1;
        if (ub > 0 && !mbar_wait(tmem_empty(b), (uint32_t)((ub - 1) & 1), epi.wait_ns)) {
          fail = kStatusTimeoutMma;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem_d + (uint32_t)(b * 256);
        for (int i = 0; i < nkb; ++i, ++g) {
          const int s = (int)(g % kStagesPair);
          if (!mbar_wait(full(s), (uint32_t)((g / kStagesPair) & 1), epi.wait_ns)) {
            fail = kStatusTimeoutTma;
            break;
          }
          tc_fence_after();
          const uint64_t da = sw128_desc(sA + s * kBytesA), db = sw128_desc(sB + s * kBytesB);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            umma_bf16_pair(acc, da + 2 * kk, db + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
          umma_commit_pair(empty(s));
        }
        umma_commit_pair(tmem_full(b));
      }
    }
  } else {
    const int quarter = warp & 3;
    int j = 0;
    for (int w = cluster; w < n_work; w += n_clusters, ++j) {
      int mp, nt, z;
      decode(w, mp, nt, z);
      const int b = j & 1;
      const bool ok = mbar_wait(tmem_full(b), (uint32_t)((j >> 1) & 1), epi.wait_ns);
      if (!ok) {
        fail = kStatusTimeoutMma;
        *epi_abort = 1;
      } else {
        tc_fence_after();
        epilogue<256>(tmem_d + (uint32_t)(b * 256), mp * 256 + (int)rank * 128, nt * 256, M, N, z, epi, quarter);
      }
      tc_fence_before();
      asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps of this CTA are done with b
      const bool stop = *epi_abort != 0;              // same value in all four warps (read after the barrier)
      if (stop) break;
      if (warp == 2 && lane == 0) mbar_arrive_remote(map_to_rank(tmem_empty(b), 0));
    }
  }
  __syncwarp();
  if (fail) atomicOr(status, fail);

  tc_fence_before();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(kCols) : "memory");
  }
}

// Fixed-order sum of the split-K partials, then the epilogue.
__global__ void k_split_reduce(const float* __restrict__ part, int split, int M, int N, GemmEpi epi) {
  const long long total = (long long)M * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < split; ++z) s += part[(size_t)z * total + i];
    const int row = (int)(i / N), col = (int)(i % N);
    const float v = epi_value(s, row, col, epi);
    if (epi.d32) epi.d32[(size_t)row * epi.ldd + col] = v;
    if (epi.d16) epi.d16[(size_t)row * epi.ldd + col] = __float2bfloat16_rn(v);
  }
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int split, int kbs,
                      const GemmEpi& epi, int* status, cudaStream_t s) {
  const size_t smem = gemm_smem_bytes(BN);
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, split);
  k_gemm_bf16<BN><<<grid, kGemmThreads, smem, s>>>(ta, tb, M, N, K, kbs, epi, status);
  return cudaGetLastError();
}

cudaError_t launch_pair(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int split, int kbs,
                        const GemmEpi& epi, int* status, cudaStream_t s) {
  const size_t smem = 1024 + (size_t)kStagesPair * (kBM * kBK * 2 + 128 * kBK * 2) + 8 * (2 * kStagesPair + 1) + 16;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(2 * ((M + 255) / 256), (N + 255) / 256, split);
  k_gemm_bf16_pair<<<grid, kGemmThreads, smem, s>>>(ta, tb, M, N, K, kbs, epi, status);
  return cudaGetLastError();
}

cudaError_t launch_pair_persistent(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int split,
                                   int kbs, const GemmEpi& epi, int* status, cudaStream_t s) {
  const size_t smem = 1024 + (size_t)kStagesPair * (kBM * kBK * 2 + 128 * kBK * 2) + 8 * (2 * kStagesPair + 4) + 16;
  cudaError_t e =
      cudaFuncSetAttribute(k_gemm_bf16_pair_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int m_pairs = (M + 255) / 256, n_tiles = (N + 255) / 256;
  const long long work = (long long)m_pairs * n_tiles * split;
  if (work > (1LL << 30)) return cudaErrorInvalidValue;
  // as many clusters as can be resident at once (not every SM need find a partner in its GPC)
  int resident = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_sm - n_sm % 2, 1, 1);
  cfg.blockDim = dim3(kPersistThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  if (cudaOccupancyMaxActiveClusters(&resident, k_gemm_bf16_pair_persistent, &cfg) != cudaSuccess || resident < 1) {
    cudaGetLastError();
    resident = std::max(1, n_sm / 2);
  }
  const int clusters = (int)std::min<long long>(work, resident);
  k_gemm_bf16_pair_persistent<<<2 * clusters, kPersistThreads, smem, s>>>(ta, tb, M, N, K, kbs, m_pairs, n_tiles,
                                                                          (int)work, epi, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- implicit-GEMM convolution
//
// 3x3, stride-2, padding-1 convolution of an NHWC BF16 activation as a GEMM
// whose A operand (output pixels x (tap, channel)) is never written to
// memory: warps 0-3 gather each 128 x 64 A stage straight from the
// activation, one output pixel (tile row) per thread, as eight 16-byte
// cp.async copies placed at their 128-byte-swizzled positions (zero fill for
// taps in the padding and for rows past M).  MODE 1 and 2 run the input
// gradient of that convolution the same way: a row is an input pixel (iy,
// ix), and tap (ky, kx) reads the output gradient at ((iy + 1 - ky) / 2,
// (ix + 1 - kx) / 2) where both are integers inside the output grid (zero
// otherwise), against the weights rearranged to [C][9 cout].  The weights [Cout][9 C] arrive
// by TMA as in k_gemm_bf16 (warp 4), one lane of warp 5 issues the MMAs, and
// warps 0-3 run the same epilogue.  K runs tap-major, k = tap * C + c, as in
// k_im2col, so the accumulation order and the results equal those of im2col
// followed by the 1-SM GEMM.  A gathering thread keeps kStages - 1 stages of
// copies in flight; it signals a stage's "full" barrier (with a proxy fence,
// the MMA reads shared memory through the async proxy) once that stage's
// copies are complete.  Every wait is bounded as in the GEMM kernels.

constexpr int kConvThreads = 192;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// x: the gathered tensor, [B][SH][SW][C]; rows of the GEMM run over the grid [B][OH][OW] (MODE 0, the
// forward convolution: the output pixels, SH = H, OH = (H + 1) / 2; MODE 1, its input gradient: the
// input pixels, SH = Ho, OH = H, every row over all 9 taps).  MODE 2 is the input gradient by parity
// class: a block's rows are input pixels (iy, ix) of one class (iy mod 2, ix mod 2) = (py, px), for
// which only taps ky = 1 (py = 0) or ky in {0, 2} (py = 1), likewise kx, have an output pixel, so the
// K loop runs over those 1, 2 or 4 taps only (C a multiple of 64: a K block never straddles taps);
// M is then the batch size, the classes' tiles follow one another in blockIdx.x (ctile: the tile
// counts of classes 0, 0-1, 0-2, 0-3), and the epilogue stores each row at its pixel's position.
template <int BN, int MODE>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv3x3s2_implicit(const __nv_bfloat16* __restrict__ x, int SH, int SW, int C, int OH, int OW,
                         const __grid_constant__ CUtensorMap tb, int M, int N, GemmEpi epi, int* status,
                         int4 ctile) {
  constexpr bool DGRAD = MODE != 0;
  constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = BN * kBK * 2;
  constexpr int kAhead = kStages - 1;  // stages of copies a gathering thread keeps in flight
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* const gbase = smem_raw + (base - raw);
  const uint32_t sA = base, sB = base + kStages * kBytesA;
  const uint32_t bars = sB + kStages * kBytesB;  // full[kStages], empty[kStages], done
  uint64_t* const bar_ptr = reinterpret_cast<uint64_t*>(gbase + (bars - base));
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 2 * kStages + 1);
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (kStages + s); };
  const uint32_t done = bars + 8u * (2 * kStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.y * BN;
  int m0 = blockIdx.x * kBM, Mrows = M, nkb = (9 * C + kBK - 1) / kBK;
  int py = 0, px = 0, Hc = OH, Wc = OW, cpt = 1;
  if (MODE == 2) {  // uniform per block: the tile's parity class and its K blocks
    const int bx = blockIdx.x;
    const int cls = bx < ctile.x ? 0 : (bx < ctile.y ? 1 : (bx < ctile.z ? 2 : 3));
    const int first = cls == 0 ? 0 : (cls == 1 ? ctile.x : (cls == 2 ? ctile.y : ctile.z));
    py = cls >> 1;
    px = cls & 1;
    Hc = (OH + 1 - py) >> 1;
    Wc = (OW + 1 - px) >> 1;
    m0 = (bx - first) * kBM;
    Mrows = M * Hc * Wc;
    cpt = C / kBK;
    nkb = (1 + py) * (1 + px) * cpt;
  }
  // MODE 2: K block i is channels c .. c + 63 of tap (ky, kx)
  auto class_tap = [&](int i, int& ky, int& kx, int& c) {
    const int j = i / cpt, ntx = 1 + px, kyi = j / ntx, kxi = j - kyi * ntx;
    c = (i - j * cpt) * kBK;
    ky = py ? 2 * kyi : 1;
    kx = px ? 2 * kxi : 1;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1 + kBM);  // the weight TMA's expect_tx arrive + one arrive per gathered row
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols<BN>())
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = *tmem_slot;
  int fail = 0;

  int out_row = -1;  // MODE 2: this thread's row of the output
  if (warp < 4) {
    const int t = threadIdx.x;  // row of the A tile
    const int m = m0 + t;
    const bool row_ok = m < Mrows;
    int iy = 0, ix = 0;
    const __nv_bfloat16* xc = x;
    if (MODE == 2 && row_ok) {
      const int jx = m % Wc, jy = (m / Wc) % Hc, bc = m / (Wc * Hc);
      iy = 2 * jy + py;
      ix = 2 * jx + px;
      out_row = (bc * OH + iy) * OW + ix;
      xc = x + (size_t)bc * SH * SW * C;
    }
    const int wo = row_ok ? m % OW : 0, ho = row_ok ? (m / OW) % OH : 0, b = row_ok ? m / (OW * OH) : 0;
    // forward: source pixel (2 ho - 1 + ky, 2 wo - 1 + kx); DGRAD: twice the source pixel is (ho + 1 - ky,
    // wo + 1 - kx)
    const int hi0 = DGRAD ? ho + 1 : 2 * ho - 1, wi0 = DGRAD ? wo + 1 : 2 * wo - 1;
    const __nv_bfloat16* xb = x + (size_t)b * SH * SW * C;
    const uint32_t row_off = (uint32_t)t * 128u, swz = (uint32_t)(t & 7);
    int i = 0;
    for (; i < nkb; ++i) {
      const int s = i % kStages;
      if (i >= kStages && !mbar_wait(empty(s), ((i / kStages) - 1) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutFree;
        break;
      }
      const uint32_t dst = sA + s * kBytesA + row_off;
      if (MODE == 2) {
        int ky, kx, c;
        class_tap(i, ky, kx, c);
        const int oy = (iy + 1 - ky) >> 1, ox = (ix + 1 - kx) >> 1;  // exact: the class has the parity
        const bool ok = row_ok && oy < SH && ox < SW;
        const __nv_bfloat16* src = ok ? xc + ((size_t)oy * SW + ox) * C + c : x;
#pragma unroll
        for (int j = 0; j < kBK / 8; ++j) cp_async16(dst + (((uint32_t)j ^ swz) << 4), ok ? src + 8 * j : x, ok ? 16u : 0u);
      }
      const int k = i * kBK;
      int tap = k / C, c = k - tap * C;
#pragma unroll
      for (int j = 0; j < (MODE == 2 ? 0 : kBK / 8); ++j) {  // 16-byte chunk j of the row: k .. k + 7 of tap `tap`
        int hi, wi;
        bool ok;
        if (DGRAD) {
          const int h2 = hi0 - tap / 3, w2 = wi0 - tap % 3;
          hi = h2 >> 1;
          wi = w2 >> 1;
          ok = row_ok && tap < 9 && h2 >= 0 && !(h2 & 1) && hi < SH && w2 >= 0 && !(w2 & 1) && wi < SW;
        } else {
          hi = hi0 + tap / 3;
          wi = wi0 + tap % 3;
          ok = row_ok && tap < 9 && hi >= 0 && hi < SH && wi >= 0 && wi < SW;
        }
        cp_async16(dst + (((uint32_t)j ^ swz) << 4), ok ? xb + ((size_t)hi * SW + wi) * C + c : x, ok ? 16u : 0u);
        c += 8;
        if (c == C) {
          c = 0;
          ++tap;
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (i >= kAhead) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kAhead) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(full((i - kAhead) % kStages));
      }
    }
    // no copy may still be writing this CTA's shared memory when it moves on
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!fail)
      for (int q = max(0, nkb - kAhead); q < nkb; ++q) mbar_arrive(full(q % kStages));
  } else if (warp == 4 && lane == 0) {
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (i >= kStages && !mbar_wait(empty(s), ((i / kStages) - 1) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutFree;
        break;
      }
      mbar_expect_tx(full(s), kBytesB);
      int kcol = i * kBK;
      if (MODE == 2) {
        int ky, kx, c;
        class_tap(i, ky, kx, c);
        kcol = (ky * 3 + kx) * C + c;
      }
      tma_load_2d(sB + s * kBytesB, &tb, full(s), kcol, n0);
    }
  } else if (warp == 5 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(full(s), (i / kStages) & 1, epi.wait_ns)) {
        fail = kStatusTimeoutTma;
        break;
      }
      tc_fence_after();
      const uint64_t da = sw128_desc(sA + s * kBytesA), db = sw128_desc(sB + s * kBytesB);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)
        umma_bf16(tmem_d, da + 2 * kk, db + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      umma_commit(empty(s));
    }
    umma_commit(done);
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0, epi.wait_ns);
  if (!ok && threadIdx.x == 0) fail |= kStatusTimeoutMma;
  if (fail) atomicOr(status, fail);
  const bool any_fail = __syncthreads_or(fail != 0 || !ok) != 0;
  tc_fence_after();

  if (!any_fail && warp < 4) epilogue<BN>(tmem_d, m0, n0, Mrows, N, 0, epi, warp, out_row);

  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(tmem_cols<BN>())
                 : "memory");
  }
}

// MODE 0 (forward): x [B][H][W][C], rows = output pixels; MODE 1 / 2 (input gradient): x = the output
// gradient [B][Ho][Wo][C] (C = the convolution's cout), rows = the B x H x W input pixels (MODE 2 in
// parity classes, C a multiple of 64)
template <int BN, int MODE>
cudaError_t launch_conv_bn(const __nv_bfloat16* x, int B, int H, int W, int C, const CUtensorMap& tb, int N,
                           const GemmEpi& epi, int* status, cudaStream_t s) {
  const size_t smem = gemm_smem_bytes(BN);
  cudaError_t e =
      cudaFuncSetAttribute(k_conv3x3s2_implicit<BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  constexpr bool DGRAD = MODE != 0;
  const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
  const int SH = DGRAD ? Ho : H, SW = DGRAD ? Wo : W, OH = DGRAD ? H : Ho, OW = DGRAD ? W : Wo;
  const long long M = (long long)B * OH * OW;
  if (M > 0x7fffffffLL) return cudaErrorInvalidValue;
  int4 ctile = make_int4(0, 0, 0, 0);
  long long blocks = (M + kBM - 1) / kBM;
  int m_arg = (int)M;
  if (MODE == 2) {
    if (C % kBK) return cudaErrorInvalidValue;
    long long acc = 0, cum[4];
    for (int c = 0; c < 4; ++c) {
      const long long rows = (long long)B * ((H + 1 - (c >> 1)) / 2) * ((W + 1 - (c & 1)) / 2);
      acc += (rows + kBM - 1) / kBM;
      cum[c] = acc;
    }
    ctile = make_int4((int)cum[0], (int)cum[1], (int)cum[2], (int)cum[3]);
    blocks = acc;
    m_arg = B;
  }
  if (blocks < 1) return cudaSuccess;
  dim3 grid((unsigned)blocks, (N + BN - 1) / BN, 1);
  k_conv3x3s2_implicit<BN, MODE><<<grid, kConvThreads, smem, s>>>(x, SH, SW, C, OH, OW, tb, m_arg, N, epi, status,
                                                                  ctile);
  return cudaGetLastError();
}

}  // namespace

size_t gemm_smem_bytes(int bn) {
  return 1024 + (size_t)kStages * (kBM * kBK * 2 + (size_t)bn * kBK * 2) + 8 * (2 * kStages + 1) + 16;
}

cudaError_t launch_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int bn, int pair,
                        int split, int kb_per_split, const GemmEpi& epi, int* status, cudaStream_t s) {
  if (pair == 2) return launch_pair_persistent(ta, tb, M, N, K, split, kb_per_split, epi, status, s);
  if (pair) return launch_pair(ta, tb, M, N, K, split, kb_per_split, epi, status, s);  // 2-SM 256 x 256 tiles
  switch (bn) {
    case 32: return launch_bn<32>(ta, tb, M, N, K, split, kb_per_split, epi, status, s);
    case 64: return launch_bn<64>(ta, tb, M, N, K, split, kb_per_split, epi, status, s);
    case 128: return launch_bn<128>(ta, tb, M, N, K, split, kb_per_split, epi, status, s);
    case 256: return launch_bn<256>(ta, tb, M, N, K, split, kb_per_split, epi, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_implicit(const __nv_bfloat16* x, int B, int H, int W, int C, const CUtensorMap& tw, int cout,
                                 int bn, const GemmEpi& epi, int* status, cudaStream_t s) {
  switch (bn) {
    case 32: return launch_conv_bn<32, 0>(x, B, H, W, C, tw, cout, epi, status, s);
    case 64: return launch_conv_bn<64, 0>(x, B, H, W, C, tw, cout, epi, status, s);
    case 128: return launch_conv_bn<128, 0>(x, B, H, W, C, tw, cout, epi, status, s);
    case 256: return launch_conv_bn<256, 0>(x, B, H, W, C, tw, cout, epi, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_conv_dgrad_implicit(const __nv_bfloat16* dy, int B, int H, int W, int cout, const CUtensorMap& twt,
                                       int C, int bn, const GemmEpi& epi, int* status, cudaStream_t s) {
  // by parity class (each input pixel only over the taps that reach an output pixel) when a K block of
  // 64 channels never straddles two taps; else every input pixel over all 9 taps
  if (cout % kBK == 0) {
    switch (bn) {
      case 32: return launch_conv_bn<32, 2>(dy, B, H, W, cout, twt, C, epi, status, s);
      case 64: return launch_conv_bn<64, 2>(dy, B, H, W, cout, twt, C, epi, status, s);
      case 128: return launch_conv_bn<128, 2>(dy, B, H, W, cout, twt, C, epi, status, s);
      case 256: return launch_conv_bn<256, 2>(dy, B, H, W, cout, twt, C, epi, status, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (bn) {
    case 32: return launch_conv_bn<32, 1>(dy, B, H, W, cout, twt, C, epi, status, s);
    case 64: return launch_conv_bn<64, 1>(dy, B, H, W, cout, twt, C, epi, status, s);
    case 128: return launch_conv_bn<128, 1>(dy, B, H, W, cout, twt, C, epi, status, s);
    case 256: return launch_conv_bn<256, 1>(dy, B, H, W, cout, twt, C, epi, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_split_reduce(const float* part, int split, int M, int N, const GemmEpi& epi, cudaStream_t s) {
  const long long total = (long long)M * N;
  long long blocks = (total + 255) / 256;
  if (blocks > 148LL * 16) blocks = 148LL * 16;
  k_split_reduce<<<(int)(blocks < 1 ? 1 : blocks), 256, 0, s>>>(part, split, M, N, epi);
  return cudaGetLastError();
}

}  // namespace pnk
