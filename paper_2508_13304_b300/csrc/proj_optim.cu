// Pose optimiser of the registration and motion-compensation loops: one Adam
// step on an [n][6] pose array in one launch (the loops the paper runs with
// Adam, Sec. II-D.3), with a per-pose step count so that a pose's bias
// correction counts only its own updates; and the whole per-iteration
// bookkeeping of a multi-start registration (hit test, stopping test, masked
// Adam step, refill of the slots of stopped starts) in one launch.
#include "proj_internal.cuh"
#include "proj_optim.cuh"

namespace projk {

namespace {

__device__ __forceinline__ void adam_row(float* __restrict__ pose, const float* __restrict__ grad,
                                         float* __restrict__ m, float* __restrict__ v, float* __restrict__ t, int i,
                                         const PoseAdam& h) {
  const float ti = t[i] + 1.f;
  t[i] = ti;
  const float c1 = 1.f - powf(h.b1, ti), c2 = 1.f - powf(h.b2, ti);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const size_t k = (size_t)i * 6 + j;
    const float g = grad[k];
    const float mj = h.b1 * m[k] + h.a1 * g;
    const float vj = h.b2 * v[k] + h.a2 * g * g;
    m[k] = mj;
    v[k] = vj;
    pose[k] -= h.lr[j] * (mj / c1) / (sqrtf(vj / c2) + h.eps);
  }
}

// One thread per pose; inactive poses are left untouched.
__global__ void k_pose_adam(float* __restrict__ pose, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float* __restrict__ t, const unsigned char* __restrict__ active,
                            int n, PoseAdam h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (active && !active[i])) return;
  adam_row(pose, grad, m, v, t, i, h);
}

constexpr int kRegThreads = 1024;

// One block: (1) mark the poses the slots list, (2) per listed pose the hit
// test, the stopping test, the masked Adam step and the loss history, (3)
// refill the slots of stopped starts with the next starts in order (a block
// scan over the slots).  Every phase reads what the previous one wrote, so
// the phases are separated by block barriers; no other block takes part.
__global__ void __launch_bounds__(kRegThreads) k_registration_step(RegStep r) {
  __shared__ int scan[kRegThreads];
  const int t = threadIdx.x;
  for (int i = t; i < r.n; i += kRegThreads) r.listed[i] = 0;
  __syncthreads();
  for (int s = t; s < r.n_slots; s += kRegThreads) {
    const int p = r.slots[s];
    if (p >= 0 && p < r.n) r.listed[p] = 1;
  }
  __syncthreads();
  for (int i = t; i < r.n; i += kRegThreads) {
    if (!r.listed[i]) continue;
    if (r.truth) {
      const float* tp = r.truth + 6 * (r.n_truth == 1 ? 0 : i);
      bool hit = true;
      for (int j = 0; j < 3; ++j) hit = hit && fabsf(r.pose[6 * i + j] - tp[j]) <= r.tol_mm;
      for (int j = 3; j < 6; ++j) hit = hit && fabsf(r.pose[6 * i + j] - tp[j]) * kDegPerRad <= r.tol_deg;
      if (hit) *r.hit_any = 1;  // every writer stores the same value
    }
    const float L = r.loss[i];
    const bool done = -L >= r.ncc_stop || fabsf(r.last[i] - L) < r.dloss_stop || r.iters[i] >= r.max_iter;
    if (done) r.alive[i] = 0;
    if (r.alive[i]) {
      r.iters[i] += 1;
      adam_row(r.pose, r.grad, r.m, r.v, r.t, i, r.adam);
    }
    r.last[i] = L;
  }
  __syncthreads();
  // refill: slot s is free when it is empty or its start has stopped; the free slots take the next
  // starts in slot order (exclusive prefix count of the free slots before s)
  const int chunks = (r.n_slots + kRegThreads - 1) / kRegThreads;
  long long base = *r.next;
  for (int c = 0; c < chunks; ++c) {
    const int s = c * kRegThreads + t;
    int p = -1;
    bool free = false;
    if (s < r.n_slots) {
      p = r.slots[s];
      free = p < 0 || p >= r.n || !r.alive[p];
    }
    scan[t] = free ? 1 : 0;
    __syncthreads();
    for (int o = 1; o < kRegThreads; o <<= 1) {
      const int add = t >= o ? scan[t - o] : 0;
      __syncthreads();
      scan[t] += add;
      __syncthreads();
    }
    const long long cand = base + scan[t] - (free ? 1 : 0);
    const int total = scan[kRegThreads - 1];
    if (s < r.n_slots && free) r.slots[s] = cand < r.n ? (int)cand : -1;
    __syncthreads();  // every thread has read scan before the next chunk overwrites it
    base += total;
  }
  if (t == 0) *r.next = base < r.n ? base : (long long)r.n;
}

}  // namespace

cudaError_t launch_pose_adam(float* d_pose, const float* d_grad, float* d_m, float* d_v, float* d_t,
                             const unsigned char* d_active, int n, const PoseAdam& h, cudaStream_t s) {
  k_pose_adam<<<ceil_div(n, 128), 128, 0, s>>>(d_pose, d_grad, d_m, d_v, d_t, d_active, n, h);
  return cudaGetLastError();
}

cudaError_t launch_registration_step(const RegStep& r, cudaStream_t s) {
  k_registration_step<<<1, kRegThreads, 0, s>>>(r);
  return cudaGetLastError();
}

}  // namespace projk
