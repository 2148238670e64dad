// Pose optimiser of the registration and motion-compensation loops: one Adam
// step on an [n][6] pose array in one launch (the loops the paper runs with
// Adam, Sec. II-D.3), with a per-pose step count so that a pose's bias
// correction counts only its own updates.
#include "proj_internal.cuh"
#include "proj_optim.cuh"

namespace projk {

namespace {

// One thread per pose; inactive poses are left untouched.
__global__ void k_pose_adam(float* __restrict__ pose, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float* __restrict__ t, const unsigned char* __restrict__ active,
                            int n, PoseAdam h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (active && !active[i])) return;
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

}  // namespace

cudaError_t launch_pose_adam(float* d_pose, const float* d_grad, float* d_m, float* d_v, float* d_t,
                             const unsigned char* d_active, int n, const PoseAdam& h, cudaStream_t s) {
  k_pose_adam<<<ceil_div(n, 128), 128, 0, s>>>(d_pose, d_grad, d_m, d_v, d_t, d_active, n, h);
  return cudaGetLastError();
}

}  // namespace projk
