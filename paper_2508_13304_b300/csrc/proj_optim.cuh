// Pose optimiser of the registration and motion-compensation loops (not part
// of the C ABI; proj_pose_adam in include/proj.h is its entry point).
#pragma once

#include <cuda_runtime.h>

namespace projk {

// Adam hyper-parameters (a1 = 1 - b1, a2 = 1 - b2 at full precision).
struct PoseAdam {
  float lr[6];
  float b1, a1, b2, a2, eps;
};

cudaError_t launch_pose_adam(float* d_pose, const float* d_grad, float* d_m, float* d_v, float* d_t,
                             const unsigned char* d_active, int n, const PoseAdam& h, cudaStream_t s);

}  // namespace projk
