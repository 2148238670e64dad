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

constexpr float kDegPerRad = 57.295779513082321f;

// One iteration's bookkeeping of a multi-start registration (proj_registration_step).
struct RegStep {
  int n, n_slots;
  float* pose;
  const float* grad;
  const float* loss;
  float* last;
  float *m, *v, *t;
  unsigned char* alive;
  long long* iters;
  int* slots;
  long long* next;
  const float* truth;  // [n_truth][6] or null
  int n_truth;
  unsigned char* hit_any;
  unsigned char* listed;  // [n] scratch
  float ncc_stop, dloss_stop, tol_mm, tol_deg;
  long long max_iter;
  PoseAdam adam;
};
cudaError_t launch_registration_step(const RegStep& r, cudaStream_t s);

}  // namespace projk
