// Instantiates the fast-path term kernels for FP32 contractions, one problem per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_launch_f32(const KParams &kp, const FastLaunch &a) { return launch_t<float>(kp, a); }

}  // namespace sg
