// Instantiates the fast-path term kernels for FP64 contractions, one problem per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_launch_f64(const KParams &kp, const FastLaunch &a) { return launch_t<double>(kp, a); }

}  // namespace sg
