// Instantiates the fast-path term kernels for double-float contractions
// (pairs of FP32 numbers on the FP32 pipes), one problem per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_launch_df(const KParams &kp, const FastLaunch &a) { return launch_t<df2>(kp, a); }

}  // namespace sg
