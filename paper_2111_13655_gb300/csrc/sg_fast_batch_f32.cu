// Instantiates the fast-path term kernels for FP32 contractions, many problems per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_batch_launch_f32(const KParams &, const FastBatchLaunch &a) { return batch_t<float>(a); }

}  // namespace sg
