// Instantiates the fast-path term kernels for FP64 contractions, many problems per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_batch_launch_f64(const KParams &, const FastBatchLaunch &a) { return batch_t<double>(a); }

}  // namespace sg
