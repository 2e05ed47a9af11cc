// Instantiates the fast-path term kernels for FP64 contractions, many problems per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_batch_launch_f64(const KParams &kp_any, const FastBatchLaunch &a)
{
    return for_variant<double>(kp_any, [&](auto v) {
        using V = decltype(v);
        return batch_t<double, V::NB1, V::NQ1, V::RMAX, V::UNI>(a);
    });
}

}  // namespace sg
