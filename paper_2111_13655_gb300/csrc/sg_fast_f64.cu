// Instantiates the fast-path term kernels for FP64 contractions, one problem per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_launch_f64(const KParams &kp, const FastLaunch &a)
{
    return for_variant<double>(kp, [&](auto v) {
        using V = decltype(v);
        return launch_t<double, V::NB1, V::NQ1, V::RMAX, V::UNI>(kp, a);
    });
}

}  // namespace sg
