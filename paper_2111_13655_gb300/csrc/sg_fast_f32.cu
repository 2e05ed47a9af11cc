// Instantiates the fast-path term kernels for FP32 contractions, one problem per launch.
#include "sg_fast.cuh"

namespace sg {

cudaError_t fast_launch_f32(const KParams &kp, const FastLaunch &a)
{
    return for_variant<float>(kp, [&](auto v) {
        using V = decltype(v);
        return launch_t<float, V::NB1, V::NQ1, V::RMAX, V::UNI>(kp, a);
    });
}

}  // namespace sg
