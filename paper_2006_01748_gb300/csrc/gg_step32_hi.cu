// FP32 step launchers for T = 5..8 steps per pass (kernel in gg_step32.cuh).
#include "gg_step32.cuh"

namespace gg {

cudaError_t launch_step32_hi(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan, cudaStream_t s)
{
    using namespace step32;
    switch (T) {
        case 5: return kahan ? launch_T<5, true>(g, r, p, s) : launch_T<5, false>(g, r, p, s);
        case 6: return kahan ? launch_T<6, true>(g, r, p, s) : launch_T<6, false>(g, r, p, s);
        case 7: return kahan ? launch_T<7, true>(g, r, p, s) : launch_T<7, false>(g, r, p, s);
        case 8: return kahan ? launch_T<8, true>(g, r, p, s) : launch_T<8, false>(g, r, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gg
