// FP32 step launchers for T = 1..4 steps per pass (kernel in gg_step32.cuh).
#include "gg_step32.cuh"

namespace gg {

cudaError_t launch_step32_lo(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan, cudaStream_t s)
{
    using namespace step32;
    switch (T) {
        case 1: return kahan ? launch_T<1, true>(g, r, p, s) : launch_T<1, false>(g, r, p, s);
        case 2: return kahan ? launch_T<2, true>(g, r, p, s) : launch_T<2, false>(g, r, p, s);
        case 3: return kahan ? launch_T<3, true>(g, r, p, s) : launch_T<3, false>(g, r, p, s);
        case 4: return kahan ? launch_T<4, true>(g, r, p, s) : launch_T<4, false>(g, r, p, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t step32_smem_bytes(const Plan32& p, bool kahan)
{
    const int sw = p.bx + 2 * p.halo;
    return (size_t)sw * sizeof(float) * (p.T * 9 + (kahan ? p.T * 6 : 0) + 3 * (p.T + 2));
}

cudaError_t launch_step32_hi(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan, cudaStream_t s);

cudaError_t launch_step32(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan, cudaStream_t s)
{
    if (T < 1 || T > kMaxT || p.halo < T) return cudaErrorInvalidValue;
    return T <= 4 ? launch_step32_lo(g, r, p, T, kahan, s) : launch_step32_hi(g, r, p, T, kahan, s);
}

cudaError_t launch_plan(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan, cudaStream_t s)
{
    if (p.kind == 1 && T <= 4) return launch_stepw(g, r, p.by, T, kahan, s);
    if (p.kind == 3 && T <= 4) return launch_stepw2(g, r, p.by, T, kahan, s);
    Plan32 q = p;
    if (q.halo < T) q.halo = T;
    return launch_step32(g, r, q, T, kahan, s);
}

}  // namespace gg
