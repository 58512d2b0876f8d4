// Launchers of the warp-register wavefront step (kernel body in gg_stepw.cuh).
//
// CTA size: for T >= 2 one warp per CTA (stepw_kernel).  The warps share
// nothing, and under a 32-thread bound the compiler keeps the Kahan kernels
// at 123 (T = 3) and 137 (T = 4) registers without spills, so that 16 (14)
// warps fit on an SM; with 4-warp CTAs the (scalar) T = 3 kernel took 135
// registers and the SM held 12 warps: 183 against 225 G cell-steps/s on the
// 8192^2 tissue.  The one-step pass (stepw1_kernel, HBM-bound, short-lived
// warps) keeps 4-warp CTAs bound to 6 or 8 per SM: 105 against 96 G
// cell-steps/s with one warp per CTA.
#include "gg_stepw.cuh"

namespace gg {
namespace {

template <int T> constexpr int warps_per_cta() { return T == 1 ? 4 : 1; }

template <int T, bool KAHAN>
__global__ void __launch_bounds__(32) stepw_kernel(const Grid32 g, const Rates32 k, const int H, const int nstrips,
                                                   const int nwarps)
{
    const int lane = threadIdx.x;
    const int gw = blockIdx.x;
    if (gw >= nwarps) return;
    chained_wait();  // launched with launch_chained
    const int strip = gw % nstrips, chunk = gw / nstrips;
    stepw::warp_pass_any<T, KAHAN>(g, live_rates(k), H, strip, chunk, lane);
}

// The one-step pass needs occupancy to hide HBM latency: 4-warp CTAs, bound
// to 8 per SM without Kahan terms (64 registers) and 6 with them (80).
template <bool KAHAN>
__global__ void __launch_bounds__(128, KAHAN ? 6 : 8) stepw1_kernel(const Grid32 g, const Rates32 k, const int H,
                                                                     const int nstrips, const int nwarps)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (gw >= nwarps) return;  // whole warps only
    chained_wait();            // launched with launch_chained
    const int strip = gw % nstrips, chunk = gw / nstrips;
    stepw::warp_pass_any<1, KAHAN>(g, live_rates(k), H, strip, chunk, lane);
}

template <int T, bool KAHAN>
cudaError_t launch_w(const Grid32& g, const Rates32& r, int H, cudaStream_t s)
{
    constexpr int OUT = 32 - 2 * T;
    const int nstrips = (g.nx + OUT - 1) / OUT;
    const int nchunks = (g.ny + H - 1) / H;
    const int nwarps = nstrips * nchunks;
    if constexpr (T == 1)
        return launch_chained(stepw1_kernel<KAHAN>, (nwarps + 3) / 4, 128, 0, s, g, r, H, nstrips, nwarps);
    else
        return launch_chained(stepw_kernel<T, KAHAN>, nwarps, 32, 0, s, g, r, H, nstrips, nwarps);
}

template <int T, bool KAHAN>
int wave_warps_T()
{
    constexpr int wpc = warps_per_cta<T>();
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if constexpr (T == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stepw1_kernel<KAHAN>, 128, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stepw_kernel<T, KAHAN>, 32, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * wpc * sms;
}

}  // namespace

int stepw_wave_warps(int T, bool kahan)
{
    switch (T) {
        case 1: return kahan ? wave_warps_T<1, true>() : wave_warps_T<1, false>();
        case 2: return kahan ? wave_warps_T<2, true>() : wave_warps_T<2, false>();
        case 3: return kahan ? wave_warps_T<3, true>() : wave_warps_T<3, false>();
        case 4: return kahan ? wave_warps_T<4, true>() : wave_warps_T<4, false>();
        default: return 0;
    }
}

cudaError_t launch_stepw(const Grid32& g, const Rates32& r, int H, int T, bool kahan, cudaStream_t s)
{
    if (H < 1) return cudaErrorInvalidValue;
    switch (T) {
        case 1: return kahan ? launch_w<1, true>(g, r, H, s) : launch_w<1, false>(g, r, H, s);
        case 2: return kahan ? launch_w<2, true>(g, r, H, s) : launch_w<2, false>(g, r, H, s);
        case 3: return kahan ? launch_w<3, true>(g, r, H, s) : launch_w<3, false>(g, r, H, s);
        case 4: return kahan ? launch_w<4, true>(g, r, H, s) : launch_w<4, false>(g, r, H, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gg
