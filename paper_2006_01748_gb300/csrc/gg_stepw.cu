// Launchers of the warp-register wavefront step (kernel body in gg_stepw.cuh).
//
// CTA size: for T >= 2 one warp per CTA.  The warps share nothing, and with
// a 32-thread bound the compiler keeps the T = 3 Kahan kernel at 120
// registers (T = 4 at 152) without spills, so that 17 (13) warps fit on an
// SM; with 4-warp CTAs it allocated 135 (168, with spills) and the SM held
// 12.  Measured on the 8192^2 tissue: T = 3 225 vs 183 G cell-steps/s.  The
// T = 1 kernel (64 registers, short-lived warps) keeps 4-warp CTAs, which
// measured 105 vs 96 G cell-steps/s.
#include "gg_stepw.cuh"

namespace gg {
namespace {

template <int T> constexpr int warps_per_cta() { return T == 1 ? 4 : 1; }

template <int T, bool KAHAN>
__global__ void __launch_bounds__(32 * warps_per_cta<T>()) stepw_kernel(const Grid32 g, const Rates32 k, const int H,
                                                                        const int nstrips, const int nwarps)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * warps_per_cta<T>() + (threadIdx.x >> 5);
    if (gw >= nwarps) return;  // whole warps only
    const int strip = gw % nstrips, chunk = gw / nstrips;
    stepw::warp_pass_any<T, KAHAN>(g, k, H, strip, chunk, lane);
}

template <int T, bool KAHAN>
__global__ void __launch_bounds__(32) stepw_stash_kernel(const Grid32 g, const Rates32 k, const int H,
                                                         const int nstrips, const int nwarps, const Stash32 st)
{
    const int lane = threadIdx.x;
    const int gw = blockIdx.x;
    if (gw >= nwarps) return;
    const int strip = gw % nstrips, chunk = gw / nstrips;
    stepw::warp_pass_any<T, KAHAN, false, true>(g, k, H, strip, chunk, lane, &st);
}

template <int T, bool KAHAN>
cudaError_t launch_ws(const Grid32& g, const Rates32& r, int H, const Stash32& st, cudaStream_t s)
{
    constexpr int OUT = 32 - 2 * T;
    const int nstrips = (g.nx + OUT - 1) / OUT;
    const int nchunks = (g.ny + H - 1) / H;
    const int nwarps = nstrips * nchunks;
    stepw_stash_kernel<T, KAHAN><<<nwarps, 32, 0, s>>>(g, r, H, nstrips, nwarps, st);
    return cudaGetLastError();
}

template <int T, bool KAHAN>
cudaError_t launch_w(const Grid32& g, const Rates32& r, int H, cudaStream_t s)
{
    constexpr int OUT = 32 - 2 * T;
    const int nstrips = (g.nx + OUT - 1) / OUT;
    const int nchunks = (g.ny + H - 1) / H;
    const int nwarps = nstrips * nchunks;
    constexpr int wpc = warps_per_cta<T>();
    stepw_kernel<T, KAHAN><<<(nwarps + wpc - 1) / wpc, 32 * wpc, 0, s>>>(g, r, H, nstrips, nwarps);
    return cudaGetLastError();
}

template <int T, bool KAHAN>
int wave_warps_T()
{
    constexpr int wpc = warps_per_cta<T>();
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stepw_kernel<T, KAHAN>, 32 * wpc, 0) != cudaSuccess) {
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

cudaError_t launch_stepw_stash(const Grid32& g, const Rates32& r, int H, int T, bool kahan, const Stash32& st,
                               cudaStream_t s)
{
    if (H < 1) return cudaErrorInvalidValue;
    switch (T) {
        case 1: return kahan ? launch_w<1, true>(g, r, H, s) : launch_w<1, false>(g, r, H, s);
        case 2: return kahan ? launch_ws<2, true>(g, r, H, st, s) : launch_ws<2, false>(g, r, H, st, s);
        case 3: return kahan ? launch_ws<3, true>(g, r, H, st, s) : launch_ws<3, false>(g, r, H, st, s);
        case 4: return kahan ? launch_ws<4, true>(g, r, H, st, s) : launch_ws<4, false>(g, r, H, st, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gg
