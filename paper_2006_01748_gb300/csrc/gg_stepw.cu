// Launchers of the warp-register wavefront step (kernel body in gg_stepw.cuh).
#include "gg_stepw.cuh"

namespace gg {
namespace {

template <int T, bool KAHAN>
__global__ void __launch_bounds__(128) stepw_kernel(const Grid32 g, const Rates32 k, const int H, const int nstrips,
                                                    const int nwarps)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= nwarps) return;  // whole warps only
    const int strip = gw % nstrips, chunk = gw / nstrips;
    stepw::warp_pass_any<T, KAHAN>(g, k, H, strip, chunk, lane);
}

template <int T, bool KAHAN>
__global__ void __launch_bounds__(128) stepw_stash_kernel(const Grid32 g, const Rates32 k, const int H,
                                                          const int nstrips, const int nwarps, const Stash32 st)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
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
    stepw_stash_kernel<T, KAHAN><<<(nwarps + 3) / 4, 128, 0, s>>>(g, r, H, nstrips, nwarps, st);
    return cudaGetLastError();
}

template <int T, bool KAHAN>
cudaError_t launch_w(const Grid32& g, const Rates32& r, int H, cudaStream_t s)
{
    constexpr int OUT = 32 - 2 * T;
    const int nstrips = (g.nx + OUT - 1) / OUT;
    const int nchunks = (g.ny + H - 1) / H;
    const int nwarps = nstrips * nchunks;
    const int wpb = 4;
    stepw_kernel<T, KAHAN><<<(nwarps + wpb - 1) / wpb, 32 * wpb, 0, s>>>(g, r, H, nstrips, nwarps);
    return cudaGetLastError();
}

}  // namespace

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
