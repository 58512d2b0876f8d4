// Launchers of the paired-column warp wavefront (kernel body in
// gg_stepw2.cuh): strips of 64 columns, two per lane.
//
// CTA size: one warp per CTA for T >= 2 (the warps share nothing, and the
// per-CTA register granule is one warp); the one-step pass, HBM-bound and
// short-lived, uses 4-warp CTAs.  Each warp has its own shared-memory ring
// (stepw2::Ring: 12 KB with Kahan terms, 9 KB without), passed as dynamic
// shared memory.
#include "gg_stepw2.cuh"

namespace gg {
namespace {

// Dynamic shared memory: one stepw2::Ring per warp of the CTA.
extern __shared__ float2 g_ring2[];

// Resident warps an SM must hold (the register cap it implies): T = 4 with
// Kahan terms fits 167 registers without spills, 12 warps per SM (182 and 11
// warps without the bound; 337 against 359 G cell-steps/s on the 8192^2
// tissue); a bound of 13 would force spills.  T <= 3 keep the compiler's
// choice: bounds of 14 (T = 3) and 16 (T = 2) measured 33 % slower.
template <int T> constexpr int min_warps2() { return T == 4 ? 12 : 1; }

template <int T, bool KAHAN>
__global__ void __launch_bounds__(32, min_warps2<T>()) stepw2_kernel(const Grid32 g, const Rates32 k, const int H, const int nstrips,
                                                    const int nwarps)
{
    const int gw = blockIdx.x;
    if (gw >= nwarps) return;
    chained_wait();  // launched with launch_chained
    stepw2::warp_pass2_any<T, KAHAN>(g, live_rates(k), H, gw % nstrips, gw / nstrips, threadIdx.x, g_ring2);
}

template <bool KAHAN>
__global__ void __launch_bounds__(128) stepw2_1_kernel(const Grid32 g, const Rates32 k, const int H,
                                                       const int nstrips, const int nwarps)
{
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * 4 + wid;
    if (gw >= nwarps) return;  // whole warps only
    chained_wait();            // launched with launch_chained
    stepw2::warp_pass2_any<1, KAHAN>(g, live_rates(k), H, gw % nstrips, gw / nstrips, threadIdx.x & 31,
                                     g_ring2 + wid * (stepw2::Ring<KAHAN>::bytes / 8));
}

// SMASK: the levels that write the stash (bit t - 1 for level t).
template <int T, bool KAHAN, int SMASK>
__global__ void __launch_bounds__(32, min_warps2<T>()) stepw2_stash_kernel(const Grid32 g, const Rates32 k, const int H,
                                                          const int nstrips, const int nwarps, const Stash32 st)
{
    const int gw = blockIdx.x;
    if (gw >= nwarps) return;
    chained_wait();  // launched with launch_chained
    stepw2::warp_pass2_any<T, KAHAN, SMASK>(g, live_rates(k), H, gw % nstrips, gw / nstrips, threadIdx.x, g_ring2,
                                            &st);
}

template <int T> inline int strips2(int nx) { return (nx + stepw2::Geom<T>::OUT - 1) / stepw2::Geom<T>::OUT; }

template <int T, bool KAHAN>
cudaError_t launch_w2(const Grid32& g, const Rates32& r, int H, cudaStream_t s)
{
    const int nstrips = strips2<T>(g.nx);
    const int nwarps = nstrips * ((g.ny + H - 1) / H);
    constexpr int rb = stepw2::Ring<KAHAN>::bytes;
    if constexpr (T == 1)
        return launch_chained(stepw2_1_kernel<KAHAN>, (nwarps + 3) / 4, 128, 4 * rb, s, g, r, H, nstrips, nwarps);
    else
        return launch_chained(stepw2_kernel<T, KAHAN>, nwarps, 32, rb, s, g, r, H, nstrips, nwarps);
}

template <int T, bool KAHAN, int SMASK>
cudaError_t launch_ws2m(const Grid32& g, const Rates32& r, int H, const Stash32& st, cudaStream_t s)
{
    const int nstrips = strips2<T>(g.nx);
    const int nwarps = nstrips * ((g.ny + H - 1) / H);
    return launch_chained(stepw2_stash_kernel<T, KAHAN, SMASK>, nwarps, 32, stepw2::Ring<KAHAN>::bytes, s, g, r, H,
                          nstrips, nwarps, st);
}

// The stash set of a pass is that of its destinations (the non-null ones).
// The adjoint stores the states at even steps, so level t of a pass from step
// s0 writes when s0 + t is even: for T = 4 levels {2} (s0 even) or {1, 3}
// (s0 odd), for T = 3 {2} or {1}, for T = 2 none or {1}.  Those sets have
// kernels; a pass that writes no level runs the plain kernel, any other set is
// refused.
template <int T, bool KAHAN>
cudaError_t launch_ws2(const Grid32& g, const Rates32& r, int H, const Stash32& st, cudaStream_t s)
{
    int m = 0;
    for (int li = 0; li < T - 1; ++li)
        if (st.u[li]) m |= 1 << li;
    if (m == 0) return launch_w2<T, KAHAN>(g, r, H, s);
    if constexpr (T == 2) {
        if (m == 1) return launch_ws2m<2, KAHAN, 1>(g, r, H, st, s);
    } else if constexpr (T == 3) {
        if (m == 2) return launch_ws2m<3, KAHAN, 2>(g, r, H, st, s);
        if (m == 1) return launch_ws2m<3, KAHAN, 1>(g, r, H, st, s);
    } else {
        if (m == 2) return launch_ws2m<4, KAHAN, 2>(g, r, H, st, s);
        if (m == 5) return launch_ws2m<4, KAHAN, 5>(g, r, H, st, s);
    }
    return cudaErrorInvalidValue;
}

template <int T, bool KAHAN>
int wave_warps2_T()
{
    constexpr int wpc = T == 1 ? 4 : 1;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        constexpr int rb = stepw2::Ring<KAHAN>::bytes;
        if constexpr (T == 1)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stepw2_1_kernel<KAHAN>, 128, 4 * rb);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stepw2_kernel<T, KAHAN>, 32, rb);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * wpc * sms;
}

}  // namespace

int stepw2_out_columns(int T) { return T <= 2 ? stepw2::Geom<1>::OUT : stepw2::Geom<3>::OUT; }

int stepw2_wave_warps(int T, bool kahan)
{
    switch (T) {
        case 1: return kahan ? wave_warps2_T<1, true>() : wave_warps2_T<1, false>();
        case 2: return kahan ? wave_warps2_T<2, true>() : wave_warps2_T<2, false>();
        case 3: return kahan ? wave_warps2_T<3, true>() : wave_warps2_T<3, false>();
        case 4: return kahan ? wave_warps2_T<4, true>() : wave_warps2_T<4, false>();
        default: return 0;
    }
}

cudaError_t launch_stepw2(const Grid32& g, const Rates32& r, int H, int T, bool kahan, cudaStream_t s)
{
    if (H < 1) return cudaErrorInvalidValue;
    switch (T) {
        case 1: return kahan ? launch_w2<1, true>(g, r, H, s) : launch_w2<1, false>(g, r, H, s);
        case 2: return kahan ? launch_w2<2, true>(g, r, H, s) : launch_w2<2, false>(g, r, H, s);
        case 3: return kahan ? launch_w2<3, true>(g, r, H, s) : launch_w2<3, false>(g, r, H, s);
        case 4: return kahan ? launch_w2<4, true>(g, r, H, s) : launch_w2<4, false>(g, r, H, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stepw2_stash(const Grid32& g, const Rates32& r, int H, int T, bool kahan, const Stash32& st,
                                cudaStream_t s)
{
    if (H < 1) return cudaErrorInvalidValue;
    switch (T) {
        case 1: return kahan ? launch_w2<1, true>(g, r, H, s) : launch_w2<1, false>(g, r, H, s);
        case 2: return kahan ? launch_ws2<2, true>(g, r, H, st, s) : launch_ws2<2, false>(g, r, H, st, s);
        case 3: return kahan ? launch_ws2<3, true>(g, r, H, st, s) : launch_ws2<3, false>(g, r, H, st, s);
        case 4: return kahan ? launch_ws2<4, true>(g, r, H, st, s) : launch_ws2<4, false>(g, r, H, st, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gg
