// The adaptive step Delta t_k (Section 2 recomputes it after each iteration
// to keep the scheme stable, without a formula), computed on the device from
// the state so that the time loop needs no host round trip.
//
// Reading (the same as the FP64 oracle's): Delta t_k is the largest step for
// which the coefficient of each unknown's own old value in eq. (3) stays at
// least 1 - cfl on the state X^k:
//   kU = U + delta W - 1                        (U' = U (1 + dt (1 - U - delta W)))
//   kV = D S - rho (1 - V),  S = sum over the interior faces f of the cell of
//        (1 - (U_P + U_nb)/2) / h_f^2           (the tumour flux of Table 1)
//   kW = c + 2 Lambda_A (1/dx^2 + 1/dy^2)       (the acid operator's bound,
//                                                static because A is)
//   Delta t_k = cfl / max(kW, max_cells kU, max_cells kV)
// (without reactions the reaction parts are left out).  adapt_reduce_kernel
// takes the two maxima over the grid (per-thread, warp-shuffle and
// shared-memory maxima, one atomicMax per block on the bit pattern of a
// non-negative value: the maxima are clamped at 0, below kW > 0, so the
// ordering of the bit patterns is that of the values); adapt_finish_kernel
// turns them into Delta t_k, advances the simulated time by the steps taken
// with the previous Delta t, and clears the maxima for the next reduction.
// The per-cell terms are evaluated in the state's precision.
#include <math.h>

#include <algorithm>

#include "gg_internal.cuh"

namespace gg {
namespace {

template <typename F> struct Bits;
template <> struct Bits<float> {
    using U = unsigned int;
    static __device__ U of(float x) { return __float_as_uint(x); }
};
template <> struct Bits<double> {
    using U = unsigned long long;
    static __device__ U of(double x) { return (U)__double_as_longlong(x); }
};

template <typename F>
__global__ void __launch_bounds__(256) adapt_reduce_kernel(const F* __restrict__ u, const F* __restrict__ v,
                                                           const F* __restrict__ w, int nx, int ny, int pitch,
                                                           AdaptRule<F> r, typename Bits<F>::U* kmax)
{
    F mU = 0, mV = 0;
    const size_t n = (size_t)nx * ny;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const size_t o = (size_t)j * pitch + i;
        const F up = u[o], vp = v[o], wp = w[o];
        F S = 0;
        if (i + 1 < nx) S += (F(1) - F(0.5) * (up + u[o + 1])) * r.ihx2;
        if (i > 0) S += (F(1) - F(0.5) * (up + u[o - 1])) * r.ihx2;
        if (j + 1 < ny) S += (F(1) - F(0.5) * (up + u[o + pitch])) * r.ihy2;
        if (j > 0) S += (F(1) - F(0.5) * (up + u[o - pitch])) * r.ihy2;
        const F ku = r.no_reaction ? F(0) : up + r.delta * wp - F(1);
        const F kv = r.D * S - (r.no_reaction ? F(0) : r.rho * (F(1) - vp));
        mU = fmax(mU, ku);  // NaN never wins
        mV = fmax(mV, kv);
    }
    for (int off = 16; off > 0; off >>= 1) {
        mU = fmax(mU, __shfl_xor_sync(0xffffffffu, mU, off));
        mV = fmax(mV, __shfl_xor_sync(0xffffffffu, mV, off));
    }
    __shared__ F sh[2][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = mU;
        sh[1][wid] = mV;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            mU = fmax(mU, sh[0][k]);
            mV = fmax(mV, sh[1][k]);
        }
        atomicMax(&kmax[0], Bits<F>::of(mU));
        atomicMax(&kmax[1], Bits<F>::of(mV));
    }
}

template <typename F>
__global__ void adapt_finish_kernel(typename Bits<F>::U* kmax, double kW, double cfl, long long steps_prev,
                                    double* dt64, float* dt32, double* t_done)
{
    F kU, kV;
    if constexpr (sizeof(F) == 4) {
        kU = __uint_as_float(kmax[0]);
        kV = __uint_as_float(kmax[1]);
    } else {
        kU = __longlong_as_double((long long)kmax[0]);
        kV = __longlong_as_double((long long)kmax[1]);
    }
    *t_done += *dt64 * (double)steps_prev;
    const double k = fmax(kW, fmax((double)kU, (double)kV));
    const double dt = cfl / k;
    *dt64 = dt;
    *dt32 = (float)dt;
    kmax[0] = 0;
    kmax[1] = 0;
}

}  // namespace

template <typename F>
cudaError_t launch_adapt(const F* u, const F* v, const F* w, int nx, int ny, int pitch, const AdaptRule<F>& r,
                         double kW, double cfl, long long steps_prev, AdaptState& st, cudaStream_t s)
{
    using U = typename Bits<F>::U;
    U* kmax = reinterpret_cast<U*>(st.kmax);
    const size_t n = (size_t)nx * ny;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    adapt_reduce_kernel<F><<<blocks, 256, 0, s>>>(u, v, w, nx, ny, pitch, r, kmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adapt_finish_kernel<F><<<1, 1, 0, s>>>(kmax, kW, cfl, steps_prev, st.dt64, st.dt32, st.t_done);
    return cudaGetLastError();
}

template cudaError_t launch_adapt<float>(const float*, const float*, const float*, int, int, int,
                                         const AdaptRule<float>&, double, double, long long, AdaptState&,
                                         cudaStream_t);
template cudaError_t launch_adapt<double>(const double*, const double*, const double*, int, int, int,
                                          const AdaptRule<double>&, double, double, long long, AdaptState&,
                                          cudaStream_t);

}  // namespace gg
