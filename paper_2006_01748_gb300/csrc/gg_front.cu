// Fronts and the interstitial gap of Section 2, measured along the four axis
// rays from one cell, and the space-averaged front speed (the LeVeque-Yee
// formula: rate of change of the ray integral of V over the jump of V across
// the front).  One CTA per ray; every reduction runs in a fixed order, so
// the result does not depend on timing.
#include <math.h>

#include "gg_sim.cuh"

using namespace gg;

namespace {

constexpr int kFrontThreads = 256;

// Block reductions in a fixed order (warp shuffle tree, then warp 0 over the
// per-warp results).
template <typename X, typename Op>
__device__ X block_reduce(X x, X identity, Op op, X* sh)
{
    for (int off = 16; off > 0; off >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, off));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();  // sh may still be read by a previous reduction
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    x = (threadIdx.x < (kFrontThreads >> 5)) ? sh[threadIdx.x] : identity;
    if (wid == 0)
        for (int off = 16; off > 0; off >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, off));
    if (threadIdx.x == 0) sh[0] = x;
    __syncthreads();
    return sh[0];
}

// out[d], [4 + d], [8 + d], [12 + d], [16 + d]: front, healthy edge, gap,
// ray integrals of V and U of ray d = blockIdx.x (east, west, north, south).
template <typename F>
__global__ void __launch_bounds__(kFrontThreads) front_rays_kernel(const F* __restrict__ U, const F* __restrict__ V,
                                                                   int nx, int ny, int pitch, int i0, int j0, double dx,
                                                                   double dy, double v_front, double u_edge,
                                                                   double eps, double* out)
{
    __shared__ double shd[32];
    __shared__ int shi[32];
    const int d = blockIdx.x;
    const int L = d == 0 ? nx - i0 : d == 1 ? i0 + 1 : d == 2 ? ny - j0 : j0 + 1;
    const int di = d == 0 ? 1 : d == 1 ? -1 : 0;
    const int dj = d == 2 ? 1 : d == 3 ? -1 : 0;
    const double h = d < 2 ? dx : dy;
    auto at = [&](int k) { return (size_t)(j0 + dj * k) * pitch + (i0 + di * k); };

    // farthest tumour cell and the two integrals (each thread walks its
    // cells in increasing k)
    int kT = -1;
    double sv = 0.0, su = 0.0;
    for (int k = threadIdx.x; k < L; k += kFrontThreads) {
        const double v = (double)V[at(k)], u = (double)U[at(k)];
        if (v > v_front) kT = k;
        sv += v;
        su += u;
    }
    auto imax = [](int a, int b) { return a > b ? a : b; };
    auto imin = [](int a, int b) { return a < b ? a : b; };
    auto iadd = [](int a, int b) { return a + b; };
    auto dadd = [](double a, double b) { return a + b; };
    kT = block_reduce(kT, -1, imax, shi);
    sv = block_reduce(sv, 0.0, dadd, shd);
    su = block_reduce(su, 0.0, dadd, shd);
    // first healthy cell beyond the front
    int kH = L;
    for (int k = kT + 1 + (int)threadIdx.x; k < L; k += kFrontThreads)
        if ((double)U[at(k)] > u_edge) { kH = k; break; }
    kH = block_reduce(kH, L, imin, shi);
    // gap cells between them
    int gap = 0;
    for (int k = kT + 1 + (int)threadIdx.x; k < kH; k += kFrontThreads) {
        const double u = (double)U[at(k)], v = (double)V[at(k)];
        if (u < eps && v < eps) ++gap;
    }
    gap = block_reduce(gap, 0, iadd, shi);
    if (threadIdx.x == 0) {
        out[d] = kT >= 0 ? (kT + 0.5) * h : 0.0;
        out[4 + d] = (kH - 0.5) * h;
        out[8 + d] = gap * h;
        out[12 + d] = sv * h;
        out[16 + d] = su * h;
    }
}

int front_args(const gg_sim* s, int32_t i0, int32_t j0, double v_front, double u_edge, double eps)
{
    if (i0 < 0 || i0 >= s->nx || j0 < 0 || j0 >= s->ny) return GG_ERR_ARG;
    if (!isfinite(v_front) || !isfinite(u_edge) || !(eps > 0.0) || !isfinite(eps)) return GG_ERR_ARG;
    return GG_OK;
}

int measure(gg_sim* s, int32_t i0, int32_t j0, double v_front, double u_edge, double eps, gg_front* out)
{
    const bool fp64 = s->params.precision == GG_FP64_PLAIN;
    double* dev = s->diag_partials;  // 20 doubles of the diagnostics scratch (same stream)
    if (fp64)
        front_rays_kernel<double><<<4, kFrontThreads, 0, s->stream>>>(s->f64[s->cur][0], s->f64[s->cur][1], s->nx,
                                                                      s->ny, s->pitch, i0, j0, s->dx, s->dy, v_front,
                                                                      u_edge, eps, dev);
    else
        front_rays_kernel<float><<<4, kFrontThreads, 0, s->stream>>>(s->f32[s->cur][0], s->f32[s->cur][1], s->nx,
                                                                     s->ny, s->pitch, i0, j0, s->dx, s->dy, v_front,
                                                                     u_edge, eps, dev);
    double host[20];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof host, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "front_rays");
    for (int d = 0; d < 4; ++d) {
        out->front[d] = host[d];
        out->edge[d] = host[4 + d];
        out->gap[d] = host[8 + d];
        out->mass_v[d] = host[12 + d];
        out->mass_u[d] = host[16 + d];
    }
    return GG_OK;
}

}  // namespace

extern "C" int gg_front_rays(gg_sim* s, int32_t i0, int32_t j0, double v_front, double u_edge, double eps,
                             gg_front* out)
{
    if (!s) return GG_ERR_ARG;
    if (!out) { s->last_error = "out is NULL"; return GG_ERR_ARG; }
    if (front_args(s, i0, j0, v_front, u_edge, eps) != GG_OK) {
        s->last_error = "front rays: centre cell outside the grid, non-finite threshold or eps <= 0";
        return GG_ERR_ARG;
    }
    return measure(s, i0, j0, v_front, u_edge, eps, out);
}

extern "C" int gg_front_speed(gg_sim* s, int32_t i0, int32_t j0, int64_t nsteps, double v_front, double u_edge,
                              double eps, gg_front* before, gg_front* after, double* speed)
{
    if (!s) return GG_ERR_ARG;
    if (!before || !after || !speed) { s->last_error = "before, after and speed must not be NULL"; return GG_ERR_ARG; }
    if (nsteps < 1) { s->last_error = "nsteps must be >= 1"; return GG_ERR_ARG; }
    if (front_args(s, i0, j0, v_front, u_edge, eps) != GG_OK) {
        s->last_error = "front speed: centre cell outside the grid, non-finite threshold or eps <= 0";
        return GG_ERR_ARG;
    }
    int rc = measure(s, i0, j0, v_front, u_edge, eps, before);
    if (rc == GG_OK) rc = gg_step(s, nsteps);
    if (rc == GG_OK) rc = measure(s, i0, j0, v_front, u_edge, eps, after);
    if (rc != GG_OK) return rc;
    const double elapsed = (double)nsteps * s->dt;
    for (int d = 0; d < 4; ++d) speed[d] = (after->mass_v[d] - before->mass_v[d]) / (elapsed * (1.0 - 0.0));
    return GG_OK;
}
