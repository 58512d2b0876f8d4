// Supporting kernels of libgg.so: the plain FP64 step, the tensor build of
// eq. (2), layout conversion between the dense host layout and the pitched
// device layout, and the FP64 diagnostics reduction.
#include <math.h>

#include <algorithm>

#include "gg_internal.cuh"

namespace gg {
namespace {

// ---------------------------------------------------------------- FP64 plain step
//
// One thread per cell, every operand read from global memory: the plain
// design (the CUDA kernel of Section 3 updates each cell from the previous
// iterate in global memory), kept as the double-precision comparison point.
__global__ void __launch_bounds__(256) step64_kernel(const Grid64 g, const Rates64 k0)
{
    const Rates64 k = live_rates(k0);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    if (i >= nx || j >= ny) return;
    const bool hasW = i > 0, hasE = i + 1 < nx, hasS = j > 0, hasN = j + 1 < ny;
    const int iw = hasW ? i - 1 : i, ie = hasE ? i + 1 : i;
    const int js = hasS ? j - 1 : j, jn = hasN ? j + 1 : j;
#define AT(f, x, y) __ldg((f) + (size_t)(y) * pitch + (x))
    const double up = AT(g.u, i, j), vp = AT(g.v, i, j), wp = AT(g.w, i, j);
    // Table 1
    const double hE = (1.0 - 0.5 * (up + AT(g.u, ie, j))) * (AT(g.v, ie, j) - vp);
    const double hW = (1.0 - 0.5 * (up + AT(g.u, iw, j))) * (AT(g.v, iw, j) - vp);
    const double hN = (1.0 - 0.5 * (up + AT(g.u, i, jn))) * (AT(g.v, i, jn) - vp);
    const double hS = (1.0 - 0.5 * (up + AT(g.u, i, js))) * (AT(g.v, i, js) - vp);
    const double d1 = (hE + hW) * k.ihx2 + (hN + hS) * k.ihy2;
    // Table 2 in flux form
    const double wE = AT(g.w, ie, j), wW = AT(g.w, iw, j), wN = AT(g.w, i, jn), wS = AT(g.w, i, js);
    const double a11P = AT(g.a11, i, j), a22P = AT(g.a22, i, j), bP = AT(g.a12, i, j);
    const double nE = (a11P + AT(g.a11, ie, j)) * (wE - wp);
    const double nW = (AT(g.a11, iw, j) + a11P) * (wp - wW);
    const double nN = (a22P + AT(g.a22, i, jn)) * (wN - wp);
    const double nS = (AT(g.a22, i, js) + a22P) * (wp - wS);
    const double tyP = wN - wS;
    const double tyE = AT(g.w, ie, jn) - AT(g.w, ie, js);
    const double tyW = AT(g.w, iw, jn) - AT(g.w, iw, js);
    const double txP = wE - wW;
    const double txN = AT(g.w, ie, jn) - AT(g.w, iw, jn);
    const double txS = AT(g.w, ie, js) - AT(g.w, iw, js);
    const double cE = hasE ? bP * tyP + AT(g.a12, ie, j) * tyE : 0.0;
    const double cW = hasW ? AT(g.a12, iw, j) * tyW + bP * tyP : 0.0;
    const double cN = hasN ? bP * txP + AT(g.a12, i, jn) * txN : 0.0;
    const double cS = hasS ? AT(g.a12, i, js) * txS + bP * txP : 0.0;
#undef AT
    const double d2 = ((nE - nW) * k.kx + (nN - nS) * k.ky) + ((cE - cW) + (cN - cS)) * k.kc;
    double fu, fv, fw;
    if (k.no_reaction) {
        fu = 0.0;
        fv = k.D * d1;
        fw = d2;
    } else {
        fu = up * (1.0 - up) - k.delta * up * wp;
        fv = k.rho * vp * (1.0 - vp) + k.D * d1;
        fw = k.c * (vp - wp) + d2;
    }
    const size_t o = (size_t)j * pitch + i;
    g.uo[o] = up + k.dt * fu;
    g.vo[o] = vp + k.dt * fv;
    g.wo[o] = wp + k.dt * fw;
}

// ---------------------------------------------------------------- eq. (2)

// A = R(theta) diag(L1, L2) R(theta)^T at one cell.
__device__ __forceinline__ void tensor_at(double th, double L1, double L2, double& A11, double& A12, double& A22)
{
    double s, c;
    sincos(th, &s, &c);
    A11 = L1 * c * c + L2 * s * s;
    A12 = (L1 - L2) * s * c;
    A22 = L1 * s * s + L2 * c * c;
}

// FP64 kernels get a11, a12, a22 per cell.  FP32 kernels get the face
// weights ax = (a11 + a11_east) kx, ay = (a22 + a22_north) ky (0 on the last
// column / row, whose east / north face is a boundary face) and b = a12 kc,
// computed in FP64 and rounded once: this kernel writes b and the cell's a11
// and a22 (dense FP64, t11 / t22), faces_kernel the two face weights.
template <bool FACES, typename F>
__global__ void coefficients_kernel(const double* __restrict__ theta, const double* __restrict__ l1,
                                    const double* __restrict__ l2, int nx, int ny, double kc, F* c0, F* c1,
                                    F* c2, double* t11, double* t22, int pitch, unsigned long long* counters,
                                    unsigned long long* lmax_bits)
{
    __shared__ double smax[32];
    __shared__ unsigned long long sbad[32];
    const size_t n = (size_t)nx * ny;
    double lmax = 0.0;
    unsigned long long bad = 0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const double th = theta[q], L1 = l1[q], L2 = l2[q];
        if (!(isfinite(th) && isfinite(L1) && isfinite(L2)) || !(L1 > 0.0) || !(L2 > 0.0)) ++bad;
        double A11, A12, A22;
        tensor_at(th, L1, L2, A11, A12, A22);
        const size_t o = (size_t)j * pitch + i;
        if constexpr (FACES) {
            t11[q] = A11;
            t22[q] = A22;
            c1[o] = (F)(A12 * kc);
        } else {
            c0[o] = (F)A11;
            c1[o] = (F)A12;
            c2[o] = (F)A22;
        }
        const double h = 0.5 * (A11 - A22);
        const double e = 0.5 * (A11 + A22) + sqrt(h * h + A12 * A12);
        if (e > lmax) lmax = e;  // NaN never wins
    }
    for (int off = 16; off > 0; off >>= 1) {
        lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
        bad += __shfl_xor_sync(0xffffffffu, bad, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        smax[wid] = lmax;
        sbad[wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        unsigned long long b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            m = fmax(m, smax[w]);
            b += sbad[w];
        }
        if (b) atomicAdd(&counters[0], b);
        atomicMax(lmax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// ax and ay of the FP32 kernels from the dense a11 / a22 of coefficients_kernel.
template <typename F>
__global__ void faces_kernel(const double* __restrict__ t11, const double* __restrict__ t22, int nx, int ny,
                             double kx, double ky, F* c0, F* c2, int pitch)
{
    const size_t n = (size_t)nx * ny;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const size_t o = (size_t)j * pitch + i;
        c0[o] = (F)(i + 1 < nx ? (t11[q] + t11[q + 1]) * kx : 0.0);
        c2[o] = (F)(j + 1 < ny ? (t22[q] + t22[q + nx]) * ky : 0.0);
    }
}

// ---------------------------------------------------------------- layout conversion

template <typename S, typename D>
__global__ void unpack_kernel(const S* __restrict__ src, D* dst, int nx, int ny, int pitch,
                              unsigned long long* nonfinite)
{
    const size_t n = (size_t)nx * ny;
    unsigned long long bad = 0;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const S v = src[q];
        if (!isfinite((double)v)) ++bad;
        dst[(size_t)j * pitch + i] = (D)v;
    }
    if (nonfinite) {
        for (int off = 16; off > 0; off >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, off);
        if ((threadIdx.x & 31) == 0 && bad) atomicAdd(nonfinite, bad);
    }
}

template <typename S, typename D>
__global__ void pack_kernel(const S* __restrict__ src, D* dst, int nx, int ny, int pitch)
{
    const size_t n = (size_t)nx * ny;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        dst[q] = (D)src[(size_t)j * pitch + i];
    }
}

int blocks_for(size_t n, int threads) { return (int)std::min<size_t>((n + threads - 1) / threads, 152 * 16); }

// ---------------------------------------------------------------- diagnostics

struct DiagAcc {
    double sum[3], mn[3], mx[3];
    double nonfinite, tumour, gap;
};

__device__ __forceinline__ void diag_merge(DiagAcc& a, const DiagAcc& b)
{
    for (int f = 0; f < 3; ++f) {
        a.sum[f] += b.sum[f];
        a.mn[f] = fmin(a.mn[f], b.mn[f]);
        a.mx[f] = fmax(a.mx[f], b.mx[f]);
    }
    a.nonfinite += b.nonfinite;
    a.tumour += b.tumour;
    a.gap += b.gap;
}

__device__ __forceinline__ DiagAcc diag_shfl(const DiagAcc& a, int off)
{
    DiagAcc b;
    for (int f = 0; f < 3; ++f) {
        b.sum[f] = __shfl_xor_sync(0xffffffffu, a.sum[f], off);
        b.mn[f] = __shfl_xor_sync(0xffffffffu, a.mn[f], off);
        b.mx[f] = __shfl_xor_sync(0xffffffffu, a.mx[f], off);
    }
    b.nonfinite = __shfl_xor_sync(0xffffffffu, a.nonfinite, off);
    b.tumour = __shfl_xor_sync(0xffffffffu, a.tumour, off);
    b.gap = __shfl_xor_sync(0xffffffffu, a.gap, off);
    return b;
}

// Warp-shuffle then shared-memory block reduction; the result is valid in
// thread 0.  The combination order is fixed, so the result is deterministic.
__device__ DiagAcc diag_block_reduce(DiagAcc a)
{
    __shared__ DiagAcc sh[32];
    for (int off = 16; off > 0; off >>= 1) diag_merge(a, diag_shfl(a, off));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) diag_merge(a, sh[w]);
    }
    return a;
}

__device__ __forceinline__ void diag_init(DiagAcc& a)
{
    for (int f = 0; f < 3; ++f) {
        a.sum[f] = 0.0;
        a.mn[f] = INFINITY;
        a.mx[f] = -INFINITY;
    }
    a.nonfinite = a.tumour = a.gap = 0.0;
}

template <typename F>
__global__ void __launch_bounds__(256) diag_partial_kernel(const F* __restrict__ u, const F* __restrict__ v,
                                                           const F* __restrict__ w, int nx, int ny, int pitch,
                                                           double eps, double* partials)
{
    DiagAcc a;
    diag_init(a);
    // Rows are distributed over blocks, columns over threads (coalesced).
    for (int j = blockIdx.x; j < ny; j += gridDim.x) {
        const size_t row = (size_t)j * pitch;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const double x[3] = {(double)u[row + i], (double)v[row + i], (double)w[row + i]};
            for (int f = 0; f < 3; ++f) {
                if (isfinite(x[f])) {
                    a.sum[f] += x[f];
                    a.mn[f] = fmin(a.mn[f], x[f]);
                    a.mx[f] = fmax(a.mx[f], x[f]);
                } else {
                    a.nonfinite += 1.0;
                }
            }
            if (x[1] > 0.5) a.tumour += 1.0;
            if (x[0] < eps && x[1] < eps) a.gap += 1.0;
        }
    }
    a = diag_block_reduce(a);
    if (threadIdx.x == 0) {
        double* p = partials + (size_t)blockIdx.x * kDiagStride;
        for (int f = 0; f < 3; ++f) {
            p[f] = a.sum[f];
            p[3 + f] = a.mn[f];
            p[6 + f] = a.mx[f];
        }
        p[9] = a.nonfinite;
        p[10] = a.tumour;
        p[11] = a.gap;
    }
}

__global__ void __launch_bounds__(256) diag_final_kernel(const double* __restrict__ partials, int nparts,
                                                         double* out)
{
    DiagAcc a;
    diag_init(a);
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const double* p = partials + (size_t)b * kDiagStride;
        DiagAcc c;
        for (int f = 0; f < 3; ++f) {
            c.sum[f] = p[f];
            c.mn[f] = p[3 + f];
            c.mx[f] = p[6 + f];
        }
        c.nonfinite = p[9];
        c.tumour = p[10];
        c.gap = p[11];
        diag_merge(a, c);
    }
    a = diag_block_reduce(a);
    if (threadIdx.x == 0) {
        for (int f = 0; f < 3; ++f) {
            out[f] = a.sum[f];
            out[3 + f] = a.mn[f];
            out[6 + f] = a.mx[f];
        }
        out[9] = a.nonfinite;
        out[10] = a.tumour;
        out[11] = a.gap;
    }
}

}  // namespace

cudaError_t launch_step64(const Grid64& g, const Rates64& r, cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8);
    step64_kernel<<<grid, block, 0, s>>>(g, r);
    return cudaGetLastError();
}

cudaError_t launch_coefficients(const double* theta, const double* l1, const double* l2, int nx, int ny, double dx,
                                double dy, void* c0, void* c1, void* c2, int pitch, bool fp64, double* scratch,
                                unsigned long long* counters, unsigned long long* lmax_bits, cudaStream_t s)
{
    const size_t n = (size_t)nx * ny;
    const int blocks = blocks_for(n, 256);
    if (fp64) {
        coefficients_kernel<false, double><<<blocks, 256, 0, s>>>(theta, l1, l2, nx, ny, 0.0, (double*)c0,
                                                                  (double*)c1, (double*)c2, nullptr, nullptr, pitch,
                                                                  counters, lmax_bits);
        return cudaGetLastError();
    }
    if (!scratch) return cudaErrorInvalidValue;
    double* t11 = scratch;
    double* t22 = scratch + n;
    coefficients_kernel<true, float><<<blocks, 256, 0, s>>>(theta, l1, l2, nx, ny, 0.25 / (dx * dy), (float*)c0,
                                                            (float*)c1, (float*)c2, t11, t22, pitch, counters,
                                                            lmax_bits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    faces_kernel<float><<<blocks, 256, 0, s>>>(t11, t22, nx, ny, 0.5 / (dx * dx), 0.5 / (dy * dy), (float*)c0,
                                               (float*)c2, pitch);
    return cudaGetLastError();
}

template <typename F>
__global__ void tensor_entry_kernel(const double* __restrict__ theta, const double* __restrict__ l1,
                                    const double* __restrict__ l2, size_t n, int which, F* dst)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        double A[3];
        tensor_at(theta[q], l1[q], l2[q], A[0], A[1], A[2]);
        dst[q] = (F)A[which];
    }
}

cudaError_t launch_tensor_entry(const double* theta, const double* l1, const double* l2, size_t n, int which,
                                void* dst, bool dst_fp64, cudaStream_t s)
{
    if (which < 0 || which > 2) return cudaErrorInvalidValue;
    const int blocks = blocks_for(n, 256);
    if (dst_fp64) tensor_entry_kernel<double><<<blocks, 256, 0, s>>>(theta, l1, l2, n, which, (double*)dst);
    else tensor_entry_kernel<float><<<blocks, 256, 0, s>>>(theta, l1, l2, n, which, (float*)dst);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void* src, bool src_fp64, void* dst, bool dst_fp64, int nx, int ny, int pitch,
                          unsigned long long* nonfinite, cudaStream_t s)
{
    const size_t n = (size_t)nx * ny;
    const int blocks = blocks_for(n, 256);
    if (src_fp64 && dst_fp64)
        unpack_kernel<double, double><<<blocks, 256, 0, s>>>((const double*)src, (double*)dst, nx, ny, pitch, nonfinite);
    else if (src_fp64)
        unpack_kernel<double, float><<<blocks, 256, 0, s>>>((const double*)src, (float*)dst, nx, ny, pitch, nonfinite);
    else if (dst_fp64)
        unpack_kernel<float, double><<<blocks, 256, 0, s>>>((const float*)src, (double*)dst, nx, ny, pitch, nonfinite);
    else
        unpack_kernel<float, float><<<blocks, 256, 0, s>>>((const float*)src, (float*)dst, nx, ny, pitch, nonfinite);
    return cudaGetLastError();
}

cudaError_t launch_pack(const void* src, bool src_fp64, void* dst, bool dst_fp64, int nx, int ny, int pitch,
                        cudaStream_t s)
{
    const size_t n = (size_t)nx * ny;
    const int blocks = blocks_for(n, 256);
    if (src_fp64 && dst_fp64)
        pack_kernel<double, double><<<blocks, 256, 0, s>>>((const double*)src, (double*)dst, nx, ny, pitch);
    else if (src_fp64)
        pack_kernel<double, float><<<blocks, 256, 0, s>>>((const double*)src, (float*)dst, nx, ny, pitch);
    else if (dst_fp64)
        pack_kernel<float, double><<<blocks, 256, 0, s>>>((const float*)src, (double*)dst, nx, ny, pitch);
    else
        pack_kernel<float, float><<<blocks, 256, 0, s>>>((const float*)src, (float*)dst, nx, ny, pitch);
    return cudaGetLastError();
}

// Each launch's own status is checked (cudaLaunchKernel returns it), so an
// error left pending on the calling thread by some earlier call is neither
// reported as this reduction's failure nor cleared.
cudaError_t launch_diagnostics(const void* u, const void* v, const void* w, bool fp64, int nx, int ny, int pitch,
                               double eps, double* partials, double* out, cudaStream_t s)
{
    int blocks = std::min(ny, kDiagBlocks);
    void* pargs[] = {(void*)&u, (void*)&v, (void*)&w, (void*)&nx, (void*)&ny, (void*)&pitch, (void*)&eps,
                     (void*)&partials};
    const void* partial = fp64 ? (const void*)diag_partial_kernel<double> : (const void*)diag_partial_kernel<float>;
    cudaError_t e = cudaLaunchKernel(partial, dim3(blocks), dim3(256), pargs, 0, s);
    if (e != cudaSuccess) return e;
    void* fargs[] = {(void*)&partials, (void*)&blocks, (void*)&out};
    return cudaLaunchKernel((const void*)diag_final_kernel, dim3(1), dim3(256), fargs, 0, s);
}

}  // namespace gg
