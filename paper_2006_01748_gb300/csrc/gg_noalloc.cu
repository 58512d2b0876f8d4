// gg_diagnostics_noalloc: the FP64 diagnostics reduction for callers that
// cannot allocate device memory.
//
// gg_diagnostics needs a gg_sim, whose device memory (including the
// per-block partial sums of the reduction) comes from cudaMalloc at
// gg_create.  Some callers cannot make that call: code that runs while a
// stream is being captured into a CUDA graph, code embedded in a framework
// whose memory pool owns the whole device and forbids untracked
// allocations, or a time-critical loop that cannot afford the implicit
// synchronisation of cudaMalloc/cudaFree.  This variant takes the fields as
// device pointers and keeps its scratch in the file-scope array below, so
// it allocates nothing.
#include <math.h>

#include <mutex>

#include "gg_internal.cuh"

namespace {

// Scratch: kSlots partial records of kRec doubles (one record per block of
// the first pass) plus one record for the final result: 609 x 128 bytes
// = 77,952 bytes, held by every device that loads the library until exit.
constexpr int kSlots = 608;
constexpr int kRec = 16;
constexpr long long kMaxCells = 1LL << 31;  // largest grid accepted (nx * ny)

static __device__ __align__(256) double g_diag_scratch[(kSlots + 1) * kRec];

struct Acc {
    double sum[3], mn[3], mx[3];
    double nonfinite, tumour, gap;
};

__device__ __forceinline__ void acc_init(Acc& a)
{
    for (int f = 0; f < 3; ++f) {
        a.sum[f] = 0.0;
        a.mn[f] = INFINITY;
        a.mx[f] = -INFINITY;
    }
    a.nonfinite = a.tumour = a.gap = 0.0;
}

__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b)
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

__device__ Acc acc_block_reduce(Acc a)
{
    __shared__ Acc sh[32];
    for (int off = 16; off > 0; off >>= 1) {
        Acc b;
        for (int f = 0; f < 3; ++f) {
            b.sum[f] = __shfl_xor_sync(0xffffffffu, a.sum[f], off);
            b.mn[f] = __shfl_xor_sync(0xffffffffu, a.mn[f], off);
            b.mx[f] = __shfl_xor_sync(0xffffffffu, a.mx[f], off);
        }
        b.nonfinite = __shfl_xor_sync(0xffffffffu, a.nonfinite, off);
        b.tumour = __shfl_xor_sync(0xffffffffu, a.tumour, off);
        b.gap = __shfl_xor_sync(0xffffffffu, a.gap, off);
        acc_merge(a, b);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) acc_merge(a, sh[w]);
    return a;
}

__device__ __forceinline__ void acc_store(double* p, const Acc& a)
{
    for (int f = 0; f < 3; ++f) {
        p[f] = a.sum[f];
        p[3 + f] = a.mn[f];
        p[6 + f] = a.mx[f];
    }
    p[9] = a.nonfinite;
    p[10] = a.tumour;
    p[11] = a.gap;
}

// First pass: block b reduces rows b, b + gridDim.x, ... into record b of
// the scratch.  Every record that the second pass reads is written here,
// so nothing left by an earlier call is ever read.
template <typename F>
__global__ void __launch_bounds__(256) noalloc_partial_kernel(const F* __restrict__ u, const F* __restrict__ v,
                                                              const F* __restrict__ w, int nx, int ny, int pitch,
                                                              double eps, double* scratch)
{
    Acc a;
    acc_init(a);
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
    a = acc_block_reduce(a);
    if (threadIdx.x == 0) acc_store(scratch + (size_t)blockIdx.x * kRec, a);
}

// Second pass: one block folds records [0, nparts) in a fixed order into
// the result record kSlots.
__global__ void __launch_bounds__(256) noalloc_final_kernel(double* scratch, int nparts)
{
    Acc a;
    acc_init(a);
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const double* p = scratch + (size_t)b * kRec;
        Acc c;
        for (int f = 0; f < 3; ++f) {
            c.sum[f] = p[f];
            c.mn[f] = p[3 + f];
            c.mx[f] = p[6 + f];
        }
        c.nonfinite = p[9];
        c.tumour = p[10];
        c.gap = p[11];
        acc_merge(a, c);
    }
    a = acc_block_reduce(a);
    if (threadIdx.x == 0) acc_store(scratch + (size_t)kSlots * kRec, a);
}

// Device address of g_diag_scratch on the current device.  In host code the
// name g_diag_scratch is only a host-side stand-in, so the address is looked
// up once per device with cudaGetSymbolAddress and cached.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

int scratch_address(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return GG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_diag_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GG_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GG_OK;
}

}  // namespace

extern "C" int gg_diagnostics_noalloc(const void* u, const void* v, const void* w, int32_t fp64, int32_t nx,
                                      int32_t ny, int32_t pitch, double dx, double dy, double eps,
                                      void* cuda_stream, gg_diag* out)
{
    if (!u || !v || !w || !out) return GG_ERR_ARG;
    if (nx < 1 || ny < 1 || pitch < nx) return GG_ERR_ARG;
    if ((long long)nx * (long long)ny > kMaxCells) return GG_ERR_ARG;
    if (!(isfinite(dx) && dx > 0.0) || !(isfinite(dy) && dy > 0.0) || !(isfinite(eps) && eps > 0.0))
        return GG_ERR_ARG;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != GG_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = ny < kSlots ? ny : kSlots;
    if (fp64)
        noalloc_partial_kernel<double><<<blocks, 256, 0, s>>>((const double*)u, (const double*)v, (const double*)w,
                                                              nx, ny, pitch, eps, scratch);
    else
        noalloc_partial_kernel<float><<<blocks, 256, 0, s>>>((const float*)u, (const float*)v, (const float*)w, nx,
                                                             ny, pitch, eps, scratch);
    noalloc_final_kernel<<<1, 256, 0, s>>>(scratch, blocks);
    double h[kRec];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, scratch + (size_t)kSlots * kRec, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return GG_ERR_CUDA;
    const double cell = dx * dy;
    for (int k = 0; k < 3; ++k) {
        out->mass[k] = h[k] * cell;
        out->min[k] = h[3 + k];
        out->max[k] = h[6 + k];
    }
    out->nonfinite = (int64_t)h[9];
    out->tumour_area = h[10] * cell;
    out->gap_area = h[11] * cell;
    out->gap_eps = eps;
    return out->nonfinite ? GG_ERR_NONFINITE : GG_OK;
}
