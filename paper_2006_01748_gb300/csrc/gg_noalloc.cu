// gg_diagnostics_noalloc: the FP64 diagnostics reduction for callers that
// cannot allocate device memory.
//
// gg_diagnostics needs a gg_sim, whose device memory (including the
// per-block partial sums of the reduction) comes from cudaMalloc at
// gg_create.  Some callers cannot make that call: code embedded in a
// framework whose memory pool owns the whole device and forbids untracked
// allocations, or a time-critical loop that cannot afford the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.  This variant takes
// the fields as device pointers and keeps the reduction's scratch in the
// file-scope array below, so it allocates nothing.  It runs the same two
// kernels as gg_diagnostics (launch_diagnostics), only with this array as
// their partial-sum and result buffers.
#include <math.h>

#include <mutex>

#include "gg_internal.cuh"

namespace {

// Scratch: the kDiagBlocks partial records of kDiagStride doubles that the
// first kernel writes (one per block), then the 16-double result record of
// the second: 608 x 128 + 128 = 77,952 bytes, held by every device that
// loads the library until exit.
constexpr int kPartials = gg::kDiagBlocks * gg::kDiagStride;
constexpr int kResult = 16;
constexpr long long kMaxCells = 1LL << 31;  // largest grid accepted (nx * ny)

static __device__ __align__(256) double g_diag_scratch[kPartials + kResult];

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
    double* result = scratch + kPartials;
    // The first kernel writes every partial record the second one reads, so
    // nothing an earlier call left in the array is read.
    cudaError_t e = gg::launch_diagnostics(u, v, w, fp64 != 0, nx, ny, pitch, eps, scratch, result, s);
    double h[12];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, result, sizeof h, cudaMemcpyDeviceToHost, s);
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
