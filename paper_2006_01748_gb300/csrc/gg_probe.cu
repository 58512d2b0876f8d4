// Arithmetic-rate probes: the measured denominators of the ALU rooflines.
//
// The forward and adjoint kernels are bound by FP32 instruction issue and the
// plain step by FP64 arithmetic, so their roofline fractions need the rate at
// which this GPU retires those operations.  Each probe launches a grid of
// whole waves (a multiple of the SM count) whose threads run CHAINS
// independent fused multiply-add chains for `iters` iterations, and times
// the launch with CUDA events: rate = 2 flops x CHAINS x iters x threads /
// time.  The chains are independent so that FMA latency is hidden, the
// multiplier and addend are kernel arguments so that nothing folds at compile
// time, and the result is stored under a condition the compiler cannot
// decide, so that nothing is eliminated.
#include <math.h>

#include "gg_internal.cuh"

namespace {

constexpr int kChains = 8;

static __device__ double g_probe_sink[4];

template <typename F>
__global__ void __launch_bounds__(256) fma_chain_kernel(long long iters, F a, F b, F guard)
{
    F x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (F)(threadIdx.x + c);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    F s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == guard) g_probe_sink[0] = (double)s;
}

// Packed FP32 pairs: one instruction carries two FMAs.
__global__ void __launch_bounds__(256) fma2_chain_kernel(long long iters, float a, float b, float guard)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == guard) g_probe_sink[1] = (double)s;
}

}  // namespace

extern "C" int gg_probe_fma_rate(int32_t kind, int64_t iters, int32_t waves, void* cuda_stream, double* flops_per_s)
{
    if (!flops_per_s || kind < 0 || kind > 2 || iters < 1 || iters > (1LL << 32) || waves < 1 || waves > 64)
        return GG_ERR_ARG;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if (kind == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<double>, 256, 0);
        else if (kind == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<float>, 256, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma2_chain_kernel, 256, 0);
    }
    if (e != cudaSuccess || sms < 1 || per_sm < 1) return GG_ERR_CUDA;
    const int blocks = sms * per_sm * waves;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return GG_ERR_CUDA;
    }
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // rep 0 warms up
        e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) break;
        if (kind == 0) fma_chain_kernel<double><<<blocks, 256, 0, s>>>(iters, 1.0000001, 1e-9, -1.0);
        else if (kind == 1) fma_chain_kernel<float><<<blocks, 256, 0, s>>>(iters, 1.0000001f, 1e-9f, -1.0f);
        else fma2_chain_kernel<<<blocks, 256, 0, s>>>(iters, 1.0000001f, 1e-9f, -1.0f);
        e = cudaPeekAtLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(ms > 0.0f)) return GG_ERR_CUDA;
    const double fmas = (double)blocks * 256.0 * (double)kChains * (double)iters * (kind == 2 ? 2.0 : 1.0);
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    return GG_OK;
}
