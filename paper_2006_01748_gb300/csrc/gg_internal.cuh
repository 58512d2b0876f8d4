// Internal declarations shared by the translation units of libgg.so.
// Nothing here is part of the public ABI (include/gg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gg.h"

namespace gg {

constexpr int kMaxT = 8;           // deepest temporal blocking supported
constexpr int kDiagBlocks = 608;   // 4 x 152 SMs: diagnostics partial sums
constexpr int kDiagStride = 16;    // doubles per diagnostics partial

// Device-side description of one FP32 state on a pitched grid.  Row j of a
// field starts at base + j * pitch; pitch is a multiple of 32 floats.
// The tensor of eq. (2) enters the FP32 kernels through three coefficient
// fields, built once per tissue in FP64 and rounded once:
//   ax(i,j) = (a11(i,j) + a11(i+1,j)) / (2 dx^2)   east face, 0 on the last column
//   ay(i,j) = (a22(i,j) + a22(i,j+1)) / (2 dy^2)   north face, 0 on the last row
//   b(i,j)  = a12(i,j) / (4 dx dy)                 cell
// (the face weights and the cross-term weight of Table 2).
struct Grid32 {
    const float* u; const float* v; const float* w;
    const float* cu; const float* cv; const float* cw;   // null without Kahan
    float* uo; float* vo; float* wo;
    float* cuo; float* cvo; float* cwo;
    const float* ax; const float* b; const float* ay;
    int nx, ny, pitch;
};

// Scalars of eq. (3) in FP32, rounded once from the FP64 host values.  With
// the adaptive step, dt_dev points at the device copy of the current
// Delta t_k and the kernels read dt there (dt itself is then unused); with the
// fixed step it is null.
struct Rates32 {
    const float* dt_dev;
    float dt, D, delta, rho, c;
    float kx, ky, kc;     // 0.5/dx^2, 0.5/dy^2, 0.25/(dx dy)
    float ihx2, ihy2;     // 1/dx^2, 1/dy^2
    float Kx, Ky;         // D/dx^2, D/dy^2 (tumour face weights, D folded in)
    float hKx, hKy;       // Kx/2, Ky/2
    float2 K2, nhK2;      // (Kx, Ky) and (-hKx, -hKy), for packed east / north faces
    int no_reaction;
};
Rates32 make_rates32(double dx, double dy, double dt, const gg_params& p);

// Launch plan of the FP32 step.  kind 0: shared-memory wavefront (strips of
// bx output columns plus a halo of `halo` columns on each side, chunks of by
// output rows, `threads` threads per CTA); kind 1: warp-register wavefront
// (strips of 32 - 2T columns per warp, chunks of by rows); kind 3: the
// paired-column warp wavefront (strips of 64 columns, 60 or 56 of them
// written, chunks of by rows).  T steps per pass.
struct Plan32 {
    int kind = 1;
    int T = 1;
    int bx = 256, by = 128, halo = 1, threads = 128;
};

size_t step32_smem_bytes(const Plan32& p, bool kahan);
cudaError_t launch_stepw(const Grid32& g, const Rates32& r, int H, int T, bool kahan, cudaStream_t s);
// Warps of the warp-register kernel with T steps per pass that the device
// holds at once (one wave); 0 if the occupancy query fails.
int stepw_wave_warps(int T, bool kahan);

// Destinations of the intermediate time levels of a pass (level t = 1..T-1
// writes u, v, w of step s0 + t to u[t-1], v[t-1], w[t-1]; a level with null
// destinations writes nothing); used to store the states of an adjoint
// segment in passes of T steps.
struct Stash32 {
    float* u[3];
    float* v[3];
    float* w[3];
};
// Paired-column warp wavefront (two columns per lane, 64-column strips):
// the same interface as launch_stepw / stepw_wave_warps, a variant that also
// writes the intermediate levels, and the columns a strip writes for T steps
// per pass.
cudaError_t launch_stepw2(const Grid32& g, const Rates32& r, int H, int T, bool kahan, cudaStream_t s);
cudaError_t launch_stepw2_stash(const Grid32& g, const Rates32& r, int H, int T, bool kahan, const Stash32& st,
                                cudaStream_t s);
int stepw2_wave_warps(int T, bool kahan);
int stepw2_out_columns(int T);
// One pass of T steps with the kernel the plan names.
cudaError_t launch_plan(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan, cudaStream_t s);
cudaError_t launch_step32(const Grid32& g, const Rates32& r, const Plan32& p, int T, bool kahan,
                          cudaStream_t s);

// FP64 plain step (one thread per cell).
struct Grid64 {
    const double* u; const double* v; const double* w;
    double* uo; double* vo; double* wo;
    const double* a11; const double* a12; const double* a22;
    int nx, ny, pitch;
};
struct Rates64 {
    const double* dt_dev;  // as Rates32::dt_dev
    double dt, D, delta, rho, c;
    double kx, ky, kc, ihx2, ihy2;
    int no_reaction;
};
cudaError_t launch_step64(const Grid64& g, const Rates64& r, cudaStream_t s);

// Coefficients of eq. (2) and validation counters.  fp64: a11, a12, a22
// per cell (pitched doubles) into c0, c1, c2; otherwise the FP32 coefficient
// fields ax, b, ay of Grid32 into c0, c1, c2 (dx, dy and scratch, two dense
// FP64 arrays of nx * ny, used only then).
// counters[0]: cells with lambda <= 0 or non-finite theta/lambda;
// counters[1]: non-finite initial values; lmax_bits: max lambda_max as the
// bit pattern of a non-negative double (atomicMax on unsigned long long).
cudaError_t launch_coefficients(const double* theta, const double* l1, const double* l2, int nx, int ny,
                                double dx, double dy, void* c0, void* c1, void* c2, int pitch, bool fp64,
                                double* scratch, unsigned long long* counters, unsigned long long* lmax_bits,
                                cudaStream_t s);
// One entry of eq. (2) (which = 0: a11, 1: a12, 2: a22) per cell from dense
// FP64 theta / lambda, into a dense buffer of n floats or doubles.
cudaError_t launch_tensor_entry(const double* theta, const double* l1, const double* l2, size_t n, int which,
                                void* dst, bool dst_fp64, cudaStream_t s);

// Dense FP64 host-layout field -> pitched FP32/FP64 device field (counts
// non-finite values into *nonfinite when it is not null).
cudaError_t launch_unpack(const void* src, bool src_fp64, void* dst, bool dst_fp64, int nx, int ny,
                          int pitch, unsigned long long* nonfinite, cudaStream_t s);
// Pitched device field -> dense device buffer.
cudaError_t launch_pack(const void* src, bool src_fp64, void* dst, bool dst_fp64, int nx, int ny,
                        int pitch, cudaStream_t s);

// Diagnostics: partials then a deterministic fixed-order final reduction.
// out[0..2] sums, [3..5] minima, [6..8] maxima, [9] non-finite count,
// [10] tumour cells, [11] gap cells (scaled by dx dy on the host).
cudaError_t launch_diagnostics(const void* u, const void* v, const void* w, bool fp64, int nx, int ny,
                               int pitch, double eps, double* partials, double* out, cudaStream_t s);

// The rates a kernel runs with: dt from the device when the step is adaptive.
__device__ __forceinline__ Rates32 live_rates(const Rates32& k)
{
    Rates32 r = k;
    if (k.dt_dev) r.dt = __ldg(k.dt_dev);
    return r;
}
__device__ __forceinline__ Rates64 live_rates(const Rates64& k)
{
    Rates64 r = k;
    if (k.dt_dev) r.dt = __ldg(k.dt_dev);
    return r;
}

// Adaptive step Delta t_k (gg_adapt.cu): per-cell terms of the rule in the
// state's precision F, and the device words it keeps.
template <typename F> struct AdaptRule {
    F D, rho, delta, ihx2, ihy2;
    int no_reaction;
};
struct AdaptState {
    double* dt64;     // current Delta t_k
    float* dt32;      // the same, rounded once, for the FP32 kernels
    double* t_done;   // simulated time up to the last recomputation
    void* kmax;       // two maxima (kU, kV) as bit patterns, zero between reductions
};
// Reduces the state's maxima, then sets Delta t_k = cfl / max(kW, kU, kV) and
// adds steps_prev times the previous Delta t to the simulated time.
template <typename F>
cudaError_t launch_adapt(const F* u, const F* v, const F* w, int nx, int ny, int pitch, const AdaptRule<F>& r,
                         double kW, double cfl, long long steps_prev, AdaptState& st, cudaStream_t s);

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Programmatic dependent launch for chains of passes on one stream (the
// adjoint's stash and reverse passes): the launch may be scheduled while the
// previous kernel of the stream is still draining, and the kernel waits for
// that kernel's completion and memory (griddepcontrol.wait) before its first
// global access; right after the wait it lets the next launch be scheduled.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                                  Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}
#ifdef __CUDACC__
// the device side of launch_chained
__device__ __forceinline__ void chained_wait()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
#endif

}  // namespace gg
