// Ensembles: many independent grids (their own size, rates, dt and tensor
// field) advanced by one persistent, cooperative, graph-captured launch.
//
// Work decomposition.  Every instance is cut into the warp tiles of the
// single-grid warp-register wavefront (strips of 32 - 2T columns, chunks of
// H rows); the tiles of all instances form one work list.  Each warp of a
// persistent CTA walks the list with a grid stride and runs one pass of T
// steps on each tile (warp_pass of gg_stepw.cuh, with L1-bypassing state
// loads), then all CTAs meet at a grid barrier before the next pass reads
// the state the previous pass wrote.  The barrier is a counter plus a
// generation word in global memory; a CTA that waits longer than the
// barrier timeout sets the device error word and leaves, so a wait can
// never hang the GPU: the next synchronizing call reports GG_ERR_TIMEOUT.
//
// Two more launch modes run the same work list as one ordinary launch per
// pass (the kernel boundary orders the passes): with the one-column warp
// tiles above, or with the tiles of the paired-column wavefront
// (gg_stepw2.cuh: 64-column strips, two columns per lane, each warp with its
// shared-memory row ring).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "gg_sim.cuh"
#include "gg_stepw.cuh"
#include "gg_stepw2.cuh"

using namespace gg;

namespace {

struct InstDesc {
    Grid32 g[2];    // g[p]: pass reading buffer p and writing buffer p ^ 1
    Rates32 r;
    int strips[2];  // warp strips for the plan's T (0) and for T = 1 (1)
};

struct InstHost {
    int nx, ny, pitch;
    double dx, dy, dt, dt_max, lambda_max;
    gg_params params;
    float* f[2][6];
    float* a[3];
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier.  bar[0] counts arrivals, bar[1] is the generation.
// Returns false (in every thread) if this CTA or another one gave up.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned expected, unsigned& gen,
                                             unsigned long long timeout_ns, int* s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned prev = atomicAdd(&bar[0], 1u);
        if (prev + 1 == expected) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (atomicAdd(&bar[1], 0u) == gen) {
                if (atomicAdd(err, 0) != 0) { ok = 0; break; }
                if (global_ns() - t0 > timeout_ns) { atomicExch(err, 1); ok = 0; break; }
                __nanosleep(100);
            }
        }
        __threadfence();
        gen += 1;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <int T, bool KAHAN>
__global__ void __launch_bounds__(128) batch_kernel(const InstDesc* __restrict__ desc, const int2* __restrict__ items,
                                                    int nitems, int npasses, int parity0, int variant, int H,
                                                    unsigned* bar, int* err, unsigned expected,
                                                    unsigned long long timeout_ns)
{
    __shared__ int s_ok;
    __shared__ unsigned s_gen;
    if (threadIdx.x == 0) s_gen = atomicAdd(&bar[1], 0u);
    __syncthreads();
    unsigned gen = s_gen;
    const int lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    // per warp: the grid and rates of its current item, staged in shared
    // memory (read there by the pass instead of from the global descriptor)
    __shared__ Grid32 sg[4];
    __shared__ Rates32 sr[4];
    const int wi = threadIdx.x >> 5;
    for (int pass = 0; pass < npasses; ++pass) {
        const int parity = (parity0 + pass) & 1;
        for (int w = blockIdx.x * wpc + wi; w < nitems; w += gridDim.x * wpc) {
            const int2 it = items[w];
            const InstDesc& d = desc[it.x];
            const int strips = d.strips[variant];
            const int sx = it.y % strips, sy = it.y / strips;
            __syncwarp();  // every lane is done with the previous item's copy
            const int* gsrc = reinterpret_cast<const int*>(&d.g[parity]);
            const int* rsrc = reinterpret_cast<const int*>(&d.r);
            for (int k = lane; k < (int)(sizeof(Grid32) / 4); k += 32) reinterpret_cast<int*>(&sg[wi])[k] = gsrc[k];
            for (int k = lane; k < (int)(sizeof(Rates32) / 4); k += 32) reinterpret_cast<int*>(&sr[wi])[k] = rsrc[k];
            __syncwarp();
            stepw::warp_pass_any<T, KAHAN, true>(sg[wi], sr[wi], H, sx, sy, lane);
        }
        if (pass + 1 < npasses && !grid_barrier(bar, err, expected, gen, timeout_ns, &s_ok)) return;
    }
}

// One pass of T steps over every work item, one warp per item (the
// "passes" mode: a graph of one launch per pass, no grid barrier; the kernel
// boundary orders the passes).  Without the persistent loop the compiler
// keeps fewer values in registers, so more warps fit on an SM.
template <int T, bool KAHAN>
__global__ void __launch_bounds__(32) pass_kernel(const InstDesc* __restrict__ desc, const int2* __restrict__ items,
                                                  int nitems, int parity, int variant, int H)
{
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const int2 it = items[w];
    const InstDesc& d = desc[it.x];
    const int strips = d.strips[variant];
    // the instance's grid and rates, staged in shared memory once: the pass
    // reads its pointers and scalars from there instead of from the
    // descriptor in global memory
    __shared__ Grid32 sg;
    __shared__ Rates32 sr;
    static_assert(sizeof(Grid32) % 4 == 0 && sizeof(Rates32) % 4 == 0, "word copy");
    const int* gsrc = reinterpret_cast<const int*>(&d.g[parity]);
    const int* rsrc = reinterpret_cast<const int*>(&d.r);
    for (int k = threadIdx.x; k < (int)(sizeof(Grid32) / 4); k += 32) reinterpret_cast<int*>(&sg)[k] = gsrc[k];
    for (int k = threadIdx.x; k < (int)(sizeof(Rates32) / 4); k += 32) reinterpret_cast<int*>(&sr)[k] = rsrc[k];
    __syncwarp();
    stepw::warp_pass_any<T, KAHAN>(sg, sr, H, it.y % strips, it.y / strips, threadIdx.x);
}

// The same pass with the paired-column tiles (one warp per tile, its
// shared-memory ring as dynamic shared memory).
extern __shared__ float2 g_batch_ring[];

// T = 3 and 4 are bound to 12 warps per SM (168 registers: three warps per
// scheduler); the T = 3 Kahan pass otherwise takes 170 registers and runs
// two warps per scheduler.
template <int T, bool KAHAN>
__global__ void __launch_bounds__(32, T >= 3 ? 12 : 1) pass2_kernel(const InstDesc* __restrict__ desc,
                                                                    const int2* __restrict__ items, int nitems,
                                                                    int parity, int variant, int H)
{
    const int w = blockIdx.x;
    if (w >= nitems) return;
    const int2 it = items[w];
    const InstDesc& d = desc[it.x];
    const int strips = d.strips[variant];
    __shared__ Grid32 sg;
    __shared__ Rates32 sr;
    const int* gsrc = reinterpret_cast<const int*>(&d.g[parity]);
    const int* rsrc = reinterpret_cast<const int*>(&d.r);
    for (int k = threadIdx.x; k < (int)(sizeof(Grid32) / 4); k += 32) reinterpret_cast<int*>(&sg)[k] = gsrc[k];
    for (int k = threadIdx.x; k < (int)(sizeof(Rates32) / 4); k += 32) reinterpret_cast<int*>(&sr)[k] = rsrc[k];
    __syncwarp();
    stepw2::warp_pass2_any<T, KAHAN>(sg, sr, H, it.y % strips, it.y / strips, threadIdx.x, g_batch_ring);
}

typedef void (*PassKernel)(const InstDesc*, const int2*, int, int, int, int);

template <bool KAHAN>
PassKernel pick_pass(int T)
{
    switch (T) {
        case 1: return pass_kernel<1, KAHAN>;
        case 2: return pass_kernel<2, KAHAN>;
        case 3: return pass_kernel<3, KAHAN>;
        default: return pass_kernel<4, KAHAN>;
    }
}

template <bool KAHAN>
PassKernel pick_pass2(int T)
{
    switch (T) {
        case 1: return pass2_kernel<1, KAHAN>;
        case 2: return pass2_kernel<2, KAHAN>;
        case 3: return pass2_kernel<3, KAHAN>;
        default: return pass2_kernel<4, KAHAN>;
    }
}

typedef void (*BatchKernel)(const InstDesc*, const int2*, int, int, int, int, int, unsigned*, int*, unsigned,
                            unsigned long long);

template <bool KAHAN>
BatchKernel pick(int T)
{
    switch (T) {
        case 1: return batch_kernel<1, KAHAN>;
        case 2: return batch_kernel<2, KAHAN>;
        case 3: return batch_kernel<3, KAHAN>;
        default: return batch_kernel<4, KAHAN>;
    }
}

constexpr int kBatchMaxT = 4;
// Launch modes of the ensemble (Plan32::kind): the persistent cooperative
// kernel with a grid barrier between passes, or one launch per pass with the
// one-column or the paired-column tiles.
constexpr int kModePersistent = 1;
constexpr int kModePasses = 2;
constexpr int kModePasses2 = 3;
inline bool per_pass(int mode) { return mode == kModePasses || mode == kModePasses2; }
// A step of more passes than this in the passes mode is launched directly
// instead of being captured into one graph.
constexpr int64_t kMaxCapturedPasses = 4096;

}  // namespace

struct gg_batch {
    int n = 0;
    int precision = GG_FP32_KAHAN;
    bool kahan = true;
    Plan32 plan;
    int cur = 0;
    int64_t steps = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<InstHost> inst;
    void* arena = nullptr;
    InstDesc* d_desc = nullptr;
    int2* d_items[2] = {nullptr, nullptr};  // work lists for the plan's T and for T = 1
    int nitems[2] = {0, 0};
    unsigned* d_bar = nullptr;  // [count, generation]
    int* d_err = nullptr;
    double* d_partials = nullptr;
    double* d_diag = nullptr;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    int ctas = 0;
    unsigned long long timeout_ns = 2000000000ull;  // 2 s per barrier wait
    unsigned extra_arrivals = 0;
    bool captured = false;          // the last gg_batch_step ran as a replayed CUDA graph
    cudaStream_t cap_stream = nullptr;  // private stream used only for stream capture
    int ctas_for_T[kBatchMaxT + 1] = {};  // persistent grid size per steps-per-pass value
    std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
    std::string last_error;
};

namespace {

int batch_fail(gg_batch* b, cudaError_t e, const char* where)
{
    if (b) b->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return GG_ERR_CUDA;
}

void build_desc(gg_batch* b, std::vector<InstDesc>& desc, std::vector<int2> items[2])
{
    desc.resize(b->n);
    items[0].clear();
    items[1].clear();
    const bool paired = b->plan.kind == kModePasses2;
    const int outs[2] = {paired ? stepw2_out_columns(b->plan.T) : 32 - 2 * b->plan.T,
                         paired ? stepw2_out_columns(1) : 30};
    for (int k = 0; k < b->n; ++k) {
        const InstHost& h = b->inst[k];
        InstDesc& d = desc[k];
        for (int p = 0; p < 2; ++p) {
            Grid32& g = d.g[p];
            const int q = p ^ 1;
            g.u = h.f[p][0]; g.v = h.f[p][1]; g.w = h.f[p][2];
            g.uo = h.f[q][0]; g.vo = h.f[q][1]; g.wo = h.f[q][2];
            g.cu = b->kahan ? h.f[p][3] : nullptr; g.cv = b->kahan ? h.f[p][4] : nullptr;
            g.cw = b->kahan ? h.f[p][5] : nullptr;
            g.cuo = b->kahan ? h.f[q][3] : nullptr; g.cvo = b->kahan ? h.f[q][4] : nullptr;
            g.cwo = b->kahan ? h.f[q][5] : nullptr;
            g.ax = h.a[0]; g.b = h.a[1]; g.ay = h.a[2];
            g.nx = h.nx; g.ny = h.ny; g.pitch = h.pitch;
        }
        d.r = make_rates32(h.dx, h.dy, h.dt, h.params);
        const int chunks = (h.ny + b->plan.by - 1) / b->plan.by;
        for (int v = 0; v < 2; ++v) {
            d.strips[v] = (h.nx + outs[v] - 1) / outs[v];
            for (int t = 0; t < d.strips[v] * chunks; ++t) items[v].push_back(make_int2(k, t));
        }
    }
}

int prepare_kernels(gg_batch* b);

// Upload descriptors and the work list for the current plan and size the
// persistent grid from the occupancy of the kernel that will run.
int configure(gg_batch* b, const Plan32& plan)
{
    b->plan = plan;
    std::vector<InstDesc> desc;
    std::vector<int2> items[2];
    build_desc(b, desc, items);
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 2; ++v) {
        if (b->d_items[v]) cudaFree(b->d_items[v]);
        b->d_items[v] = nullptr;
        e = cudaMalloc(&b->d_items[v], std::max<size_t>(items[v].size(), 1) * sizeof(int2));
        if (e != cudaSuccess) { cudaGetLastError(); b->last_error = "work list allocation failed"; return GG_ERR_OOM; }
        b->nitems[v] = (int)items[v].size();
    }
    e = cudaMemcpyAsync(b->d_desc, desc.data(), desc.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream);
    for (int v = 0; v < 2 && e == cudaSuccess; ++v)
        e = cudaMemcpyAsync(b->d_items[v], items[v].data(), items[v].size() * sizeof(int2), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch configure");
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return prepare_kernels(b);
}

int occupancy_ctas(gg_batch* b, BatchKernel k, size_t smem, int threads, int* out)
{
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, threads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return batch_fail(b, e, "occupancy");
    if (per_sm < 1) { b->last_error = "batch kernel does not fit on an SM"; return GG_ERR_ARG; }
    *out = per_sm * sms;
    return GG_OK;
}

BatchKernel kernel_for(const gg_batch* b, int T) { return b->kahan ? pick<true>(T) : pick<false>(T); }

// Sizes the persistent grids of the kernels for the plan's T and for T = 1
// from their occupancy.  Called outside stream capture: during capture only
// kernel launches are enqueued.
int prepare_kernels(gg_batch* b)
{
    if (per_pass(b->plan.kind)) return GG_OK;  // one CTA per work item, no persistent grid
    const int Ts[2] = {b->plan.T, 1};
    for (int v = 0; v < 2; ++v) {
        int ctas = 0;
        int rc = occupancy_ctas(b, kernel_for(b, Ts[v]), 0, b->plan.threads, &ctas);
        if (rc != GG_OK) return rc;
        const int warps_per_cta = b->plan.threads / 32;
        b->ctas_for_T[Ts[v]] = std::min(ctas, std::max((b->nitems[v] + warps_per_cta - 1) / warps_per_cta, 1));
    }
    return GG_OK;
}

// Enqueue one cooperative launch of `npasses` passes of T steps on stream st
// (variant 0: the plan's T; variant 1: T = 1).
int launch_passes(gg_batch* b, int T, int variant, int npasses, int parity0, cudaStream_t st)
{
    if (per_pass(b->plan.kind)) {
        const bool paired = b->plan.kind == kModePasses2;
        PassKernel pk = paired ? (b->kahan ? pick_pass2<true>(T) : pick_pass2<false>(T))
                               : (b->kahan ? pick_pass<true>(T) : pick_pass<false>(T));
        const size_t smem = paired ? (b->kahan ? stepw2::Ring<true>::bytes : stepw2::Ring<false>::bytes) : 0;
        const int nit = b->nitems[variant];
        for (int p = 0; p < npasses; ++p) {
            pk<<<std::max(nit, 1), 32, smem, st>>>(b->d_desc, b->d_items[variant], nit, (parity0 + p) & 1, variant,
                                                   b->plan.by);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return batch_fail(b, e, "batch pass launch");
        }
        b->ctas = nit;
        return GG_OK;
    }
    BatchKernel k = kernel_for(b, T);
    const int ctas = b->ctas_for_T[T];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(b->plan.threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const unsigned expected = (unsigned)ctas + b->extra_arrivals;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, (const InstDesc*)b->d_desc, (const int2*)b->d_items[variant],
                                       b->nitems[variant], npasses, parity0, variant, b->plan.by, b->d_bar,
                                       b->d_err, expected, b->timeout_ns);
    if (e != cudaSuccess) return batch_fail(b, e, "batch launch");
    b->ctas = ctas;
    return GG_OK;
}

// All launches of one gg_batch_step(nsteps) from buffer parity `parity`.
int enqueue_steps(gg_batch* b, int64_t nsteps, int parity, cudaStream_t st)
{
    const int T = b->plan.T;
    const int64_t main_passes = nsteps / T;
    const int rem = (int)(nsteps % T);
    int par = parity;
    int64_t left = main_passes;
    while (left > 0) {
        const int np = (int)std::min<int64_t>(left, 1 << 30);
        int rc = launch_passes(b, T, 0, np, par, st);
        if (rc != GG_OK) return rc;
        par = (par + np) & 1;
        left -= np;
    }
    if (rem) {
        int rc = launch_passes(b, 1, 1, rem, par, st);  // the remainder as single steps
        if (rc != GG_OK) return rc;
    }
    return GG_OK;
}

int check_error_word(gg_batch* b)
{
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, b->d_err, sizeof err, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch sync");
    if (err) {
        b->last_error = "a grid-barrier wait exceeded its time limit; the state of this batch is unreliable";
        // reset the barrier so that later launches start clean
        cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream);
        cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
        cudaStreamSynchronize(b->stream);
        return GG_ERR_TIMEOUT;
    }
    return GG_OK;
}

}  // namespace

extern "C" {

int gg_batch_create(int32_t n, const gg_grid* grids, const gg_params* params, const double* const* fields,
                    void* cuda_stream, gg_batch** out)
{
    if (!out) return GG_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !grids || !params || !fields) return GG_ERR_ARG;
    const int prec = params[0].precision;
    if (prec != GG_FP32 && prec != GG_FP32_KAHAN) return GG_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        if (params[k].precision != prec) return GG_ERR_ARG;
        if (params[k].adapt_every != 0) return GG_ERR_ARG;  // ensembles run fixed steps
        for (int m = 0; m < 6; ++m)
            if (!fields[6 * k + m]) return GG_ERR_ARG;
        if (params[k].steps_per_pass > kBatchMaxT || params[k].steps_per_pass != params[0].steps_per_pass)
            return GG_ERR_ARG;
    }
    gg_batch* b = new gg_batch();
    b->n = n;
    b->precision = prec;
    b->kahan = prec == GG_FP32_KAHAN;
    b->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&b->device);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->cap_stream = nullptr;  // no capture: gg_batch_step launches directly
    }
    b->inst.resize(n);
    // Each instance is created as a gg_sim (validation, tensor build, dt),
    // then its device state is copied into the batch arena and the sim freed.
    size_t total = 0;
    std::vector<size_t> fstride(n);
    const int nstate = b->kahan ? 6 : 3;
    for (int k = 0; k < n; ++k) {
        const int pitch = round_up(grids[k].nx, 32);
        fstride[k] = ((size_t)pitch * std::max(grids[k].ny, 1) * 4 + 255) / 256 * 256;
        total += fstride[k] * (2 * nstate + 3);
    }
    const size_t desc_bytes = ((size_t)n * sizeof(InstDesc) + 255) / 256 * 256;
    const size_t diag_bytes = (size_t)kDiagBlocks * kDiagStride * 8 + 32 * 8;
    total += desc_bytes + 256 + diag_bytes;
    cudaError_t e = cudaMalloc(&b->arena, total);
    if (e != cudaSuccess) { cudaGetLastError(); delete b; return GG_ERR_OOM; }
    e = cudaMemsetAsync(b->arena, 0, total, b->stream);
    char* p = (char*)b->arena;
    b->d_desc = (InstDesc*)p; p += desc_bytes;
    b->d_bar = (unsigned*)p;
    b->d_err = (int*)(p + 16);
    p += 256;
    b->d_partials = (double*)p; p += (size_t)kDiagBlocks * kDiagStride * 8;
    b->d_diag = (double*)p; p += 32 * 8;
    int rc = GG_OK;
    for (int k = 0; k < n && rc == GG_OK && e == cudaSuccess; ++k) {
        gg_sim* s = nullptr;
        gg_params pk = params[k];
        rc = gg_create(&grids[k], &pk, fields[6 * k], fields[6 * k + 1], fields[6 * k + 2], fields[6 * k + 3],
                       fields[6 * k + 4], fields[6 * k + 5], cuda_stream, &s);
        if (rc != GG_OK) {
            char buf[256];
            snprintf(buf, sizeof buf, "instance %d: %s", k, gg_last_error(nullptr));
            b->last_error = buf;
            break;
        }
        InstHost& h = b->inst[k];
        h.nx = s->nx; h.ny = s->ny; h.pitch = s->pitch;
        h.dx = s->dx; h.dy = s->dy; h.dt = s->dt; h.dt_max = s->dt_max; h.lambda_max = s->lambda_max;
        h.params = s->params;
        for (int bb = 0; bb < 2; ++bb)
            for (int f = 0; f < 6; ++f) h.f[bb][f] = nullptr;
        for (int bb = 0; bb < 2; ++bb)
            for (int f = 0; f < nstate; ++f) { h.f[bb][f] = (float*)p; p += fstride[k]; }
        for (int f = 0; f < 3; ++f) { h.a[f] = (float*)p; p += fstride[k]; }
        const size_t fb = (size_t)s->pitch * s->ny * 4;
        for (int f = 0; f < nstate && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(h.f[0][f], s->f32[s->cur][f], fb, cudaMemcpyDeviceToDevice, b->stream);
        for (int f = 0; f < 3 && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(h.a[f], s->a32[f], fb, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        gg_destroy(s);
    }
    if (rc == GG_OK && e != cudaSuccess) rc = batch_fail(b, e, "batch create");
    if (rc != GG_OK) {
        std::string why = b->last_error;
        gg_batch_destroy(b);
        (void)why;
        return rc;
    }
    // Launch plan: one tile shape for the whole ensemble.  The autotuner of
    // gg_batch_autotune may replace it.
    int maxnx = 0;
    for (auto& h : b->inst) maxnx = std::max(maxnx, h.nx);
    Plan32 plan;
    plan.kind = 1;
    plan.T = params[0].steps_per_pass > 0 ? params[0].steps_per_pass : 1;
    plan.halo = plan.T;
    plan.bx = 32 - 2 * plan.T;
    plan.by = 64;
    plan.threads = 128;
    (void)maxnx;
    rc = configure(b, plan);
    if (rc != GG_OK) { gg_batch_destroy(b); return rc; }
    *out = b;
    return GG_OK;
}

int gg_batch_step(gg_batch* b, int64_t nsteps)
{
    if (!b) return GG_ERR_ARG;
    if (nsteps < 0) { b->last_error = "nsteps < 0"; return GG_ERR_ARG; }
    if (nsteps == 0) return GG_OK;
    const auto key = std::make_pair(nsteps, b->cur);
    auto it = b->graphs.find(key);
    cudaError_t e = cudaSuccess;
    const int64_t npass = nsteps / b->plan.T + nsteps % b->plan.T;
    const bool capturable = !per_pass(b->plan.kind) || npass <= kMaxCapturedPasses;
    if (it == b->graphs.end() && b->cap_stream && capturable) {
        // Capture the launches of this (nsteps, parity) once on the private
        // stream, replay the graph on the caller's stream afterwards.
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int rc = enqueue_steps(b, nsteps, b->cur, b->cap_stream);
            const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
            if (rc != GG_OK || e2 != cudaSuccess) e = e2 != cudaSuccess ? e2 : cudaErrorStreamCaptureInvalidated;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) {
            it = b->graphs.emplace(key, exec).first;
        } else {
            cudaGetLastError();
            b->last_error = std::string("stream capture of the persistent launch failed (") + cudaGetErrorString(e) +
                            "); launching it directly";
        }
    }
    if (it != b->graphs.end()) {
        e = cudaGraphLaunch(it->second, b->stream);
        if (e != cudaSuccess) return batch_fail(b, e, "batch graph launch");
        b->captured = true;
    } else {
        const int rc = enqueue_steps(b, nsteps, b->cur, b->stream);
        if (rc != GG_OK) return rc;
        b->captured = false;
    }
    const int64_t passes = nsteps / b->plan.T + nsteps % b->plan.T;
    b->cur = (int)((b->cur + passes) & 1);
    b->steps += nsteps;
    return GG_OK;
}

int gg_batch_launch_info(const gg_batch* b, int32_t* info)
{
    if (!b || !info) return GG_ERR_ARG;
    info[0] = b->plan.T;
    info[1] = b->plan.bx;
    info[2] = b->plan.by;
    info[3] = b->plan.threads;
    info[4] = b->ctas;
    info[5] = b->nitems[0];
    info[6] = b->captured ? 1 : 0;
    info[7] = b->plan.kind == kModePasses ? 1 : (b->plan.kind == kModePasses2 ? 2 : 0);
    return GG_OK;
}

int gg_batch_read(gg_batch* b, int32_t inst, int32_t field, void* dst, int32_t dst_on_device, int32_t dst_fp64)
{
    if (!b) return GG_ERR_ARG;
    if (inst < 0 || inst >= b->n || !dst) { b->last_error = "bad instance or dst"; return GG_ERR_ARG; }
    int rc = check_error_word(b);
    if (rc != GG_OK) return rc;
    InstHost& h = b->inst[inst];
    const float* src = nullptr;
    if (field >= GG_FIELD_U && field <= GG_FIELD_W) src = h.f[b->cur][field];
    else if (field >= GG_FIELD_COMP_U && field <= GG_FIELD_COMP_W) src = b->kahan ? h.f[b->cur][field] : nullptr;
    else if (field >= GG_FIELD_A11 && field <= GG_FIELD_A22) src = h.a[field - GG_FIELD_A11];
    if (!src) { b->last_error = "field not available"; return GG_ERR_ARG; }
    const size_t n = (size_t)h.nx * h.ny;
    const size_t bytes = n * (dst_fp64 ? 8 : 4);
    cudaError_t e;
    if (dst_on_device) {
        e = launch_pack(src, false, dst, dst_fp64 != 0, h.nx, h.ny, h.pitch, b->stream);
    } else {
        if (b->staging_bytes < bytes) {
            if (b->staging) cudaFree(b->staging);
            b->staging = nullptr;
            b->staging_bytes = 0;
            e = cudaMalloc(&b->staging, bytes);
            if (e != cudaSuccess) { cudaGetLastError(); b->last_error = "staging allocation failed"; return GG_ERR_OOM; }
            b->staging_bytes = bytes;
        }
        e = launch_pack(src, false, b->staging, dst_fp64 != 0, h.nx, h.ny, h.pitch, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, b->staging, bytes, cudaMemcpyDeviceToHost, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch read");
    return GG_OK;
}

int gg_batch_diagnostics(gg_batch* b, int32_t inst, gg_diag* out)
{
    if (!b) return GG_ERR_ARG;
    if (inst < 0 || inst >= b->n || !out) { b->last_error = "bad instance or out"; return GG_ERR_ARG; }
    int rc = check_error_word(b);
    if (rc != GG_OK) return rc;
    InstHost& h = b->inst[inst];
    double hd[12];
    cudaError_t e = launch_diagnostics(h.f[b->cur][0], h.f[b->cur][1], h.f[b->cur][2], false, h.nx, h.ny, h.pitch,
                                       0.01, b->d_partials, b->d_diag, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd, b->d_diag, sizeof hd, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "batch diagnostics");
    const double cell = h.dx * h.dy;
    for (int k = 0; k < 3; ++k) {
        out->mass[k] = hd[k] * cell;
        out->min[k] = hd[3 + k];
        out->max[k] = hd[6 + k];
    }
    out->nonfinite = (int64_t)hd[9];
    out->tumour_area = hd[10] * cell;
    out->gap_area = hd[11] * cell;
    out->gap_eps = 0.01;
    return out->nonfinite ? GG_ERR_NONFINITE : GG_OK;
}

int gg_batch_autotune(gg_batch* b, int64_t trial_steps, int32_t* chosen)
{
    if (!b) return GG_ERR_ARG;
    if (trial_steps < 1) trial_steps = 8;
    int maxnx = 0;
    for (auto& h : b->inst) maxnx = std::max(maxnx, h.nx);
    // Candidates: steps per pass and chunk height of the warp tiles.
    std::vector<Plan32> cands;
    for (int mode : {kModePersistent, kModePasses, kModePasses2})
        for (int T = 1; T <= kBatchMaxT; ++T) {
            // intermediate heights: on the 256-instance workload 40-56-row chunks
            // ran 4 % faster than 32 or 64 (halo rows against whole waves)
            const std::vector<int> bys = {32, 40, 48, 56, 64, 96, 128, 256};
            for (int by : bys) {
                if (by < 4 * T + 8) continue;
                Plan32 p;
                p.kind = mode; p.T = T; p.halo = T; p.by = by;
                p.bx = mode == kModePasses2 ? stepw2_out_columns(T) : 32 - 2 * T;
                p.threads = per_pass(mode) ? 32 : 128;
                cands.push_back(p);
            }
        }
    // Tuning runs advance the state: save it and restore it afterwards.
    const int nstate = b->kahan ? 6 : 3;
    size_t bytes = 0;
    for (auto& h : b->inst) bytes += (size_t)h.pitch * h.ny * 4 * nstate;
    void* save = nullptr;
    cudaError_t e = cudaMalloc(&save, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); b->last_error = "autotune save buffer allocation failed"; return GG_ERR_OOM; }
    auto copy_state = [&](bool to_save) {
        char* q = (char*)save;
        cudaError_t ee = cudaSuccess;
        for (auto& h : b->inst)
            for (int f = 0; f < nstate && ee == cudaSuccess; ++f) {
                const size_t fb = (size_t)h.pitch * h.ny * 4;
                ee = to_save ? cudaMemcpyAsync(q, h.f[b->cur][f], fb, cudaMemcpyDeviceToDevice, b->stream)
                             : cudaMemcpyAsync(h.f[b->cur][f], q, fb, cudaMemcpyDeviceToDevice, b->stream);
                q += fb;
            }
        return ee;
    };
    e = copy_state(true);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Plan32 orig = b->plan;
    const int orig_cur = b->cur;
    Plan32 bestp = orig;
    int rc = GG_OK;
    // per-step device time of plan p over about `steps` steps, the least of
    // `reps` timed runs after one untimed run
    auto time_plan = [&](const Plan32& p, int64_t steps, int reps) -> double {
        double t = 1e300;
        rc = configure(b, p);
        if (rc != GG_OK) return t;
        const int64_t n = std::max<int64_t>(steps / p.T, 1) * p.T;
        rc = enqueue_steps(b, n, b->cur, b->stream);  // warm-up
        for (int rep = 0; rep < reps && rc == GG_OK && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, b->stream);
            rc = enqueue_steps(b, n, b->cur, b->stream);
            cudaEventRecord(e1, b->stream);
            if (rc != GG_OK) break;
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, ms / (double)n);
        }
        return t;
    };
    // a short trial of every candidate, then the three fastest again over
    // four times as many steps, best of two
    std::vector<std::pair<double, size_t>> trial;
    for (size_t i = 0; i < cands.size() && rc == GG_OK && e == cudaSuccess; ++i)
        trial.push_back({time_plan(cands[i], trial_steps, 1), i});
    std::sort(trial.begin(), trial.end());
    double best = 1e300;
    for (size_t j = 0; j < trial.size() && j < 3 && rc == GG_OK && e == cudaSuccess; ++j) {
        const double t = time_plan(cands[trial[j].second], 4 * trial_steps, 2);
        if (rc == GG_OK && e == cudaSuccess && t < best) {
            best = t;
            bestp = cands[trial[j].second];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cur = orig_cur;
    if (e == cudaSuccess) e = copy_state(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(save);
    if (rc == GG_OK && e != cudaSuccess) rc = batch_fail(b, e, "autotune");
    int rc2 = configure(b, rc == GG_OK ? bestp : orig);
    if (rc == GG_OK) rc = rc2;
    if (rc == GG_OK) rc = check_error_word(b);
    if (chosen) {
        chosen[0] = b->plan.T; chosen[1] = b->plan.bx; chosen[2] = b->plan.by; chosen[3] = b->plan.threads;
    }
    return rc;
}

int gg_batch_set_plan(gg_batch* b, int32_t passes_mode, int32_t T, int32_t chunk)
{
    if (!b) return GG_ERR_ARG;
    if (T < 1 || T > kBatchMaxT || chunk < 0 || passes_mode < 0 || passes_mode > 2) {
        b->last_error = "set_plan: T must be 1..4, chunk >= 0 and passes_mode 0, 1 or 2";
        return GG_ERR_ARG;
    }
    Plan32 p;
    p.kind = passes_mode == 2 ? kModePasses2 : (passes_mode == 1 ? kModePasses : kModePersistent);
    p.T = T; p.halo = T;
    p.bx = passes_mode == 2 ? stepw2_out_columns(T) : 32 - 2 * T;
    p.by = chunk > 0 ? chunk : 64;
    p.threads = passes_mode ? 32 : 128;
    return configure(b, p);
}

int gg_batch_set_barrier_timeout(gg_batch* b, double seconds, int32_t extra_arrivals)
{
    if (!b || !(seconds > 0.0) || seconds > 60.0 || extra_arrivals < 0 || extra_arrivals > 1) return GG_ERR_ARG;
    b->timeout_ns = (unsigned long long)(seconds * 1e9);
    b->extra_arrivals = (unsigned)extra_arrivals;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return GG_OK;
}

int32_t gg_batch_steps_per_pass(const gg_batch* b) { return b ? b->plan.T : 0; }

double gg_batch_dt(const gg_batch* b, int32_t inst)
{
    if (!b || inst < 0 || inst >= b->n) return 0.0;
    return b->inst[inst].dt;
}

const char* gg_batch_last_error(const gg_batch* b) { return b ? b->last_error.c_str() : ""; }

int gg_batch_destroy(gg_batch* b)
{
    if (!b) return GG_OK;
    cudaStreamSynchronize(b->stream);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int v = 0; v < 2; ++v)
        if (b->d_items[v]) cudaFree(b->d_items[v]);
    if (b->staging) cudaFree(b->staging);
    if (b->arena) cudaFree(b->arena);
    delete b;
    return GG_OK;
}

}  // extern "C"
