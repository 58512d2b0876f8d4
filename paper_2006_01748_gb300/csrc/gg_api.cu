// Host side of the C ABI declared in include/gg.h: argument validation,
// device memory of a simulation, the fixed time step, the launch plan and
// the read / write / diagnostics entry points.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gg_internal.cuh"
#include "gg_sim.cuh"

using namespace gg;

namespace gg {

void set_error(gg_sim* s, const char* fmt, const char* detail)
{
    if (!s) return;
    char buf[512];
    snprintf(buf, sizeof buf, fmt, detail ? detail : "");
    s->last_error = buf;
}

int cuda_fail(gg_sim* s, cudaError_t e, const char* where)
{
    if (s) s->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return GG_ERR_CUDA;
}

double stable_dt_max(double dx, double dy, double Lambda, const gg_params& p)
{
    const double L = std::max(Lambda, p.D);
    return 1.0 / (2.0 * L * (1.0 / (dx * dx) + 1.0 / (dy * dy)) + (p.c + p.rho + 1.0 + p.delta));
}

Rates32 make_rates32(double dx, double dy, double dt, const gg_params& p)
{
    Rates32 r;
    r.dt_dev = nullptr;
    r.dt = (float)dt;
    r.D = (float)p.D;
    r.delta = (float)p.delta;
    r.rho = (float)p.rho;
    r.c = (float)p.c;
    r.kx = (float)(0.5 / (dx * dx));
    r.ky = (float)(0.5 / (dy * dy));
    r.kc = (float)(0.25 / (dx * dy));
    r.ihx2 = (float)(1.0 / (dx * dx));
    r.ihy2 = (float)(1.0 / (dy * dy));
    r.Kx = (float)(p.D / (dx * dx));
    r.Ky = (float)(p.D / (dy * dy));
    r.hKx = (float)(0.5 * p.D / (dx * dx));
    r.hKy = (float)(0.5 * p.D / (dy * dy));
    r.K2 = make_float2(r.Kx, r.Ky);
    r.nhK2 = make_float2(-r.hKx, -r.hKy);
    r.no_reaction = (p.flags & GG_FLAG_NO_REACTION) ? 1 : 0;
    return r;
}

Rates32 rates32(const gg_sim* s)
{
    Rates32 r = make_rates32(s->dx, s->dy, s->dt, s->params);
    if (s->params.adapt_every > 0) r.dt_dev = s->adapt.dt32;
    return r;
}

cudaError_t adapt_now(gg_sim* s)
{
    const bool fp64 = s->params.precision == GG_FP64_PLAIN;
    const int nr = (s->params.flags & GG_FLAG_NO_REACTION) ? 1 : 0;
    const double ihx2 = 1.0 / (s->dx * s->dx), ihy2 = 1.0 / (s->dy * s->dy);
    cudaError_t e;
    if (fp64) {
        AdaptRule<double> r{s->params.D, s->params.rho, s->params.delta, ihx2, ihy2, nr};
        e = launch_adapt<double>(s->f64[s->cur][0], s->f64[s->cur][1], s->f64[s->cur][2], s->nx, s->ny, s->pitch, r,
                                 s->kW, s->params.cfl, s->since_adapt, s->adapt, s->stream);
    } else {
        AdaptRule<float> r{(float)s->params.D, (float)s->params.rho, (float)s->params.delta, (float)ihx2,
                           (float)ihy2, nr};
        e = launch_adapt<float>(s->f32[s->cur][0], s->f32[s->cur][1], s->f32[s->cur][2], s->nx, s->ny, s->pitch, r,
                                s->kW, s->params.cfl, s->since_adapt, s->adapt, s->stream);
    }
    if (e == cudaSuccess) s->since_adapt = 0;
    return e;
}

Grid32 grid32(const gg_sim* s, int cur)
{
    Grid32 g;
    const int nxt = cur ^ 1;
    g.u = s->f32[cur][0]; g.v = s->f32[cur][1]; g.w = s->f32[cur][2];
    g.uo = s->f32[nxt][0]; g.vo = s->f32[nxt][1]; g.wo = s->f32[nxt][2];
    const bool k = s->params.precision == GG_FP32_KAHAN;
    g.cu = k ? s->f32[cur][3] : nullptr; g.cv = k ? s->f32[cur][4] : nullptr; g.cw = k ? s->f32[cur][5] : nullptr;
    g.cuo = k ? s->f32[nxt][3] : nullptr; g.cvo = k ? s->f32[nxt][4] : nullptr; g.cwo = k ? s->f32[nxt][5] : nullptr;
    g.ax = s->a32[0]; g.b = s->a32[1]; g.ay = s->a32[2];
    g.nx = s->nx; g.ny = s->ny; g.pitch = s->pitch;
    return g;
}

// Default launch plan: the warp-register wavefront with chunks of rows sized
// so that the grid holds about 16 warps per SM (152 SMs) when the domain
// allows it, never below 4T + 8 rows and never above 256 rows.  For T > 4 the
// shared-memory wavefront (strips of at most 256 columns, chunks of 8T..128
// rows, about 4 CTAs per SM).
Plan32 default_plan(int nx, int ny, int T)
{
    Plan32 p;
    p.T = T;
    p.halo = T;
    p.threads = 128;
    if (T <= 4) {
        // warp-register wavefront, two columns per lane for T >= 2 (the
        // faster kernel at every T >= 2 on the 8192 x 8192 tissue); chunk
        // heights from the 8192 x 8192 sweeps (64 rows for T <= 2, 128 for
        // T = 3 and for the paired T = 4, 256 for the one-column T = 4),
        // lowered when the grid would give fewer than about 16 warps per SM
        if (T >= 2) {
            p.kind = 3;
            const int out = stepw2_out_columns(T);
            const int nstrips = (nx + out - 1) / out;
            const int preferred = T <= 2 ? 64 : 128;
            const int chunks = std::max(1, (12 * 152 + nstrips - 1) / nstrips);
            int H = round_up((ny + chunks - 1) / chunks, 8);
            H = std::max(std::min(H, preferred), 4 * T + 8);
            p.by = std::min(ny, H);
            p.bx = out;
            return p;
        }
        p.kind = 1;
        const int out = 32 - 2 * T;
        const int nstrips = (nx + out - 1) / out;
        const int preferred = T <= 2 ? 64 : (T == 3 ? 128 : 256);
        const int target_warps = 16 * 152;
        const int chunks = std::max(1, (target_warps + nstrips - 1) / nstrips);
        int H = round_up((ny + chunks - 1) / chunks, 8);
        H = std::max(std::min(H, preferred), 4 * T + 8);
        p.by = std::min(ny, H);
        p.bx = out;
        return p;
    }
    p.kind = 0;
    const int ns = (nx + 255) / 256;
    p.bx = round_up((nx + ns - 1) / ns, 4);
    const int target_ctas = 4 * 152;
    const int chunks = (target_ctas + ns - 1) / ns;
    int by = round_up((ny + chunks - 1) / chunks, 8);
    by = std::max(by, std::max(16, 8 * T));
    by = std::min(by, 128);
    p.by = std::min(ny, by);
    return p;
}

// ---------------------------------------------------------------- autotuner
//
// Times every candidate plan on the simulation itself and keeps the fastest
// per step: the warp-register wavefront with T in {1, 2, 3, 4} and chunk
// heights {16, 32, 64, 128, 256}, and the shared-memory wavefront with T in
// {1, 2, 4, 8} and chunk heights {32, 64, 128}.  The state it advances is
// saved first and restored afterwards, so tuning leaves the run unchanged
// (every plan computes the same bits).  Results are cached per process by
// (nx, ny, precision).
namespace {
struct TuneKey {
    int nx, ny, precision;
    bool operator<(const TuneKey& o) const
    {
        return nx != o.nx ? nx < o.nx : ny != o.ny ? ny < o.ny : precision < o.precision;
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, Plan32> g_tune_cache;
}  // namespace

Plan32 tune_plan(gg_sim* s, int64_t trial_steps)
{
    const bool kahan = s->params.precision == GG_FP32_KAHAN;
    const int nstate = kahan ? 6 : 3;
    if (trial_steps < 1) trial_steps = 48;
    const int64_t n = (trial_steps + 23) / 24 * 24;  // a multiple of every T tried
    std::vector<Plan32> cands;
    for (int T = 1; T <= 4; ++T) {
        // fixed heights, and the four largest heights (at most 256 rows) for
        // which the grid fills a whole number of waves of resident warps (a
        // partial last wave costs nearly a full one)
        std::vector<int> Hs = {16, 32, 64, 128, 256};
        const int wave = stepw_wave_warps(T, kahan);
        const int strips = (s->nx + 32 - 2 * T - 1) / (32 - 2 * T);
        if (wave > 0 && strips <= wave) {
            int added = 0;
            for (int m = 1; added < 4; ++m) {
                const int nch = (int)((int64_t)m * wave / strips);  // chunk rows filling m waves
                const int H = (s->ny + nch - 1) / nch;
                if (H < 4 * T + 8) break;
                if (H > 256) continue;
                if (std::find(Hs.begin(), Hs.end(), H) == Hs.end()) Hs.push_back(H);
                ++added;
            }
        }
        for (int H : Hs) {
            if (H < 4 * T + 8 && H != 256) continue;
            Plan32 p = default_plan(s->nx, s->ny, T);
            p.kind = 1;
            p.bx = 32 - 2 * T;
            p.by = std::min(s->ny, H);
            cands.push_back(p);
        }
        // the paired-column warp wavefront: fixed heights and the whole-wave ones
        std::vector<int> H2 = {16, 32, 64, 128, 256};
        const int wave2 = stepw2_wave_warps(T, kahan);
        const int strips2 = (s->nx + stepw2_out_columns(T) - 1) / stepw2_out_columns(T);
        if (wave2 > 0 && strips2 <= wave2) {
            int added = 0;
            for (int m = 1; added < 4; ++m) {
                const int nch = (int)((int64_t)m * wave2 / strips2);  // chunk rows filling m waves
                const int H = (s->ny + nch - 1) / nch;
                if (H < 4 * T + 8) break;
                if (H > 256) continue;
                if (std::find(H2.begin(), H2.end(), H) == H2.end()) H2.push_back(H);
                ++added;
            }
        }
        for (int H : H2) {
            if (H < 4 * T + 8 && H != 256) continue;
            Plan32 p = default_plan(s->nx, s->ny, T);
            p.kind = 3;
            p.bx = stepw2_out_columns(T);
            p.by = std::min(s->ny, H);
            cands.push_back(p);
        }
    }
    for (int T : {1, 2, 4, 8})
        for (int by : {32, 64, 128}) {
            if (by < 8 * T) continue;
            Plan32 p = default_plan(s->nx, s->ny, 8);  // shared-memory geometry
            p.T = T;
            p.halo = T;
            p.by = std::min(s->ny, by);
            cands.push_back(p);
        }
    const size_t fbytes = (size_t)s->pitch * s->ny * 4;
    void* save = nullptr;
    Plan32 best = s->plan;
    if (cudaMalloc(&save, fbytes * nstate) != cudaSuccess) {
        cudaGetLastError();
        return best;  // no room to tune: keep the default plan
    }
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < nstate && e == cudaSuccess; ++f)
        e = cudaMemcpyAsync((char*)save + f * fbytes, s->f32[s->cur][f], fbytes, cudaMemcpyDeviceToDevice, s->stream);
    const Rates32 r = rates32(s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int cur = s->cur;
    // device time of `steps` steps of plan p, the least of `reps` timed runs
    // after one untimed run
    auto time_plan = [&](const Plan32& p, int64_t steps, int reps) -> double {
        double t = 1e300;
        for (int rep = 0; rep <= reps && e == cudaSuccess; ++rep) {
            if (rep > 0) e = cudaEventRecord(e0, s->stream);
            for (int64_t k = 0; k < steps && e == cudaSuccess; k += p.T) {
                e = launch_plan(grid32(s, cur), r, p, p.T, kahan, s->stream);
                cur ^= 1;
            }
            if (rep == 0) continue;
            if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess) t = std::min(t, (double)ms);
        }
        return t;
    };
    // a short trial of every candidate, then the four fastest again over four
    // times as many steps, three times each: single short trials picked a
    // plan 9 % slower than the best in some runs at 2048 x 2048
    std::vector<std::pair<double, size_t>> trial;
    for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) trial.push_back({time_plan(cands[i], n, 1), i});
    std::sort(trial.begin(), trial.end());
    double best_ms = 1e300;
    for (size_t j = 0; j < trial.size() && j < 4 && e == cudaSuccess; ++j) {
        const double t = time_plan(cands[trial[j].second], 4 * n, 3);
        if (e == cudaSuccess && t < best_ms) {
            best_ms = t;
            best = cands[trial[j].second];
        }
    }
    // restore the state into the current buffer
    for (int f = 0; f < nstate && e == cudaSuccess; ++f)
        e = cudaMemcpyAsync(s->f32[s->cur][f], (char*)save + f * fbytes, fbytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->last_error = std::string("autotune: ") + cudaGetErrorString(e);
        return s->plan;
    }
    return best;
}

Plan32 cached_plan(gg_sim* s)
{
    const TuneKey key{s->nx, s->ny, s->params.precision};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return it->second;
    }
    const Plan32 p = tune_plan(s, 24);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = p;
    return p;
}

}  // namespace gg

namespace {

bool finite_nonneg(double x) { return isfinite(x) && x >= 0.0; }

int validate(const gg_grid* grid, const gg_params* params, std::string& why)
{
    if (!grid || !params) { why = "grid or params is NULL"; return GG_ERR_ARG; }
    if (grid->nx < 1 || grid->ny < 1) { why = "nx and ny must be >= 1"; return GG_ERR_ARG; }
    if ((int64_t)grid->nx * grid->ny > (int64_t)1 << 31) { why = "nx*ny must be <= 2^31"; return GG_ERR_ARG; }
    if (!(isfinite(grid->lx) && grid->lx >= 0) || !(isfinite(grid->ly) && grid->ly >= 0)) {
        why = "lx, ly must be finite and >= 0"; return GG_ERR_ARG;
    }
    const gg_params& p = *params;
    if (!finite_nonneg(p.delta) || !finite_nonneg(p.rho) || !finite_nonneg(p.D) || !finite_nonneg(p.c)) {
        why = "delta, rho, D, c must be finite and >= 0"; return GG_ERR_ARG;
    }
    if (!(isfinite(p.cfl) && p.cfl >= 0.0 && p.cfl <= 1.0)) { why = "cfl must lie in [0, 1]"; return GG_ERR_ARG; }
    if (!(isfinite(p.dt) && p.dt >= 0.0)) { why = "dt must be finite and >= 0"; return GG_ERR_ARG; }
    if (p.precision != GG_FP64_PLAIN && p.precision != GG_FP32 && p.precision != GG_FP32_KAHAN) {
        why = "unknown precision"; return GG_ERR_ARG;
    }
    if (p.flags & ~(GG_FLAG_NO_REACTION | GG_FLAG_ALLOW_UNSTABLE)) { why = "unknown flag bits"; return GG_ERR_ARG; }
    if (p.steps_per_pass < 0 || p.steps_per_pass > kMaxT) { why = "steps_per_pass must lie in [0, 8]"; return GG_ERR_ARG; }
    if (p.adapt_every < 0) { why = "adapt_every must be >= 0"; return GG_ERR_ARG; }
    if (p.adapt_every > 0 && p.dt != 0.0) { why = "an explicit dt and the adaptive step exclude each other"; return GG_ERR_ARG; }
    return GG_OK;
}

thread_local std::string g_create_error;

}  // namespace

extern "C" {

const char* gg_error_string(int32_t status)
{
    switch (status) {
        case GG_OK: return "ok";
        case GG_ERR_ARG: return "invalid argument";
        case GG_ERR_NOT_SPD: return "diffusion tensor not positive definite (lambda <= 0)";
        case GG_ERR_CFL: return "time step above the stable bound";
        case GG_ERR_OOM: return "device out of memory";
        case GG_ERR_CUDA: return "CUDA error";
        case GG_ERR_NONFINITE: return "non-finite state";
        case GG_ERR_TIMEOUT: return "device-side wait timed out";
        case GG_ERR_STATE: return "call not valid in this state";
        default: return "unknown status";
    }
}

const char* gg_last_error(const gg_sim* s) { return s ? s->last_error.c_str() : g_create_error.c_str(); }

int gg_create(const gg_grid* grid, const gg_params* params, const double* theta, const double* lambda1,
              const double* lambda2, const double* u0, const double* v0, const double* w0, void* cuda_stream,
              gg_sim** out)
{
    g_create_error.clear();
    if (!out) { g_create_error = "out is NULL"; return GG_ERR_ARG; }
    *out = nullptr;
    std::string why;
    int rc = validate(grid, params, why);
    if (rc == GG_OK && (!theta || !lambda1 || !lambda2 || !u0 || !v0 || !w0)) {
        why = "a field pointer is NULL";
        rc = GG_ERR_ARG;
    }
    if (rc != GG_OK) { g_create_error = why; return rc; }

    gg_sim* s = new gg_sim();
    s->params = *params;
    if (s->params.cfl == 0.0) s->params.cfl = 0.9;
    s->nx = grid->nx;
    s->ny = grid->ny;
    s->lx = grid->lx > 0 ? grid->lx : 1.0;
    s->ly = grid->ly > 0 ? grid->ly : 1.0;
    s->dx = s->lx / s->nx;
    s->dy = s->ly / s->ny;
    s->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&s->device);
    const bool fp64 = s->params.precision == GG_FP64_PLAIN;
    const bool kahan = s->params.precision == GG_FP32_KAHAN;
    s->pitch = fp64 ? round_up(s->nx, 16) : round_up(s->nx, 32);
    const size_t n = (size_t)s->nx * s->ny;
    const size_t esz = fp64 ? 8 : 4;
    const size_t fbytes = (size_t)s->pitch * s->ny * esz;
    const size_t fstride = (fbytes + 255) / 256 * 256;
    const int nstate = kahan ? 6 : 3;
    const size_t dense_stride = (n * 8 + 255) / 256 * 256;
    const size_t diag_bytes = (size_t)kDiagBlocks * kDiagStride * 8 + 40 * 8;
    // arena: 2 x nstate state fields, 3 tensor fields, theta/l1/l2 (FP64 dense), diagnostics
    const size_t keep_tensor = fp64 ? 0 : 3;
    const size_t arena = fstride * (2 * nstate + 3) + dense_stride * keep_tensor + diag_bytes + 256;
    cudaError_t e = cudaMalloc(&s->arena, arena);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "device allocation of the simulation arena failed";
        delete s;
        return GG_ERR_OOM;
    }
    s->arena_bytes = arena;
    char* p = (char*)s->arena;
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < nstate; ++f) {
            if (fp64) s->f64[b][f] = (double*)p; else s->f32[b][f] = (float*)p;
            p += fstride;
        }
    for (int f = 0; f < 3; ++f) {
        if (fp64) s->a64[f] = (double*)p; else s->a32[f] = (float*)p;
        p += fstride;
    }
    for (size_t f = 0; f < keep_tensor; ++f) {
        s->tensor[f] = (double*)p;
        p += dense_stride;
    }
    s->diag_partials = (double*)p;
    p += (size_t)kDiagBlocks * kDiagStride * 8;
    s->diag_out = (double*)p;            // 16 doubles
    s->counters = (unsigned long long*)(s->diag_out + 16);  // [0] bad lambda, [1] nonfinite, [2] lmax bits
    // adaptive step words: Delta t_k (FP64), simulated time, Delta t_k (FP32), two maxima
    s->adapt.dt64 = s->diag_out + 32;
    s->adapt.t_done = s->diag_out + 33;
    s->adapt.dt32 = (float*)(s->diag_out + 34);
    s->adapt.kmax = (void*)(s->diag_out + 36);
    // Zero the whole arena once: padding columns and compensation terms start at 0.
    e = cudaMemsetAsync(s->arena, 0, arena, s->stream);
    if (e != cudaSuccess) { rc = cuda_fail(s, e, "memset"); g_create_error = s->last_error; gg_destroy(s); return rc; }

    // Stage the six host arrays on the device (dense FP64), then build the
    // tensor and the pitched state.
    double* staging = nullptr;
    // FP32 keeps theta/l1/l2 in the arena and stages a11 / a22 for the face weights
    const size_t nstage = fp64 ? 6 : 5;
    e = cudaMalloc(&staging, dense_stride * nstage);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "device allocation of the upload staging buffer failed";
        gg_destroy(s);
        return GG_ERR_OOM;
    }
    double* dth = fp64 ? staging : s->tensor[0];
    double* dl1 = fp64 ? (double*)((char*)staging + dense_stride) : s->tensor[1];
    double* dl2 = fp64 ? (double*)((char*)staging + 2 * dense_stride) : s->tensor[2];
    double* du0 = (double*)((char*)staging + (fp64 ? 3 : 0) * dense_stride);
    double* dv0 = (double*)((char*)du0 + dense_stride);
    double* dw0 = (double*)((char*)dv0 + dense_stride);
    const double* hsrc[6] = {theta, lambda1, lambda2, u0, v0, w0};
    double* ddst[6] = {dth, dl1, dl2, du0, dv0, dw0};
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(ddst[k], hsrc[k], n * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = launch_coefficients(dth, dl1, dl2, s->nx, s->ny, s->dx, s->dy, fp64 ? (void*)s->a64[0] : (void*)s->a32[0],
                                fp64 ? (void*)s->a64[1] : (void*)s->a32[1], fp64 ? (void*)s->a64[2] : (void*)s->a32[2],
                                s->pitch, fp64, fp64 ? nullptr : (double*)((char*)staging + 3 * dense_stride),
                                s->counters, s->counters + 2, s->stream);
    const double* dstate[3] = {du0, dv0, dw0};
    for (int f = 0; f < 3 && e == cudaSuccess; ++f)
        e = launch_unpack(dstate[f], true, fp64 ? (void*)s->f64[0][f] : (void*)s->f32[0][f], fp64, s->nx, s->ny,
                          s->pitch, s->counters + 1, s->stream);
    unsigned long long cnt[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, s->counters, sizeof cnt, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(staging);
    if (e != cudaSuccess) { rc = cuda_fail(s, e, "create"); g_create_error = s->last_error; gg_destroy(s); return rc; }
    if (cnt[0]) {
        char b[128];
        snprintf(b, sizeof b, "%llu cells with lambda <= 0 or non-finite theta/lambda", cnt[0]);
        g_create_error = b;
        gg_destroy(s);
        return GG_ERR_NOT_SPD;
    }
    if (cnt[1]) {
        char b[128];
        snprintf(b, sizeof b, "%llu non-finite initial values", cnt[1]);
        g_create_error = b;
        gg_destroy(s);
        return GG_ERR_ARG;
    }
    double lmax;
    memcpy(&lmax, &cnt[2], sizeof lmax);
    s->lambda_max = lmax;
    s->dt_max = stable_dt_max(s->dx, s->dy, lmax, s->params);
    if (s->params.adapt_every > 0) {
        // acid part of the rule; Delta t_0 from the initial state
        s->kW = 2.0 * lmax * (1.0 / (s->dx * s->dx) + 1.0 / (s->dy * s->dy)) +
                ((s->params.flags & GG_FLAG_NO_REACTION) ? 0.0 : s->params.c);
        s->since_adapt = 0;
        e = adapt_now(s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&s->dt, s->adapt.dt64, 8, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) { rc = cuda_fail(s, e, "adaptive step"); g_create_error = s->last_error; gg_destroy(s); return rc; }
    } else if (s->params.dt > 0.0) {
        if (s->params.dt > s->dt_max && !(s->params.flags & GG_FLAG_ALLOW_UNSTABLE)) {
            char b[160];
            snprintf(b, sizeof b, "dt = %.6g exceeds the stable bound %.6g", s->params.dt, s->dt_max);
            g_create_error = b;
            gg_destroy(s);
            return GG_ERR_CFL;
        }
        s->dt = s->params.dt;
    } else {
        s->dt = s->params.cfl * s->dt_max;
    }
    if (!fp64) {
        const int T = s->params.steps_per_pass > 0 ? s->params.steps_per_pass : 1;
        s->plan = default_plan(s->nx, s->ny, T);
        // steps_per_pass == 0: tuned (grids below 2^18 cells keep the default,
        // they finish in microseconds either way)
        if (s->params.steps_per_pass == 0 && (int64_t)s->nx * s->ny >= (int64_t)1 << 18) {
            s->plan = cached_plan(s);
            s->last_error.clear();
        }
    }
    *out = s;
    return GG_OK;
}

// Steps of the fixed-step path; with the adaptive step gg_step calls it for
// the stretches between recomputations of Delta t_k.
static cudaError_t run_steps(gg_sim* s, int64_t nsteps)
{
    cudaError_t e = cudaSuccess;
    if (s->params.precision == GG_FP64_PLAIN) {
        Rates64 r;
        r.dt_dev = s->params.adapt_every > 0 ? s->adapt.dt64 : nullptr;
        r.dt = s->dt; r.D = s->params.D; r.delta = s->params.delta; r.rho = s->params.rho; r.c = s->params.c;
        r.kx = 0.5 / (s->dx * s->dx); r.ky = 0.5 / (s->dy * s->dy); r.kc = 0.25 / (s->dx * s->dy);
        r.ihx2 = 1.0 / (s->dx * s->dx); r.ihy2 = 1.0 / (s->dy * s->dy);
        r.no_reaction = (s->params.flags & GG_FLAG_NO_REACTION) ? 1 : 0;
        for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
            Grid64 g;
            const int c = s->cur, nn = c ^ 1;
            g.u = s->f64[c][0]; g.v = s->f64[c][1]; g.w = s->f64[c][2];
            g.uo = s->f64[nn][0]; g.vo = s->f64[nn][1]; g.wo = s->f64[nn][2];
            g.a11 = s->a64[0]; g.a12 = s->a64[1]; g.a22 = s->a64[2];
            g.nx = s->nx; g.ny = s->ny; g.pitch = s->pitch;
            e = launch_step64(g, r, s->stream);
            if (e == cudaSuccess) { s->cur = nn; s->steps++; }
        }
    } else {
        const Rates32 r = rates32(s);
        const bool kahan = s->params.precision == GG_FP32_KAHAN;
        int64_t left = nsteps;
        while (left > 0 && e == cudaSuccess) {
            const int T = (int)std::min<int64_t>(left, s->plan.T);
            e = launch_plan(grid32(s, s->cur), r, s->plan, T, kahan, s->stream);
            if (e == cudaSuccess) { s->cur ^= 1; s->steps += T; left -= T; }
        }
    }
    return e;
}

int gg_step(gg_sim* s, int64_t nsteps)
{
    if (!s) return GG_ERR_ARG;
    if (nsteps < 0) { s->last_error = "nsteps < 0"; return GG_ERR_ARG; }
    cudaError_t e = cudaSuccess;
    if (s->params.adapt_every > 0) {
        // passes never straddle a recomputation of Delta t_k, so every plan
        // takes the same steps with the same Delta t_k
        const int64_t every = s->params.adapt_every;
        int64_t left = nsteps;
        while (left > 0 && e == cudaSuccess) {
            if (s->since_adapt == every) e = adapt_now(s);
            if (e != cudaSuccess) break;
            const int64_t n = std::min<int64_t>(left, every - s->since_adapt);
            e = run_steps(s, n);
            if (e == cudaSuccess) { s->since_adapt += n; left -= n; }
        }
    } else {
        e = run_steps(s, nsteps);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    return GG_OK;
}

double gg_dt(const gg_sim* s)
{
    if (!s) return 0.0;
    if (s->params.adapt_every <= 0) return s->dt;
    double dt = 0.0;
    if (cudaMemcpyAsync(&dt, s->adapt.dt64, 8, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return dt;
}

double gg_time(const gg_sim* s)
{
    if (!s) return 0.0;
    if (s->params.adapt_every <= 0) return (double)s->steps * s->dt;
    double w[2] = {0.0, 0.0};  // Delta t_k, time up to its recomputation
    if (cudaMemcpyAsync(w, s->adapt.dt64, 16, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return w[1] + w[0] * (double)s->since_adapt;
}
double gg_dt_max(const gg_sim* s) { return s ? s->dt_max : 0.0; }
int64_t gg_step_count(const gg_sim* s) { return s ? s->steps : 0; }
int32_t gg_steps_per_pass(const gg_sim* s) { return s ? (s->params.precision == GG_FP64_PLAIN ? 1 : s->plan.T) : 0; }

static void* field_ptr(gg_sim* s, int32_t field, bool& fp64)
{
    fp64 = s->params.precision == GG_FP64_PLAIN;
    const bool kahan = s->params.precision == GG_FP32_KAHAN;
    if (field >= GG_FIELD_U && field <= GG_FIELD_W)
        return fp64 ? (void*)s->f64[s->cur][field] : (void*)s->f32[s->cur][field];
    if (field >= GG_FIELD_COMP_U && field <= GG_FIELD_COMP_W) return kahan ? (void*)s->f32[s->cur][field] : nullptr;
    if (field >= GG_FIELD_A11 && field <= GG_FIELD_A22) {
        // FP32 simulations keep face weights, not the cell entries: gg_read
        // computes those from theta / lambda (field_ptr is not used for them)
        const int f = field - GG_FIELD_A11;
        return fp64 ? (void*)s->a64[f] : nullptr;
    }
    if (field >= GG_FIELD_FACE_X && field <= GG_FIELD_CROSS) {
        static const int slot[3] = {0, 2, 1};  // face_x -> ax, face_y -> ay, cross -> b
        return fp64 ? nullptr : (void*)s->a32[slot[field - GG_FIELD_FACE_X]];
    }
    return nullptr;
}

static int ensure_staging(gg_sim* s)
{
    if (s->staging) return GG_OK;
    const size_t bytes = (size_t)s->nx * s->ny * 8;
    cudaError_t e = cudaMalloc(&s->staging, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->staging = nullptr;
        s->last_error = "staging allocation failed";
        return GG_ERR_OOM;
    }
    return GG_OK;
}

int gg_read(gg_sim* s, int32_t field, void* dst, int32_t dst_on_device, int32_t dst_fp64)
{
    if (!s) return GG_ERR_ARG;
    if (!dst) { s->last_error = "dst is NULL"; return GG_ERR_ARG; }
    bool fp64;
    void* src = field_ptr(s, field, fp64);
    const bool cell_tensor = !fp64 && field >= GG_FIELD_A11 && field <= GG_FIELD_A22;
    if (!src && !cell_tensor) { s->last_error = "field not available for this precision"; return GG_ERR_ARG; }
    const size_t n = (size_t)s->nx * s->ny;
    const size_t bytes = n * (dst_fp64 ? 8 : 4);
    cudaError_t e;
    if (cell_tensor) {
        // the entries of eq. (2) in FP64 from theta / lambda, rounded to dst's type
        void* d = dst;
        if (!dst_on_device) {
            int rc = ensure_staging(s);
            if (rc) return rc;
            d = s->staging;
        }
        e = launch_tensor_entry(s->tensor[0], s->tensor[1], s->tensor[2], n, field - GG_FIELD_A11, d,
                                dst_fp64 != 0, s->stream);
        if (e == cudaSuccess && !dst_on_device)
            e = cudaMemcpyAsync(dst, s->staging, bytes, cudaMemcpyDeviceToHost, s->stream);
    } else if (dst_on_device) {
        e = launch_pack(src, fp64, dst, dst_fp64 != 0, s->nx, s->ny, s->pitch, s->stream);
    } else {
        int rc = ensure_staging(s);
        if (rc) return rc;
        e = launch_pack(src, fp64, s->staging, dst_fp64 != 0, s->nx, s->ny, s->pitch, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, s->staging, bytes, cudaMemcpyDeviceToHost, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "read");
    return GG_OK;
}

int gg_write(gg_sim* s, int32_t field, const void* src, int32_t src_on_device, int32_t src_fp64)
{
    if (!s) return GG_ERR_ARG;
    if (!src) { s->last_error = "src is NULL"; return GG_ERR_ARG; }
    if (field > GG_FIELD_COMP_W) { s->last_error = "tensor and coefficient fields are read-only"; return GG_ERR_ARG; }
    bool fp64;
    void* dstp = field_ptr(s, field, fp64);
    if (!dstp) { s->last_error = "field not available for this precision"; return GG_ERR_ARG; }
    const size_t n = (size_t)s->nx * s->ny;
    cudaError_t e = cudaSuccess;
    const void* dsrc = src;
    if (!src_on_device) {
        int rc = ensure_staging(s);
        if (rc) return rc;
        e = cudaMemcpyAsync(s->staging, src, n * (src_fp64 ? 8 : 4), cudaMemcpyHostToDevice, s->stream);
        dsrc = s->staging;
    }
    if (e == cudaSuccess) e = launch_unpack(dsrc, src_fp64 != 0, dstp, fp64, s->nx, s->ny, s->pitch, nullptr, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "write");
    return GG_OK;
}

int gg_diagnostics_eps(gg_sim* s, double eps, gg_diag* out)
{
    if (!s) return GG_ERR_ARG;
    if (!out || !(eps > 0.0) || !isfinite(eps)) { s->last_error = "out is NULL or eps <= 0"; return GG_ERR_ARG; }
    const bool fp64 = s->params.precision == GG_FP64_PLAIN;
    const void* f[3];
    for (int k = 0; k < 3; ++k) f[k] = fp64 ? (const void*)s->f64[s->cur][k] : (const void*)s->f32[s->cur][k];
    double h[12];
    cudaError_t e = launch_diagnostics(f[0], f[1], f[2], fp64, s->nx, s->ny, s->pitch, eps, s->diag_partials,
                                       s->diag_out, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, s->diag_out, sizeof h, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "diagnostics");
    const double cell = s->dx * s->dy;
    for (int k = 0; k < 3; ++k) {
        out->mass[k] = h[k] * cell;
        out->min[k] = h[3 + k];
        out->max[k] = h[6 + k];
    }
    out->nonfinite = (int64_t)h[9];
    out->tumour_area = h[10] * cell;
    out->gap_area = h[11] * cell;
    out->gap_eps = eps;
    if (out->nonfinite) {
        s->last_error = "state holds non-finite values";
        return GG_ERR_NONFINITE;
    }
    return GG_OK;
}

int gg_diagnostics(gg_sim* s, gg_diag* out) { return gg_diagnostics_eps(s, 0.01, out); }

int gg_autotune(gg_sim* s, int64_t trial_steps, int32_t* chosen)
{
    if (!s) return GG_ERR_ARG;
    if (s->params.precision == GG_FP64_PLAIN) {
        if (chosen) { chosen[0] = 1; chosen[1] = 0; chosen[2] = 0; chosen[3] = 0; }
        return GG_OK;
    }
    const Plan32 best = tune_plan(s, trial_steps);
    if (!s->last_error.empty() && s->last_error.rfind("autotune", 0) == 0) return GG_ERR_CUDA;
    s->plan = best;
    if (chosen) { chosen[0] = best.T; chosen[1] = best.kind; chosen[2] = best.bx; chosen[3] = best.by; }
    return GG_OK;
}

int gg_set_plan(gg_sim* s, int32_t kind, int32_t T, int32_t strip, int32_t chunk)
{
    if (!s) return GG_ERR_ARG;
    if (s->params.precision == GG_FP64_PLAIN) { s->last_error = "FP64 has a single plan"; return GG_ERR_STATE; }
    if (kind != 0 && kind != 1 && kind != 3) { s->last_error = "kind must be 0, 1 or 3"; return GG_ERR_ARG; }
    if (T < 1 || T > (kind != 0 ? 4 : kMaxT)) { s->last_error = "T out of range for this kernel"; return GG_ERR_ARG; }
    if (chunk < 0 || strip < 0 || chunk > (1 << 20) || strip > 1024) { s->last_error = "bad strip or chunk"; return GG_ERR_ARG; }
    Plan32 p = default_plan(s->nx, s->ny, kind != 0 ? T : kMaxT);
    p.kind = kind;
    p.T = T;
    p.halo = T;
    if (kind == 0) {
        if (strip > 0) p.bx = round_up(strip, 4);
        const int sw = p.bx + 2 * p.halo;
        if ((sw + p.threads - 1) / p.threads > 3) { s->last_error = "strip too wide"; return GG_ERR_ARG; }
    }
    if (chunk > 0) p.by = std::min(s->ny, chunk);
    if (kind != 0 && chunk == 0) p.by = default_plan(s->nx, s->ny, T).by;
    if (kind == 3) p.bx = stepw2_out_columns(T);
    if (kind == 1) p.bx = 32 - 2 * T;
    s->plan = p;
    return GG_OK;
}

int gg_plan_info(const gg_sim* s, int32_t* info)
{
    if (!s || !info) return GG_ERR_ARG;
    const bool fp64 = s->params.precision == GG_FP64_PLAIN;
    info[0] = fp64 ? 2 : s->plan.kind;
    info[1] = fp64 ? 1 : s->plan.T;
    info[2] = fp64 ? 32 : s->plan.bx;
    info[3] = fp64 ? 8 : s->plan.by;
    return GG_OK;
}

int gg_destroy(gg_sim* s)
{
    if (!s) return GG_OK;
    cudaStreamSynchronize(s->stream);
    gg_release_extras(s);
    if (s->staging) cudaFree(s->staging);
    if (s->arena) cudaFree(s->arena);
    delete s;
    return GG_OK;
}

}  // extern "C"
