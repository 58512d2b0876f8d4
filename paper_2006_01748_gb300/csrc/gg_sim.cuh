// The opaque simulation object behind gg_sim* (internal to libgg.so).
#pragma once

#include <string>

#include "gg_internal.cuh"

struct gg_sim {
    gg_params params{};
    int nx = 0, ny = 0, pitch = 0;   // pitch in elements (32 floats / 16 doubles)
    double lx = 1, ly = 1, dx = 0, dy = 0;
    double dt = 0, dt_max = 0, lambda_max = 0;
    int64_t steps = 0;
    int cur = 0;                     // ping-pong index of the current state
    int device = 0;
    cudaStream_t stream = nullptr;
    gg::Plan32 plan;

    // adaptive step (params.adapt_every > 0)
    int64_t since_adapt = 0;         // steps taken since Delta t_k was last recomputed
    double kW = 0;                   // static acid part of the rule
    gg::AdaptState adapt{};          // device words, inside the arena

    void* arena = nullptr;           // one allocation for state, tensor, diagnostics
    size_t arena_bytes = 0;
    float* f32[2][6] = {};           // [buffer][u, v, w, cu, cv, cw]
    double* f64[2][3] = {};          // [buffer][u, v, w]
    float* a32[3] = {};              // a11, a12, a22 (pitched)
    double* a64[3] = {};
    double* tensor[3] = {};          // theta, lambda1, lambda2 (dense FP64, FP32 sims only)
    double* diag_partials = nullptr;
    double* diag_out = nullptr;
    unsigned long long* counters = nullptr;
    void* staging = nullptr;         // dense nx*ny*8 bytes, allocated on first use

    void* adj = nullptr;             // adjoint workspace (gg_adjoint.cu)
    std::string last_error;
};

namespace gg {
void set_error(gg_sim* s, const char* fmt, const char* detail);
int cuda_fail(gg_sim* s, cudaError_t e, const char* where);
Rates32 rates32(const gg_sim* s);
Grid32 grid32(const gg_sim* s, int cur);
Plan32 default_plan(int nx, int ny, int T);
double stable_dt_max(double dx, double dy, double Lambda, const gg_params& p);
Plan32 tune_plan(gg_sim* s, int64_t trial_steps);
// Recomputes Delta t_k from the current state (adaptive step), adding
// since_adapt steps of the previous Delta t to the simulated time.
cudaError_t adapt_now(gg_sim* s);
}  // namespace gg

// Frees workspaces owned by other translation units (adjoint).
void gg_release_extras(gg_sim* s);
