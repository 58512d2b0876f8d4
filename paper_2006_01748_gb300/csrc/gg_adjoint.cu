// Discrete adjoint of eq. (3) (placeholder until the adjoint kernels land).
#include "gg_sim.cuh"

void gg_release_extras(gg_sim* s) { (void)s; }

extern "C" int gg_adjoint(gg_sim* s, int64_t nsteps, const float* dLdu_N, const float* dLdv_N, const float* dLdw_N,
                          float* g_theta, float* g_lambda1, float* g_lambda2, float* g_u0, float* g_v0, float* g_w0,
                          double* g_scalars, int64_t checkpoint_every)
{
    (void)nsteps; (void)dLdu_N; (void)dLdv_N; (void)dLdw_N; (void)g_theta; (void)g_lambda1; (void)g_lambda2;
    (void)g_u0; (void)g_v0; (void)g_w0; (void)g_scalars; (void)checkpoint_every;
    if (!s) return GG_ERR_ARG;
    s->last_error = "adjoint not available in this build";
    return GG_ERR_STATE;
}
