// Ensembles of independent grids (placeholder until the persistent kernel lands).
#include "gg_sim.cuh"

struct gg_batch {
    std::string last_error;
};

extern "C" {

int gg_batch_create(int32_t n, const gg_grid* grids, const gg_params* params, const double* const* fields,
                    void* cuda_stream, gg_batch** out)
{
    (void)n; (void)grids; (void)params; (void)fields; (void)cuda_stream;
    if (out) *out = nullptr;
    return GG_ERR_STATE;
}
int gg_batch_step(gg_batch* b, int64_t nsteps) { (void)b; (void)nsteps; return GG_ERR_STATE; }
int gg_batch_read(gg_batch* b, int32_t inst, int32_t field, void* dst, int32_t on_dev, int32_t fp64)
{
    (void)b; (void)inst; (void)field; (void)dst; (void)on_dev; (void)fp64;
    return GG_ERR_STATE;
}
int gg_batch_diagnostics(gg_batch* b, int32_t inst, gg_diag* out) { (void)b; (void)inst; (void)out; return GG_ERR_STATE; }
double gg_batch_dt(const gg_batch* b, int32_t inst) { (void)b; (void)inst; return 0.0; }
const char* gg_batch_last_error(const gg_batch* b) { return b ? b->last_error.c_str() : ""; }
int gg_batch_destroy(gg_batch* b) { delete b; return GG_OK; }

}  // extern "C"
