// Discrete adjoint of the FP32 step of eq. (3) with sqrt(N) checkpointing.
//
// One step is X' = X + dt F(X; a11, a12, a22, delta, rho, D, c).  Its
// adjoint maps lam' = dL/dX' to lam = lam' + dt J(X)^T lam' and adds
// dt (dF/dp)^T lam' to the parameter gradients.  The kernel below evaluates
// J^T in gather form (each thread produces its own cell, no atomics):
//
//   lamU <- lamU + dt [ (1 - 2U - delta W) lamU
//                       + D/2 sum_faces (V_nb - V)(lamV_nb - lamV)/h^2 ]
//   lamV <- lamV + dt [ rho (1 - 2V) lamV + D D1(lamV; U) + c lamW ]
//   lamW <- lamW + dt [ -delta U lamU - c lamW + D2^T lamW ]
//
// D1 of Table 1 is symmetric in V for fixed U.  D2 of Table 2 is symmetric
// in the interior but not next to the boundary, where the mirror ghosts of
// the tangential differences enter; its transpose is written from the face
// fluxes: with Lx(f) = lamW_left - lamW_right on interior x-faces (0 on
// boundary faces) and Sx_ij = kc a12_ij (Lx(i+1/2,j) + Lx(i-1/2,j)),
//   D2^T lamW = sum_faces coef (lamW_nb - lamW)
//             + Ty(Sx) + Tx(Sy),
//   Ty(S)_j = S_{j-1}[j>=1] - S_{j+1}[j<=ny-2] + S_j([j=ny-1] - [j=0])
// (the transpose of the mirrored central difference), and the same in x.
// Parameter gradients per cell:
//   g_a11 += dt kx [ (W_E - W) Lx_E + (W - W_W) Lx_W ]
//   g_a22 += dt ky [ (W_N - W) Ly_N + (W - W_S) Ly_S ]
//   g_a12 += dt kc [ (Lx_E + Lx_W)(W_N - W_S) + (Ly_N + Ly_S)(W_E - W_W) ]
// and the four rate gradients are FP64 block partials (deterministic order).
// dt is a fixed input: its dependence on the tensor and the rates is not
// differentiated.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "gg_adjoint2.cuh"
#include "gg_sim.cuh"

using namespace gg;

namespace {

// Geometry of the warp-marching adjoint launches.  A grid of strips x chunks
// warps runs in waves of `cap` resident warps (152 SMs times the warps an SM
// holds).  The chunk height is chosen so that the grid fills a whole number
// of waves where it can: a grid of one wave plus a few CTAs takes about two
// warp lifetimes.
inline int wave_chunk(int strips, int ny, int cap, int hmax)
{
    constexpr int hmin = 8;
    if (strips > cap) return std::min(hmax, std::max(hmin, ny));
    const int per_wave = cap / strips;  // chunk rows of warps per wave
    const int waves = std::max(1, (ny + per_wave * hmax - 1) / (per_wave * hmax));
    const int nch = waves * per_wave;
    return std::min(hmax, std::max(hmin, (ny + nch - 1) / nch));
}
constexpr int kFlushEvery = 64;  // FP32 per-cell gradient sums are folded into FP64 this often

// The reverse passes (gg_adjoint2.cuh): paired columns, 64-column strips (60
// columns written by the one-step pass, 56 by the two-step pass), one warp per
// CTA with its shared-memory ring.
extern __shared__ float2 g_adj_ring[];

// The two-step pass carries three levels (the rebuilt forward step and two
// reverse steps) in about 200 registers: two warps on each of the SM's four
// schedulers (a scheduler's register file holds 16384 registers, so a third
// warp needs 170 or fewer).  Measured, a cap of 168 registers (three warps a
// scheduler) spilled and ran 1.8x slower, and passing the carried rows
// through shared memory instead (166 registers, twelve warps per SM) made the
// pass bound by shared-memory traffic and 23 % slower.
template <int STEPS, bool KAHAN>
__global__ void __launch_bounds__(32) adjw_kernel(const adjw::PassArgs a, const Rates32 k, const int H, const int nstrips,
                                             const int nwarps)
{
    const int gw = blockIdx.x;
    if (gw >= nwarps) return;
    chained_wait();  // launched with launch_chained
    const int strip = gw % nstrips, chunk = gw / nstrips;
    const int x0 = strip * adjw::Geom<STEPS>::OUT - adjw::Geom<STEPS>::HLP;
    const int ys = chunk * H;
    double* part = a.partials + (size_t)gw * 4;
    // interior chunks: every row the march touches (from five rows above the
    // chunk to three below) has a south and a north face
    const bool yin = ys - 5 >= 1 && ys + H + 3 <= a.ny - 1;
    if (x0 >= 1 && x0 + 63 <= a.nx - 2) {
        if (yin) adjw::march<STEPS, KAHAN, false, false>(a, k, H, strip, chunk, threadIdx.x, g_adj_ring, part);
        else adjw::march<STEPS, KAHAN, false, true>(a, k, H, strip, chunk, threadIdx.x, g_adj_ring, part);
    } else {
        adjw::march<STEPS, KAHAN, true, true>(a, k, H, strip, chunk, threadIdx.x, g_adj_ring, part);
    }
}

template <int STEPS> inline int adjw_strips(int nx)
{
    return (nx + adjw::Geom<STEPS>::OUT - 1) / adjw::Geom<STEPS>::OUT;
}

// Resident warps of one wave of adjw_kernel<STEPS, KAHAN> (16 per SM if the
// occupancy query fails).
template <int STEPS, bool KAHAN>
int adjw_wave()
{
    int dev = 0, sms = 152, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjw_kernel<STEPS, KAHAN>, 32, adjw::kRingBytes) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return 16 * 152;
    }
    return per_sm * sms;
}

struct AdjGeom {
    int H, strips, warps;
};
template <int STEPS, bool KAHAN>
AdjGeom adjw_geom(int nx, int ny)
{
    AdjGeom g;
    g.strips = adjw_strips<STEPS>(nx);
    g.H = wave_chunk(g.strips, ny, adjw_wave<STEPS, KAHAN>(), 128);
    g.warps = g.strips * ((ny + g.H - 1) / g.H);
    return g;
}
AdjGeom adj_geom(int steps, bool kahan, int nx, int ny)
{
    if (steps == 1) return kahan ? adjw_geom<1, true>(nx, ny) : adjw_geom<1, false>(nx, ny);
    return kahan ? adjw_geom<2, true>(nx, ny) : adjw_geom<2, false>(nx, ny);
}

// g64 += g32; g32 = 0 for the 3 fields, over the whole pitched area in
// groups of 4 (the pitch is a multiple of 32 cells and the padding columns
// hold zeros, which the reverse passes never write).
__device__ __forceinline__ void flush4(float* g, double* h, size_t q)
{
    const float4 a = reinterpret_cast<const float4*>(g)[q];
    double2* hp = reinterpret_cast<double2*>(h) + 2 * q;
    double2 h0 = hp[0], h1 = hp[1];
    h0.x += (double)a.x; h0.y += (double)a.y; h1.x += (double)a.z; h1.y += (double)a.w;
    hp[0] = h0; hp[1] = h1;
    reinterpret_cast<float4*>(g)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}
__global__ void flush_kernel(float* g1, float* g2, float* g3, double* h1, double* h2, double* h3, size_t n4)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (size_t)gridDim.x * blockDim.x) {
        flush4(g1, h1, q);
        flush4(g2, h2, q);
        flush4(g3, h3, q);
    }
}

// dL/d(theta, l1, l2) from dL/d(a11, a12, a22) through eq. (2); FP32 outputs
// in the dense host layout (null outputs are skipped).
__global__ void chain_rule_kernel(const double* g11, const double* g12, const double* g22, int pitch,
                                  const double* theta, const double* l1, const double* l2, int nx, int ny,
                                  float* gth, float* gl1, float* gl2)
{
    const size_t n = (size_t)nx * ny;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / nx), i = (int)(q % nx);
        const size_t o = (size_t)j * pitch + i;
        double s, c;
        sincos(theta[q], &s, &c);
        const double d = l1[q] - l2[q];
        const double G11 = g11[o], G12 = g12[o], G22 = g22[o];
        if (gth) gth[q] = (float)(G11 * (-2.0 * d * s * c) + G12 * (d * (c * c - s * s)) + G22 * (2.0 * d * s * c));
        if (gl1) gl1[q] = (float)(G11 * c * c + G12 * s * c + G22 * s * s);
        if (gl2) gl2[q] = (float)(G11 * s * s - G12 * s * c + G22 * c * c);
    }
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

struct AdjWork {
    size_t bytes = 0;
    void* base = nullptr;
    int K = 0, nseg = 0, nstate = 0;
    std::vector<float*> ckpt;     // nseg x nstate fields
    std::vector<float*> stash;    // (K - 1) / 2 states of 3 fields: the even offsets 2, 4, .. of a segment
    float* scratch[3] = {};       // one state: the odd pass boundaries of a recomputation
    float* scomp[2][3] = {};      // Kahan terms of the recomputed states
    float* lam[2][6] = {};        // lam and its Kahan terms, ping-pong
    float* g32[3] = {};
    double* g64[3] = {};
    double* partials = nullptr;
    int nblocks = 0;
    // states of the trailing segments kept from the forward pass (no recompute)
    void* big = nullptr;
    size_t big_bytes = 0;
};

}  // namespace

void gg_release_extras(gg_sim* s)
{
    if (s && s->adj) {
        AdjWork* w = (AdjWork*)s->adj;
        if (w->base) cudaFree(w->base);
        if (w->big) cudaFree(w->big);
        delete w;
        s->adj = nullptr;
    }
}

extern "C" int gg_adjoint_release(gg_sim* s)
{
    if (!s) return GG_ERR_ARG;
    gg_release_extras(s);
    return GG_OK;
}

static int adj_workspace(gg_sim* s, int K, int nseg, bool kahan, AdjWork** out)
{
    const size_t fb = ((size_t)s->pitch * s->ny * 4 + 255) / 256 * 256;
    const size_t db = ((size_t)s->pitch * s->ny * 8 + 255) / 256 * 256;
    const int nstate = kahan ? 6 : 3;
    // one FP64 record of rate gradients per warp of the larger of the two adjoint launches
    const int nblocks = std::max(adj_geom(1, kahan, s->nx, s->ny).warps, adj_geom(2, kahan, s->nx, s->ny).warps);
    const size_t need = fb * ((size_t)nseg * nstate + (size_t)((K - 1) / 2) * 3 + 3 + 6 + 12 + 3) + db * 3 +
                        (((size_t)nblocks * 4 * 8 + 255) / 256 * 256);
    AdjWork* w = (AdjWork*)s->adj;
    if (w && w->bytes >= need && w->nstate == nstate) {
        // reuse: just re-carve for the new K / nseg
    } else {
        gg_release_extras(s);
        w = new AdjWork();
        cudaError_t e = cudaMalloc(&w->base, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete w;
            s->last_error = "adjoint workspace allocation failed (checkpoints + recompute stash)";
            return GG_ERR_OOM;
        }
        w->bytes = need;
        s->adj = w;
    }
    w->K = K;
    w->nseg = nseg;
    w->nstate = nstate;
    w->nblocks = nblocks;
    char* p = (char*)w->base;
    w->ckpt.assign((size_t)nseg * nstate, nullptr);
    for (auto& f : w->ckpt) { f = (float*)p; p += fb; }
    w->stash.assign((size_t)((K - 1) / 2) * 3, nullptr);
    for (auto& f : w->stash) { f = (float*)p; p += fb; }
    for (int f = 0; f < 3; ++f) { w->scratch[f] = (float*)p; p += fb; }
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < 3; ++f) { w->scomp[b][f] = (float*)p; p += fb; }
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < 6; ++f) { w->lam[b][f] = (float*)p; p += fb; }
    for (int f = 0; f < 3; ++f) { w->g32[f] = (float*)p; p += fb; }
    for (int f = 0; f < 3; ++f) { w->g64[f] = (double*)p; p += db; }
    w->partials = (double*)p;
    *out = w;
    return GG_OK;
}

extern "C" int gg_adjoint(gg_sim* s, int64_t nsteps, const float* dLdu_N, const float* dLdv_N, const float* dLdw_N,
                          float* g_theta, float* g_lambda1, float* g_lambda2, float* g_u0, float* g_v0, float* g_w0,
                          double* g_scalars, int64_t checkpoint_every)
{
    if (!s) return GG_ERR_ARG;
    if (nsteps < 0 || checkpoint_every < 0) { s->last_error = "nsteps and checkpoint_every must be >= 0"; return GG_ERR_ARG; }
    if (s->params.precision == GG_FP64_PLAIN) {
        s->last_error = "the adjoint is provided for the FP32 precisions";
        return GG_ERR_STATE;
    }
    if (s->params.adapt_every > 0) {
        s->last_error = "the adjoint holds dt fixed: not available with the adaptive step";
        return GG_ERR_STATE;
    }
    const bool kahan = s->params.precision == GG_FP32_KAHAN;
    const int64_t N = nsteps;
    int K = (int)(checkpoint_every > 0 ? checkpoint_every : (int64_t)ceil(sqrt((double)std::max<int64_t>(N, 1))));
    K = std::max(1, (int)std::min<int64_t>(K, std::max<int64_t>(N, 1)));
    const int nseg = (int)((N + K - 1) / K);
    AdjWork* w = nullptr;
    int rc = adj_workspace(s, K, std::max(nseg, 1), kahan, &w);
    if (rc != GG_OK) return rc;
    cudaStream_t st = s->stream;
    const size_t fbytes = (size_t)s->pitch * s->ny * 4;
    const size_t dbytes = (size_t)s->pitch * s->ny * 8;
    const int nstate = w->nstate;
    cudaError_t e = cudaSuccess;

    const Rates32 r = rates32(s);
    // Passes that also write the intermediate states (the kept segments'
    // forward and the recomputation of the others) run the paired-column
    // kernel with the simulation's depth and chunk height (at 2048^2 the tuned
    // T = 3 with 42-row chunks took 21.6 us per step with the stash writes,
    // four steps deep in whole waves 24.2 us), T = 3 when the plan is not a
    // warp plan.  Every plan gives the same bits, so these states are exactly
    // those of the simulation's own plan.
    const bool warp_plan = s->plan.kind == 1 || s->plan.kind == 3;
    const int TR = warp_plan ? s->plan.T : 3;
    const int HR = warp_plan ? s->plan.by : default_plan(s->nx, s->ny, 3).by;
    // Runs nsteps steps from the state `in` (u, v, w, cu, cv, cw) in passes of
    // up to TR steps.  Only the states at even steps are stored: the state
    // after an even step kk (2 <= kk < nsteps, and nsteps itself when fin is
    // null) is written to slot(kk) (u, v, w); a pass boundary at an odd step
    // goes through the scratch state, and an intermediate level at an odd step
    // writes nothing.  The last state goes to fin (u, v, w and Kahan terms)
    // when fin is given.  Kahan terms between passes alternate between the two
    // scomp buffers.
    auto passes = [&](float* const in[6], int nsteps, auto slot, float* const* fin) -> cudaError_t {
        auto place = [&](int kk) -> float* const* { return (kk & 1) ? w->scratch : slot(kk); };
        int kk = 0, pass = 0;
        cudaError_t ee = cudaSuccess;
        while (kk < nsteps && ee == cudaSuccess) {
            const int Tp = std::min(TR, nsteps - kk);
            const bool last = kk + Tp == nsteps && fin;
            Grid32 g;
            if (kk == 0) { g.u = in[0]; g.v = in[1]; g.w = in[2]; }
            else { float* const* x = place(kk); g.u = x[0]; g.v = x[1]; g.w = x[2]; }
            g.cu = kahan ? (kk == 0 ? in[3] : w->scomp[pass & 1][0]) : nullptr;
            g.cv = kahan ? (kk == 0 ? in[4] : w->scomp[pass & 1][1]) : nullptr;
            g.cw = kahan ? (kk == 0 ? in[5] : w->scomp[pass & 1][2]) : nullptr;
            if (last) {
                g.uo = fin[0]; g.vo = fin[1]; g.wo = fin[2];
                g.cuo = kahan ? fin[3] : nullptr; g.cvo = kahan ? fin[4] : nullptr; g.cwo = kahan ? fin[5] : nullptr;
            } else {
                float* const* x = place(kk + Tp);
                g.uo = x[0]; g.vo = x[1]; g.wo = x[2];
                g.cuo = kahan ? w->scomp[(pass + 1) & 1][0] : nullptr;
                g.cvo = kahan ? w->scomp[(pass + 1) & 1][1] : nullptr;
                g.cwo = kahan ? w->scomp[(pass + 1) & 1][2] : nullptr;
            }
            g.ax = s->a32[0]; g.b = s->a32[1]; g.ay = s->a32[2];
            g.nx = s->nx; g.ny = s->ny; g.pitch = s->pitch;
            Stash32 sh = {};
            for (int t = 1; t < Tp; ++t) {
                if ((kk + t) & 1) continue;  // odd steps are rebuilt by the reverse pass
                float* const* x = slot(kk + t);
                sh.u[t - 1] = x[0]; sh.v[t - 1] = x[1]; sh.w[t - 1] = x[2];
            }
            ee = launch_stepw2_stash(g, r, HR, Tp, kahan, sh, st);
            kk += Tp;
            ++pass;
        }
        return ee;
    };

    // Trailing segments whose states fit in 85 % of the free device memory are
    // kept from the forward pass and need no recomputation.
    int ns = 0;
    {
        size_t freeb = 0, totalb = 0;
        if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) { cudaGetLastError(); freeb = 0; }
        const size_t per_seg = (size_t)((K - 1) / 2) * 3 * ((fbytes + 255) / 256 * 256);
        const size_t have = w->big_bytes;
        // 85 % of (what this workspace already holds + what is free): the same
        // budget on every call, so a second call reuses the first call's buffer
        const size_t budget = (have + freeb) / 20 * 17;
        ns = (int)std::min<size_t>((size_t)nseg, per_seg ? budget / per_seg : 0);
        const size_t need = (size_t)ns * per_seg;
        if (ns > 0 && need > have) {
            if (w->big) cudaFree(w->big);
            w->big = nullptr;
            w->big_bytes = 0;
            if (cudaMalloc(&w->big, need) != cudaSuccess) {
                cudaGetLastError();
                w->big = nullptr;
                ns = 0;
            } else {
                w->big_bytes = need;
            }
        }
    }
    const int seg_kept = nseg - ns;  // segments >= seg_kept are stored, not recomputed
    const size_t fstride = (fbytes + 255) / 256 * 256;
    // the kept state at the even step kk >= 2 of segment seg
    const int per_seg_states = (K - 1) / 2;
    auto big_slot = [&](int seg, int kk, float** out3) {
        char* b = (char*)w->big + ((size_t)(seg - seg_kept) * per_seg_states + (kk / 2 - 1)) * 3 * fstride;
        out3[0] = (float*)b; out3[1] = (float*)(b + fstride); out3[2] = (float*)(b + 2 * fstride);
    };

    // 1. forward pass, storing the state at the start of every segment (with
    // its Kahan terms where the segment is recomputed from it) and the states
    // at even steps of the trailing segments
    for (int seg = 0; seg < nseg && e == cudaSuccess; ++seg) {
        const int nf = seg < seg_kept ? nstate : 3;
        for (int f = 0; f < nf && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(w->ckpt[(size_t)seg * nstate + f], s->f32[s->cur][f], fbytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) break;
        const int64_t len = std::min<int64_t>(K, N - (int64_t)seg * K);
        if (seg < seg_kept) {
            rc = gg_step(s, len);
            if (rc != GG_OK) return rc;
        } else {
            float* in[6] = {s->f32[s->cur][0], s->f32[s->cur][1], s->f32[s->cur][2],
                            kahan ? s->f32[s->cur][3] : nullptr, kahan ? s->f32[s->cur][4] : nullptr,
                            kahan ? s->f32[s->cur][5] : nullptr};
            const int o = s->cur ^ 1;
            float* fin[6] = {s->f32[o][0], s->f32[o][1], s->f32[o][2], kahan ? s->f32[o][3] : nullptr,
                             kahan ? s->f32[o][4] : nullptr, kahan ? s->f32[o][5] : nullptr};
            float* tmp[3];
            auto slot = [&](int kk) -> float* const* {
                big_slot(seg, kk, tmp);
                return tmp;
            };
            e = passes(in, (int)len, slot, fin);
            if (e == cudaSuccess) { s->cur ^= 1; s->steps += len; }
        }
    }
    // 2. lam^N = dL/dX^N (zero when not given); Kahan terms and gradient sums start at 0
    const float* dl[3] = {dLdu_N, dLdv_N, dLdw_N};
    for (int f = 0; f < 6 && e == cudaSuccess; ++f) e = cudaMemsetAsync(w->lam[0][f], 0, fbytes, st);
    for (int f = 0; f < 3 && e == cudaSuccess; ++f)
        if (dl[f]) e = launch_unpack(dl[f], false, w->lam[0][f], false, s->nx, s->ny, s->pitch, nullptr, st);
    for (int f = 0; f < 3 && e == cudaSuccess; ++f) e = cudaMemsetAsync(w->g32[f], 0, fbytes, st);
    for (int f = 0; f < 3 && e == cudaSuccess; ++f) e = cudaMemsetAsync(w->g64[f], 0, dbytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->partials, 0, (size_t)w->nblocks * 4 * 8, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "adjoint setup");

    const AdjGeom g1 = adj_geom(1, kahan, s->nx, s->ny), g2 = adj_geom(2, kahan, s->nx, s->ny);
    int lb = 0;          // current lam buffer
    int since_flush = 0;
    auto flush = [&]() {
        const size_t n4 = (size_t)s->pitch * s->ny / 4;
        flush_kernel<<<blocks_for(n4), 256, 0, st>>>(w->g32[0], w->g32[1], w->g32[2], w->g64[0], w->g64[1], w->g64[2],
                                                     n4);
        since_flush = 0;
        return cudaGetLastError();
    };
    // 3. segments in reverse: recompute the states of the segment, then run its adjoint steps
    for (int seg = nseg - 1; seg >= 0 && e == cudaSuccess; --seg) {
        const int len = (int)std::min<int64_t>(K, N - (int64_t)seg * K);
        const bool kept = seg >= seg_kept;
        auto state = [&](int kk, int f) -> float* {  // u, v, w of X^{seg*K + kk}, kk even
            if (kk == 0) return w->ckpt[(size_t)seg * nstate + f];
            if (kept) {
                float* x[3];
                big_slot(seg, kk, x);
                return x[f];
            }
            return w->stash[(size_t)(kk / 2 - 1) * 3 + f];
        };
        if (!kept && len > 2) {
            // recompute X^{seg K + 2, + 4 .. < seg K + len} into the stash
            float* in[6] = {state(0, 0), state(0, 1), state(0, 2),
                            kahan ? w->ckpt[(size_t)seg * nstate + 3] : nullptr,
                            kahan ? w->ckpt[(size_t)seg * nstate + 4] : nullptr,
                            kahan ? w->ckpt[(size_t)seg * nstate + 5] : nullptr};
            float* tmp[3];
            auto slot = [&](int kk) -> float* const* {
                tmp[0] = w->stash[(size_t)(kk / 2 - 1) * 3 + 0];
                tmp[1] = w->stash[(size_t)(kk / 2 - 1) * 3 + 1];
                tmp[2] = w->stash[(size_t)(kk / 2 - 1) * 3 + 2];
                return tmp;
            };
            e = passes(in, len - 1, slot, nullptr);
        }
        // reverse sweep of the segment: an odd first step alone (from the
        // stored state at the even step len - 1), then pairs of steps
        // (kk, kk - 1), kk odd, in one pass from the stored state kk - 1
        int kr = len - 1;
        // one reverse pass from the stored state k0 (even): lam[lb] -> lam[lb ^ 1]
        auto pass_args = [&](int k0) {
            adjw::PassArgs a;
            a.u = state(k0, 0); a.v = state(k0, 1); a.w = state(k0, 2);
            a.lu = w->lam[lb][0]; a.lv = w->lam[lb][1]; a.lw = w->lam[lb][2];
            a.clu = w->lam[lb][3]; a.clv = w->lam[lb][4]; a.clw = w->lam[lb][5];
            a.luo = w->lam[lb ^ 1][0]; a.lvo = w->lam[lb ^ 1][1]; a.lwo = w->lam[lb ^ 1][2];
            a.cluo = w->lam[lb ^ 1][3]; a.clvo = w->lam[lb ^ 1][4]; a.clwo = w->lam[lb ^ 1][5];
            a.ax = s->a32[0]; a.b = s->a32[1]; a.ay = s->a32[2];
            a.g11 = w->g32[0]; a.g12 = w->g32[1]; a.g22 = w->g32[2];
            a.partials = w->partials;
            a.nx = s->nx; a.ny = s->ny; a.pitch = s->pitch;
            return a;
        };
        auto single = [&](int k1) {
            const adjw::PassArgs a = pass_args(k1);
            const cudaError_t le =
                kahan ? launch_chained(adjw_kernel<1, true>, g1.warps, 32, adjw::kRingBytes, st, a, r, g1.H, g1.strips,
                                       g1.warps)
                      : launch_chained(adjw_kernel<1, false>, g1.warps, 32, adjw::kRingBytes, st, a, r, g1.H, g1.strips,
                                       g1.warps);
            lb ^= 1;
            since_flush += 1;
            return le;
        };
        auto pair = [&](int k1) {  // steps k1 and k1 - 1
            const adjw::PassArgs a = pass_args(k1 - 1);
            const cudaError_t le =
                kahan ? launch_chained(adjw_kernel<2, true>, g2.warps, 32, adjw::kRingBytes, st, a, r, g2.H, g2.strips,
                                       g2.warps)
                      : launch_chained(adjw_kernel<2, false>, g2.warps, 32, adjw::kRingBytes, st, a, r, g2.H, g2.strips,
                                       g2.warps);
            lb ^= 1;
            since_flush += 2;
            return le;
        };
        if ((len & 1) && e == cudaSuccess) {
            e = single(kr);
            --kr;
        }
        for (; kr >= 1 && e == cudaSuccess; kr -= 2) {
            e = pair(kr);
            if (e == cudaSuccess && since_flush >= kFlushEvery) e = flush();
        }
    }
    if (e == cudaSuccess && since_flush) e = flush();
    if (e != cudaSuccess) return cuda_fail(s, e, "adjoint");

    // 4. outputs
    if (g_theta || g_lambda1 || g_lambda2) {
        chain_rule_kernel<<<blocks_for((size_t)s->nx * s->ny), 256, 0, st>>>(
            w->g64[0], w->g64[1], w->g64[2], s->pitch, s->tensor[0], s->tensor[1], s->tensor[2], s->nx, s->ny,
            g_theta, g_lambda1, g_lambda2);
        e = cudaGetLastError();
    }
    float* g0[3] = {g_u0, g_v0, g_w0};
    for (int f = 0; f < 3 && e == cudaSuccess; ++f)
        if (g0[f]) e = launch_pack(w->lam[lb][f], false, g0[f], false, s->nx, s->ny, s->pitch, st);
    std::vector<double> hp;
    if (e == cudaSuccess && g_scalars) {
        hp.resize((size_t)w->nblocks * 4);
        e = cudaMemcpyAsync(hp.data(), w->partials, hp.size() * 8, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(s, e, "adjoint outputs");
    if (g_scalars) {
        for (int q = 0; q < 4; ++q) g_scalars[q] = 0.0;
        for (int b = 0; b < w->nblocks; ++b)
            for (int q = 0; q < 4; ++q) g_scalars[q] += hp[(size_t)b * 4 + q];
    }
    return GG_OK;
}
