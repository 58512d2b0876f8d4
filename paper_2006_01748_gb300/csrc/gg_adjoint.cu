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

#include "gg_sim.cuh"

using namespace gg;

namespace {

constexpr int kAdjBX = 32, kAdjBY = 8;
constexpr int kFlushEvery = 16;  // FP32 per-cell gradient sums are folded into FP64 this often

struct AdjArgs {
    const float *u, *v, *w;                          // X^k
    const float *lu, *lv, *lw, *clu, *clv, *clw;     // lam^{k+1} and its Kahan terms
    float *luo, *lvo, *lwo, *cluo, *clvo, *clwo;     // lam^k
    const float *a11, *a12, *a22;
    float *g11, *g12, *g22;                          // FP32 per-cell sums (in place)
    double* partials;                                // [blocks][4]: delta, rho, D, c
    int nx, ny, pitch;
};

__device__ __forceinline__ void kahan_add(float x, float inc, float comp, float& xo, float& compo)
{
    const float y = __fsub_rn(inc, comp);
    const float t = __fadd_rn(x, y);
    compo = __fsub_rn(__fsub_rn(t, x), y);
    xo = t;
}

template <bool KAHAN>
__global__ void __launch_bounds__(kAdjBX* kAdjBY) adjoint_step_kernel(const AdjArgs a, const Rates32 k)
{
    const int i = blockIdx.x * kAdjBX + threadIdx.x;
    const int j = blockIdx.y * kAdjBY + threadIdx.y;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    double s_delta = 0.0, s_rho = 0.0, s_D = 0.0, s_c = 0.0;
    if (i < nx && j < ny) {
        const bool hasW = i > 0, hasE = i + 1 < nx, hasS = j > 0, hasN = j + 1 < ny;
        const int iw = hasW ? i - 1 : i, ie = hasE ? i + 1 : i;
        const int js = hasS ? j - 1 : j, jn = hasN ? j + 1 : j;
#define L(f, x, y) __ldg((f) + (size_t)(y) * pitch + (x))
        // lamW on the 3x3 neighbourhood (mirrored at the boundary).  With Kahan
        // terms the stored value x and its compensation c represent x - c, so
        // differences are taken as (x_a - x_b) - (c_a - c_b): the first part is
        // exact for nearby values and the second restores the low-order bits
        // that plain FP32 differences of a large smooth lam would lose.
        auto cw = [&](int x, int y) { return KAHAN ? L(a.clw, x, y) : 0.0f; };
        const float lwP0 = L(a.lw, i, j), cwP = cw(i, j);
        auto rel = [&](int x, int y) { return (L(a.lw, x, y) - lwP0) - (cw(x, y) - cwP); };
        // lamW relative to the centre cell: lwP = 0, neighbours carry the differences
        const float lwP = 0.0f, lwE = rel(ie, j), lwW = rel(iw, j);
        const float lwN = rel(i, jn), lwS = rel(i, js);
        const float lwNE = rel(ie, jn), lwNW = rel(iw, jn), lwSE = rel(ie, js), lwSW = rel(iw, js);
        const float a11P = L(a.a11, i, j), a11E = L(a.a11, ie, j), a11W = L(a.a11, iw, j);
        const float a22P = L(a.a22, i, j), a22N = L(a.a22, i, jn), a22S = L(a.a22, i, js);
        const float bP = L(a.a12, i, j), bE = L(a.a12, ie, j), bW = L(a.a12, iw, j);
        const float bN = L(a.a12, i, jn), bS = L(a.a12, i, js);
        // face differences of lamW seen from this cell (0 on boundary faces)
        const float LxE = hasE ? lwP - lwE : 0.0f, LxW = hasW ? lwW - lwP : 0.0f;
        const float LyN = hasN ? lwP - lwN : 0.0f, LyS = hasS ? lwS - lwP : 0.0f;
        // Sx on rows j-1, j, j+1 of column i; Sy on columns i-1, i, i+1 of row j
        auto sumx = [&](float c, float e, float w) { return (hasE ? c - e : 0.0f) + (hasW ? w - c : 0.0f); };
        auto sumy = [&](float c, float n, float s) { return (hasN ? c - n : 0.0f) + (hasS ? s - c : 0.0f); };
        const float SxP = bP * sumx(lwP, lwE, lwW);
        const float SxN = bN * sumx(lwN, lwNE, lwNW);
        const float SxS = bS * sumx(lwS, lwSE, lwSW);
        const float SyP = bP * sumy(lwP, lwN, lwS);
        const float SyE = bE * sumy(lwE, lwNE, lwSE);
        const float SyW = bW * sumy(lwW, lwNW, lwSW);
        const float Ty = (hasS ? SxS : 0.0f) - (hasN ? SxN : 0.0f) + SxP * ((hasN ? 0.0f : 1.0f) - (hasS ? 0.0f : 1.0f));
        const float Tx = (hasW ? SyW : 0.0f) - (hasE ? SyE : 0.0f) + SyP * ((hasE ? 0.0f : 1.0f) - (hasW ? 0.0f : 1.0f));
        const float D2T = ((a11P + a11E) * (lwE - lwP) + (a11W + a11P) * (lwW - lwP)) * k.kx +
                          ((a22P + a22N) * (lwN - lwP) + (a22S + a22P) * (lwS - lwP)) * k.ky + (Tx + Ty) * k.kc;

        const float uP = L(a.u, i, j), uE = L(a.u, ie, j), uW = L(a.u, iw, j), uN = L(a.u, i, jn), uS = L(a.u, i, js);
        const float vP = L(a.v, i, j), vE = L(a.v, ie, j), vW = L(a.v, iw, j), vN = L(a.v, i, jn), vS = L(a.v, i, js);
        const float wP = L(a.w, i, j), wE = L(a.w, ie, j), wW = L(a.w, iw, j), wN = L(a.w, i, jn), wS = L(a.w, i, js);
        const float luP = L(a.lu, i, j);
        auto cv = [&](int x, int y) { return KAHAN ? L(a.clv, x, y) : 0.0f; };
        const float lvP = L(a.lv, i, j), cvP = cv(i, j);
        auto relv = [&](int x, int y) { return (L(a.lv, x, y) - lvP) - (cv(x, y) - cvP); };
        // Table 1 pieces: mobility, V differences, lamV differences
        const float mE = 1.0f - 0.5f * (uP + uE), mW = 1.0f - 0.5f * (uP + uW);
        const float mN = 1.0f - 0.5f * (uP + uN), mS = 1.0f - 0.5f * (uP + uS);
        const float dvE = vE - vP, dvW = vW - vP, dvN = vN - vP, dvS = vS - vP;
        const float dlE = relv(ie, j), dlW = relv(iw, j), dlN = relv(i, jn), dlS = relv(i, js);
        const float d1 = (mE * dvE + mW * dvW) * k.ihx2 + (mN * dvN + mS * dvS) * k.ihy2;
        const float d1T = (mE * dlE + mW * dlW) * k.ihx2 + (mN * dlN + mS * dlS) * k.ihy2;
        const float dU = 0.5f * ((dvE * dlE + dvW * dlW) * k.ihx2 + (dvN * dlN + dvS * dlS) * k.ihy2);

        float fu, fv, fw;
        if (k.no_reaction) {
            fu = k.D * dU;
            fv = k.D * d1T;
            fw = D2T;
        } else {
            fu = (1.0f - 2.0f * uP - k.delta * wP) * luP + k.D * dU;
            fv = k.rho * (1.0f - 2.0f * vP) * lvP + k.D * d1T + k.c * lwP0;
            fw = -k.delta * uP * luP - k.c * lwP0 + D2T;
            s_delta = -(double)luP * (double)uP * (double)wP;
            s_rho = (double)lvP * (double)vP * (1.0 - (double)vP);
            s_c = (double)lwP0 * ((double)vP - (double)wP);
        }
        s_D = (double)lvP * (double)d1;
        const size_t o = (size_t)j * pitch + i;
        if constexpr (KAHAN) {
            float x, cx;
            kahan_add(luP, k.dt * fu, a.clu[o], x, cx); a.luo[o] = x; a.cluo[o] = cx;
            kahan_add(lvP, k.dt * fv, cvP, x, cx); a.lvo[o] = x; a.clvo[o] = cx;
            kahan_add(lwP0, k.dt * fw, cwP, x, cx); a.lwo[o] = x; a.clwo[o] = cx;
        } else {
            a.luo[o] = luP + k.dt * fu;
            a.lvo[o] = lvP + k.dt * fv;
            a.lwo[o] = lwP0 + k.dt * fw;
        }
        // tensor gradients (FP32 sums, folded into FP64 every kFlushEvery steps)
        a.g11[o] += k.dt * (((wE - wP) * LxE + (wP - wW) * LxW) * k.kx);
        a.g22[o] += k.dt * (((wN - wP) * LyN + (wP - wS) * LyS) * k.ky);
        a.g12[o] += k.dt * (((LxE + LxW) * (wN - wS) + (LyN + LyS) * (wE - wW)) * k.kc);
#undef L
    }
    // FP64 block reduction of the rate gradients, accumulated per block
    __shared__ double sh[4][kAdjBX * kAdjBY / 32];
    double s4[4] = {s_delta, s_rho, s_D, s_c};
    for (int q = 0; q < 4; ++q)
        for (int off = 16; off > 0; off >>= 1) s4[q] += __shfl_xor_sync(0xffffffffu, s4[q], off);
    const int tid = threadIdx.y * kAdjBX + threadIdx.x;
    if ((tid & 31) == 0)
        for (int q = 0; q < 4; ++q) sh[q][tid >> 5] = s4[q];
    __syncthreads();
    if (tid == 0) {
        double* p = a.partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4;
        const double dtd = (double)k.dt;
        for (int q = 0; q < 4; ++q) {
            double t = 0.0;
            for (int wq = 0; wq < kAdjBX * kAdjBY / 32; ++wq) t += sh[q][wq];
            p[q] += dtd * t;
        }
    }
}

// g64 += g32; g32 = 0 (pitched, 3 fields)
__global__ void flush_kernel(float* g1, float* g2, float* g3, double* h1, double* h2, double* h3, int nx, int ny,
                             int pitch)
{
    const size_t n = (size_t)ny * pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        if ((int)(q % pitch) >= nx) continue;
        h1[q] += (double)g1[q]; g1[q] = 0.0f;
        h2[q] += (double)g2[q]; g2[q] = 0.0f;
        h3[q] += (double)g3[q]; g3[q] = 0.0f;
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
    std::vector<float*> stash;    // K x 3 fields (slot 0 unused)
    float* scomp[2][3] = {};      // Kahan terms of the recomputed states
    float* lam[2][6] = {};        // lam and its Kahan terms, ping-pong
    float* g32[3] = {};
    double* g64[3] = {};
    double* partials = nullptr;
    int nblocks = 0;
};

}  // namespace

void gg_release_extras(gg_sim* s)
{
    if (s && s->adj) {
        AdjWork* w = (AdjWork*)s->adj;
        if (w->base) cudaFree(w->base);
        delete w;
        s->adj = nullptr;
    }
}

static int adj_workspace(gg_sim* s, int K, int nseg, bool kahan, AdjWork** out)
{
    const size_t fb = ((size_t)s->pitch * s->ny * 4 + 255) / 256 * 256;
    const size_t db = ((size_t)s->pitch * s->ny * 8 + 255) / 256 * 256;
    const int nstate = kahan ? 6 : 3;
    const dim3 grid((s->nx + kAdjBX - 1) / kAdjBX, (s->ny + kAdjBY - 1) / kAdjBY);
    const int nblocks = grid.x * grid.y;
    const size_t need = fb * ((size_t)nseg * nstate + (size_t)K * 3 + 6 + 12 + 3) + db * 3 +
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
    w->stash.assign((size_t)K * 3, nullptr);
    for (auto& f : w->stash) { f = (float*)p; p += fb; }
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

    // 1. forward pass, storing the state (with Kahan terms) at the start of every segment
    for (int seg = 0; seg < nseg && e == cudaSuccess; ++seg) {
        for (int f = 0; f < nstate && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(w->ckpt[(size_t)seg * nstate + f], s->f32[s->cur][f], fbytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) break;
        const int64_t len = std::min<int64_t>(K, N - (int64_t)seg * K);
        rc = gg_step(s, len);
        if (rc != GG_OK) return rc;
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

    const Rates32 r = rates32(s);
    Plan32 plan1 = s->plan;
    plan1.T = 1;
    const dim3 agrid((s->nx + kAdjBX - 1) / kAdjBX, (s->ny + kAdjBY - 1) / kAdjBY);
    const dim3 ablock(kAdjBX, kAdjBY);
    int lb = 0;          // current lam buffer
    int since_flush = 0;
    auto flush = [&]() {
        flush_kernel<<<blocks_for((size_t)s->pitch * s->ny), 256, 0, st>>>(w->g32[0], w->g32[1], w->g32[2], w->g64[0],
                                                                          w->g64[1], w->g64[2], s->nx, s->ny, s->pitch);
        since_flush = 0;
        return cudaGetLastError();
    };
    // 3. segments in reverse: recompute the states of the segment, then run its adjoint steps
    for (int seg = nseg - 1; seg >= 0 && e == cudaSuccess; --seg) {
        const int len = (int)std::min<int64_t>(K, N - (int64_t)seg * K);
        auto state = [&](int kk, int f) -> float* {  // u, v, w of X^{seg*K + kk}
            return kk == 0 ? w->ckpt[(size_t)seg * nstate + f] : w->stash[(size_t)kk * 3 + f];
        };
        auto comp = [&](int kk, int f) -> float* {
            if (!kahan) return nullptr;
            return kk == 0 ? w->ckpt[(size_t)seg * nstate + 3 + f] : w->scomp[kk & 1][f];
        };
        for (int kk = 0; kk + 1 < len && e == cudaSuccess; ++kk) {
            Grid32 g;
            g.u = state(kk, 0); g.v = state(kk, 1); g.w = state(kk, 2);
            g.cu = comp(kk, 0); g.cv = comp(kk, 1); g.cw = comp(kk, 2);
            g.uo = state(kk + 1, 0); g.vo = state(kk + 1, 1); g.wo = state(kk + 1, 2);
            g.cuo = kahan ? w->scomp[(kk + 1) & 1][0] : nullptr;
            g.cvo = kahan ? w->scomp[(kk + 1) & 1][1] : nullptr;
            g.cwo = kahan ? w->scomp[(kk + 1) & 1][2] : nullptr;
            g.a11 = s->a32[0]; g.a12 = s->a32[1]; g.a22 = s->a32[2];
            g.nx = s->nx; g.ny = s->ny; g.pitch = s->pitch;
            e = launch_plan(g, r, plan1, 1, kahan, st);
        }
        for (int kk = len - 1; kk >= 0 && e == cudaSuccess; --kk) {
            AdjArgs a;
            a.u = state(kk, 0); a.v = state(kk, 1); a.w = state(kk, 2);
            a.lu = w->lam[lb][0]; a.lv = w->lam[lb][1]; a.lw = w->lam[lb][2];
            a.clu = w->lam[lb][3]; a.clv = w->lam[lb][4]; a.clw = w->lam[lb][5];
            a.luo = w->lam[lb ^ 1][0]; a.lvo = w->lam[lb ^ 1][1]; a.lwo = w->lam[lb ^ 1][2];
            a.cluo = w->lam[lb ^ 1][3]; a.clvo = w->lam[lb ^ 1][4]; a.clwo = w->lam[lb ^ 1][5];
            a.a11 = s->a32[0]; a.a12 = s->a32[1]; a.a22 = s->a32[2];
            a.g11 = w->g32[0]; a.g12 = w->g32[1]; a.g22 = w->g32[2];
            a.partials = w->partials;
            a.nx = s->nx; a.ny = s->ny; a.pitch = s->pitch;
            if (kahan) adjoint_step_kernel<true><<<agrid, ablock, 0, st>>>(a, r);
            else adjoint_step_kernel<false><<<agrid, ablock, 0, st>>>(a, r);
            e = cudaGetLastError();
            lb ^= 1;
            if (e == cudaSuccess && ++since_flush == kFlushEvery) e = flush();
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
