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

// Geometry of the warp-marching adjoint launches.  A grid of strips x chunks
// warps runs in waves of `cap` resident warps (152 SMs times the warps per SM
// that the launch bounds guarantee).  The chunk height is chosen so that the
// grid fills a whole number of waves where it can: a grid of one wave plus a
// few CTAs takes about two warp lifetimes.
inline int wave_chunk(int strips, int ny, int cap, int hmax)
{
    constexpr int hmin = 8;
    if (strips > cap) return std::min(hmax, std::max(hmin, ny));
    const int per_wave = cap / strips;  // chunk rows of warps per wave
    const int waves = std::max(1, (ny + per_wave * hmax - 1) / (per_wave * hmax));
    const int nch = waves * per_wave;
    return std::min(hmax, std::max(hmin, (ny + nch - 1) / nch));
}
// Single step: 30 written columns per warp, 5 CTAs of 4 warps per SM.
constexpr int kAdjOut = 30;
inline int adj_strips(int nx) { return (nx + kAdjOut - 1) / kAdjOut; }
inline int adj_chunk(int nx, int ny) { return wave_chunk(adj_strips(nx), ny, 20 * 152, 128); }
inline int adj_warps(int nx, int ny) { const int H = adj_chunk(nx, ny); return adj_strips(nx) * ((ny + H - 1) / H); }
// Two steps: 28 written columns per warp, 4 CTAs of 4 warps per SM.
inline int adj2_strips(int nx) { return (nx + 27) / 28; }
inline int adj2_chunk(int nx, int ny) { return wave_chunk(adj2_strips(nx), ny, 16 * 152, 128); }
inline int adj2_warps(int nx, int ny) { const int H = adj2_chunk(nx, ny); return adj2_strips(nx) * ((ny + H - 1) / H); }
constexpr int kFlushEvery = 32;  // FP32 per-cell gradient sums are folded into FP64 this often

struct AdjArgs {
    const float *u, *v, *w;                          // X^k
    const float *lu, *lv, *lw, *clu, *clv, *clw;     // lam^{k+1} and its Kahan terms
    float *luo, *lvo, *lwo, *cluo, *clvo, *clwo;     // lam^k
    const float *ax, *b, *ay;                        // face / cross weights (Grid32)
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

constexpr unsigned kFull = 0xffffffffu;
__device__ __forceinline__ float from_west(float x) { return __shfl_up_sync(kFull, x, 1); }
__device__ __forceinline__ float from_east(float x) { return __shfl_down_sync(kFull, x, 1); }

// One row of the inputs of an adjoint step at one column: the fields read on
// rows q and q+1 (AdjRow; of row q-1 only w is read) and those read on row q
// only (AdjOwn).
struct AdjRow {
    float u, v, w, lv, lw, clv, clw, b, ay;
};
struct AdjOwn {
    float lu, clu, ax, g11, g12, g22;
};
// Result of one adjoint level at one cell: lam at step k with its Kahan
// terms, dt times the tensor-gradient increments, the four rate terms.
struct AdjOut {
    float lu, clu, lv, clv, lw, clw;
    float d11, d12, d22;
    float s_delta, s_rho, s_D, s_c;
};

// What one adjoint level passes from row q-1 to row q.  The level reads row
// q+1 as its north row when it processes row q; at the next tick that row
// is its own row.  So the x-face differences of lamW and the cross sums of
// a row are computed once, when it is the north row, and every south-face
// term of row q is the north-face term of row q-1 (of equal value, or of
// opposite sign where the difference changes direction: it is kept with the
// sign of the north face and subtracted).
struct AdjCarry {
    float LxE = 0.f, LxW = 0.f;  // lamW differences across the east / west faces of row q
    float Sx = 0.f, SxS = 0.f;   // b (LxE + LxW) of rows q and q-1
    float Ly = 0.f;              // lamW difference across the north face of row q-1
    float f = 0.f, e = 0.f, g = 0.f, qq = 0.f;  // north-face terms of row q-1 (below)
};

// One adjoint step at row q of one lane, from the state and lam of rows P (q)
// and N (q+1), w of row q-1 and the own-row fields lu, clu and ax (east-face
// weight), with the carry c of row q-1 (updated for row q+1).  All lanes of
// the warp call it (it shuffles).  Face terms, each with the factor 1/h^2 of
// its direction: with m = 1 - (U_P + U_nb)/2, dv = V_nb - V_P, dl the
// compensated difference of lamV (neighbour minus own),
//   f = m dl (D1^T of lamV),  e = dv dl (dD1/dU),
// the east / north terms are computed here, the west ones are the west
// lane's east ones and the south ones the carried north ones of row q-1:
//   D1^T = (fE - fW) + (fN - fS),  dD1/dU = (eE + eW + eN + eS) / 2.
// The rate term of D, sum_cells lamV D1(V; U), is taken in its transposed
// form sum_cells V D1^T(lamV; U): D1(.; U) is a symmetric matrix (Table 1's
// face fluxes with zero flux through boundary faces), so the two sums are
// equal, and the second needs no second difference of the FP32 state V
// (whose rounding, divided by h^2, swamps the smooth part of D1(V) on fine
// grids) but only the compensated differences of lamV.
template <bool KAHAN, bool EDGE, bool YEDGE = true>
__device__ __forceinline__ AdjOut adj_level(const Rates32& k, float Sw, const AdjRow& P, const AdjRow& N, float lu,
                                            float clu, float ax, bool hasW, bool hasE, bool hasS_, bool hasN_,
                                            AdjCarry& c)
{
    // interior chunks (YEDGE false) have both the south and the north face
    const bool hasS = YEDGE ? hasS_ : true, hasN = YEDGE ? hasN_ : true;
    // compensated difference of lam between two (value, Kahan term) pairs
    auto dW = [](float la, float ca, float lb, float cb) { return __fsub_rn(__fsub_rn(la, lb), __fsub_rn(ca, cb)); };
    // x-face differences of lamW on the north row (0 on boundary faces)
    const float lwE = from_east(N.lw), cwE = from_east(N.clw);
    const float LxE_N = hasE ? dW(N.lw, N.clw, lwE, cwE) : 0.0f;
    float LxW_N = from_west(LxE_N);
    if (EDGE && !hasW) LxW_N = 0.0f;
    const float LxE_P = c.LxE, LxW_P = c.LxW;
    const float LyN = hasN ? dW(P.lw, P.clw, N.lw, N.clw) : 0.0f;
    const float LyS = hasS ? c.Ly : 0.0f;
    // transpose of the a12 cross terms (mirrored central differences; b
    // carries the factor 1/(4 dx dy))
    const float SxN = N.b * (LxE_N + LxW_N), SxP = c.Sx, SxS = c.SxS;
    const float SyP = P.b * (LyN + LyS);
    float SyE = from_east(SyP), SyW = from_west(SyP);
    const float Ty = (hasS ? SxS : 0.0f) - (hasN ? SxN : 0.0f) + SxP * ((hasN ? 0.0f : 1.0f) - (hasS ? 0.0f : 1.0f));
    float Tx;
    if (EDGE) Tx = (hasW ? SyW : 0.0f) - (hasE ? SyE : 0.0f) + SyP * ((hasE ? 0.0f : 1.0f) - (hasW ? 0.0f : 1.0f));
    else Tx = SyW - SyE;
    // face weights: east ax, west = the west lane's ax, north P.ay, south the
    // carried product of row q-1 (a boundary face has L = 0)
    const float axW = from_west(ax);
    const float gN = P.ay * LyN;
    const float D2T = (ax * (-LxE_P) + axW * LxW_P) + ((hasS ? c.g : 0.0f) - gN) + (Tx + Ty);

    // state and lamV neighbourhood (mirrored at the boundary)
    float uE = from_east(P.u), vE = from_east(P.v), wE = from_east(P.w), wW = from_west(P.w);
    float lvE = from_east(P.lv), cvE = from_east(P.clv);
    if (EDGE) {
        if (!hasE) { uE = P.u; vE = P.v; wE = P.w; lvE = P.lv; cvE = P.clv; }
        if (!hasW) wW = P.w;
    }
    const float uN = hasN ? N.u : P.u, vN = hasN ? N.v : P.v, wN = hasN ? N.w : P.w;
    const float wS = hasS ? Sw : P.w;
    const float mE = 1.0f - 0.5f * (P.u + uE), mN = 1.0f - 0.5f * (P.u + uN);
    const float dvE = (vE - P.v) * k.ihx2, dvN = (vN - P.v) * k.ihy2;
    const float dlE = dW(lvE, cvE, P.lv, P.clv), dlN = hasN ? dW(N.lv, N.clv, P.lv, P.clv) : 0.0f;
    const float fE = mE * dlE * k.ihx2, eE = dvE * dlE;
    const float fN = mN * dlN * k.ihy2, eN = dvN * dlN;
    float fW = from_west(fE), eW = from_west(eE);
    if (EDGE && !hasW) { fW = 0.0f; eW = 0.0f; }
    const float fS = hasS ? c.f : 0.0f, eS = hasS ? c.e : 0.0f;
    const float d1T = (fE - fW) + (fN - fS);
    const float dU = 0.5f * ((eE + eW) + (eN + eS));

    float fu, fvv, fw;
    AdjOut o;
    if (k.no_reaction) {
        fu = k.D * dU;
        fvv = k.D * d1T;
        fw = D2T;
        o.s_delta = o.s_rho = o.s_c = 0.0f;
    } else {
        fu = (1.0f - 2.0f * P.u - k.delta * P.w) * lu + k.D * dU;
        fvv = k.rho * (1.0f - 2.0f * P.v) * P.lv + k.D * d1T + k.c * P.lw;
        fw = -k.delta * P.u * lu - k.c * P.lw + D2T;
        o.s_delta = -lu * P.u * P.w;
        o.s_rho = P.lv * P.v * (1.0f - P.v);
        o.s_c = P.lw * (P.v - P.w);
    }
    o.s_D = P.v * d1T;
    if (KAHAN) {
        kahan_add(lu, k.dt * fu, clu, o.lu, o.clu);
        kahan_add(P.lv, k.dt * fvv, P.clv, o.lv, o.clv);
        kahan_add(P.lw, k.dt * fw, P.clw, o.lw, o.clw);
    } else {
        o.lu = lu + k.dt * fu;
        o.lv = P.lv + k.dt * fvv;
        o.lw = P.lw + k.dt * fw;
        o.clu = o.clv = o.clw = 0.0f;
    }
    const float qN = (wN - P.w) * LyN;
    o.d11 = k.dt * (((wE - P.w) * LxE_P + (P.w - wW) * LxW_P) * k.kx);
    o.d22 = k.dt * ((qN + (hasS ? c.qq : 0.0f)) * k.ky);
    o.d12 = k.dt * (((LxE_P + LxW_P) * (wN - wS) + (LyN + LyS) * (wE - wW)) * k.kc);
    // row q becomes row q-1 of the next tick
    c.LxE = LxE_N; c.LxW = LxW_N;
    c.SxS = SxP; c.Sx = SxN;
    c.Ly = LyN;
    c.f = fN; c.e = eN; c.g = gN; c.qq = qN;
    return o;
}

// Per-lane FP32 compensated sums of the four rate terms, folded into one
// FP64 record per warp at the end of the chunk (fixed order).  delta, rho and
// c use Kahan's update; the D term, V D1^T(lamV), sums to a small fraction of
// the sum of its magnitudes (D1^T(lamV) sums to zero over the domain), so it
// keeps the exact rounding error of every addition (TwoSum) in a second
// accumulator: the result is then accurate to about one FP32 rounding of the
// sum itself rather than of the sum of magnitudes.
struct RateSums {
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, accc[4] = {0.f, 0.f, 0.f, 0.f};
    __device__ __forceinline__ void add(int q, float x)
    {
        const float y = __fsub_rn(x, accc[q]);
        const float t = __fadd_rn(acc[q], y);
        accc[q] = __fsub_rn(__fsub_rn(t, acc[q]), y);
        acc[q] = t;
    }
    // acc + x = s + e exactly (TwoSum); e is gathered in -accc (so that the
    // fold below, acc - accc, stays the same for both kinds of sum)
    __device__ __forceinline__ void add_two_sum(int q, float x)
    {
        const float s = __fadd_rn(acc[q], x);
        const float z = __fsub_rn(s, acc[q]);
        const float e = __fadd_rn(__fsub_rn(acc[q], __fsub_rn(s, z)), __fsub_rn(x, z));
        accc[q] = __fsub_rn(accc[q], e);
        acc[q] = s;
    }
    __device__ __forceinline__ void add_all(const AdjOut& o)
    {
        add(0, o.s_delta);
        add(1, o.s_rho);
        add_two_sum(2, o.s_D);
        add(3, o.s_c);
    }
    __device__ __forceinline__ void fold(double* part, int lane, float dt)
    {
        double s4[4];
        for (int qq = 0; qq < 4; ++qq) {
            s4[qq] = (double)acc[qq] - (double)accc[qq];
            for (int off = 16; off > 0; off >>= 1) s4[qq] += __shfl_xor_sync(kFull, s4[qq], off);
        }
        if (lane == 0) {
            const double dtd = (double)dt;
            for (int qq = 0; qq < 4; ++qq) part[qq] += dtd * s4[qq];
        }
    }
};

// Loads of one row at one column (zeros outside the domain).
template <bool KAHAN>
__device__ __forceinline__ void load_row(const float* u, const float* v, const float* w, const float* lv,
                                         const float* lw, const float* clv, const float* clw, const float* b,
                                         const float* ay, bool in, size_t o, AdjRow& x)
{
    if (in) {
        x.u = __ldg(u + o); x.v = __ldg(v + o); x.w = __ldg(w + o);
        x.lv = __ldg(lv + o); x.lw = __ldg(lw + o);
        if (KAHAN) { x.clv = __ldg(clv + o); x.clw = __ldg(clw + o); }
        else { x.clv = x.clw = 0.0f; }
        x.b = __ldg(b + o); x.ay = __ldg(ay + o);
    } else {
        x.u = x.v = x.w = x.lv = x.lw = x.clv = x.clw = x.b = x.ay = 0.0f;
    }
}

// Adjoint step as a warp march: the warp owns 32 columns (30 written) and a
// chunk of H rows, keeps rows q, q+1 (and w of q-1) of its inputs in
// registers (window rows fetched two ahead, own-row fields one ahead) and
// takes east / west values by shuffle.  The march starts two rows above the
// chunk (not above row -1), so that the carry of the first written row is
// complete.
template <bool KAHAN, bool EDGE, bool YEDGE>
__device__ __forceinline__ void adj_warp(const AdjArgs& a, const Rates32& k, const int H, const int strip,
                                         const int chunk, const int lane, double* part)
{
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const int gx = strip * 30 - 1 + lane;
    const bool ind = EDGE ? (gx >= 0 && gx < nx) : true;
    const bool hasW = EDGE ? gx > 0 : true, hasE = EDGE ? gx + 1 < nx : true;
    const bool outc = ind && lane >= 1 && lane < 31;
    const int ys = chunk * H;
    const int ye = min(ny, ys + H);
    const int q0 = max(-1, ys - 2);
    auto load = [&](int r, AdjRow& x) {
        load_row<KAHAN>(a.u, a.v, a.w, a.lv, a.lw, a.clv, a.clw, a.b, a.ay, ind && r >= 0 && r < ny,
                        (size_t)r * pitch + gx, x);
    };
    auto load_own = [&](int r, AdjOwn& x) {
        if (ind && r >= 0 && r < ny) {
            const size_t o = (size_t)r * pitch + gx;
            x.lu = __ldg(a.lu + o);
            x.clu = KAHAN ? __ldg(a.clu + o) : 0.0f;
            x.ax = __ldg(a.ax + o);
            x.g11 = __ldg(a.g11 + o); x.g12 = __ldg(a.g12 + o); x.g22 = __ldg(a.g22 + o);
        } else {
            x.lu = x.clu = x.ax = x.g11 = x.g12 = x.g22 = 0.0f;
        }
    };
    RateSums sums;
    AdjCarry cy;
    AdjRow P, N, nxt;
    AdjOwn PO, NO;
    float Sw = (ind && q0 - 1 >= 0) ? __ldg(a.w + (size_t)(q0 - 1) * pitch + gx) : 0.0f;
    load(q0, P);
    load(q0 + 1, N);
    load(q0 + 2, nxt);
    load_own(q0, PO);
    for (int q = q0; q < ye; ++q) {
        AdjRow nn;
        load(q + 3, nn);
        load_own(q + 1, NO);
        const AdjOut o = adj_level<KAHAN, EDGE, YEDGE>(k, Sw, P, N, PO.lu, PO.clu, PO.ax, hasW, hasE, q > 0,
                                                       q + 1 < ny, cy);
        if (q >= ys && outc) {
            const size_t off = (size_t)q * pitch + gx;
            sums.add_all(o);
            a.luo[off] = o.lu; a.lvo[off] = o.lv; a.lwo[off] = o.lw;
            if (KAHAN) { a.cluo[off] = o.clu; a.clvo[off] = o.clv; a.clwo[off] = o.clw; }
            a.g11[off] = PO.g11 + o.d11;
            a.g12[off] = PO.g12 + o.d12;
            a.g22[off] = PO.g22 + o.d22;
        }
        Sw = P.w;
        P = N;
        N = nxt;
        nxt = nn;
        PO = NO;
    }
    sums.fold(part, lane, k.dt);
}

template <bool KAHAN>
__global__ void __launch_bounds__(128, 5) adjoint_step_kernel(const AdjArgs a, const Rates32 k, const int H,
                                                              const int nstrips, const int nwarps)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= nwarps) return;
    const int strip = gw % nstrips, chunk = gw / nstrips;
    const int gx0 = strip * 30 - 1;
    double* part = a.partials + (size_t)gw * 4;
    const int ys = chunk * H;
    const bool yin = ys - 1 >= 1 && ys + H + 1 <= a.ny - 1;
    if (gx0 >= 1 && gx0 + 31 <= a.nx - 2) {
        if (yin) adj_warp<KAHAN, false, false>(a, k, H, strip, chunk, lane, part);
        else adj_warp<KAHAN, false, true>(a, k, H, strip, chunk, lane, part);
    } else {
        adj_warp<KAHAN, true, true>(a, k, H, strip, chunk, lane, part);
    }
}

// Two adjoint steps per pass (steps k+1 and k of the reverse sweep).  Level 1
// turns lam^{k+2} into lam^{k+1} with X^{k+1}; level 2 turns lam^{k+1} into
// lam^k with X^k one row behind, so lam^{k+1} never leaves registers and the
// per-cell gradient sums are read and written once per two steps.  Lanes
// [2, 30) of a warp are written; level 1 also produces the halo row and
// column the second level needs.  At tick r the input row r enters; level 1
// computes row r - 1, level 2 row r - 2.
struct AdjArgs2 {
    const float *u1, *v1, *w1;  // X^{k+1}
    const float *u0, *v0, *w0;  // X^k
    const float *lu, *lv, *lw, *clu, *clv, *clw;  // lam^{k+2}
    float *luo, *lvo, *lwo, *cluo, *clvo, *clwo;  // lam^k
    const float *ax, *b, *ay;
    float *g11, *g12, *g22;
    double* partials;
    int nx, ny, pitch;
};

template <bool KAHAN, bool EDGE, bool YEDGE>
__device__ __forceinline__ void adj2_warp(const AdjArgs2& a, const Rates32& k, const int H, const int strip,
                                          const int chunk, const int lane, double* part)
{
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const int gx = strip * 28 - 2 + lane;
    const bool ind = EDGE ? (gx >= 0 && gx < nx) : true;
    const bool hasW = EDGE ? gx > 0 : true, hasE = EDGE ? gx + 1 < nx : true;
    const bool outc = ind && lane >= 2 && lane < 30;
    const int ys = chunk * H;
    const int ye = min(ny, ys + H);
    const int lo0 = max(0, ys - 2);
    const int nticks = ye + 2 - lo0;  // level 2 reaches row ye - 1 at tick ye + 1
    auto inrow = [&](int r) { return ind && r >= 0 && r < ny; };
    // level-1 input row (lam^{k+2}, X^{k+1}, tensor) and own fields
    auto load1 = [&](int r, AdjRow& x, float& lu, float& clu, float& ax) {
        const bool in = inrow(r);
        const size_t o = (size_t)r * pitch + gx;
        load_row<KAHAN>(a.u1, a.v1, a.w1, a.lv, a.lw, a.clv, a.clw, a.b, a.ay, in, o, x);
        lu = in ? __ldg(a.lu + o) : 0.0f;
        clu = (in && KAHAN) ? __ldg(a.clu + o) : 0.0f;
        ax = in ? __ldg(a.ax + o) : 0.0f;
    };
    // level-2 state row (X^k)
    auto load0 = [&](int r, float& u, float& v, float& w) {
        if (inrow(r)) {
            const size_t o = (size_t)r * pitch + gx;
            u = __ldg(a.u0 + o); v = __ldg(a.v0 + o); w = __ldg(a.w0 + o);
        } else {
            u = v = w = 0.0f;
        }
    };
    RateSums sums;
    // Level 1 computes row r - 1 at tick r, level 2 row r - 2; each has its
    // own carry.  Before the first written rows each level passes over two
    // rows (from lo0), which completes its carry (at the top of the domain
    // the missing south faces need none).
    AdjCarry c1, c2;
    // level-1 window: rows r-1 (P1), r (N1), w of r-2
    AdjRow P1{}, N1{};
    float S1w = 0.f;
    float luP = 0.f, cluP = 0.f, axP = 0.f, luN = 0.f, cluN = 0.f, axN = 0.f;
    // level-2 window: lam^{k+1} and X^k of rows r-2 (P2), r-1 (N2), w of r-3
    AdjRow P2{}, N2{};
    float S2w = 0.f;
    float d11c = 0.f, d12c = 0.f, d22c = 0.f;      // level-1 gradient increments of level 2's row
    // prefetch the first level-1 input row
    AdjRow in1;
    float inlu, inclu, inax;
    load1(lo0, in1, inlu, inclu, inax);
    float lu1prev = 0.f, clu1prev = 0.f, axprev = 0.f;  // level-1 outputs of the previous tick
    AdjOut prev1{};
    bool prev_own = false;
    for (int tk = 0; tk < nticks; ++tk) {
        const int r = lo0 + tk;
        // input row r enters level 1's window; X^k row r - 1 enters level 2's
        S1w = P1.w; P1 = N1; N1 = in1;
        luP = luN; cluP = cluN; axP = axN;
        luN = inlu; cluN = inclu; axN = inax;
        // loads issued here are used after level 1 (X^k of row r - 1) and
        // after level 2 (the gradient sums of row r - 2); the next level-1
        // row is used at the next tick
        float x0u, x0v, x0w;
        load0(r - 1, x0u, x0v, x0w);
        const int q2 = r - 2;
        const bool own2 = q2 >= ys && q2 < ye && outc;
        float g11 = 0.f, g12 = 0.f, g22 = 0.f;
        if (own2) {
            const size_t off = (size_t)q2 * pitch + gx;
            g11 = __ldg(a.g11 + off); g12 = __ldg(a.g12 + off); g22 = __ldg(a.g22 + off);
        }
        load1(r + 1, in1, inlu, inclu, inax);
        // level 1: row q1 = r - 1
        const int q1 = r - 1;
        const AdjOut o1 = adj_level<KAHAN, EDGE, YEDGE>(k, S1w, P1, N1, luP, cluP, axP, hasW, hasE, q1 > 0,
                                                        q1 + 1 < ny, c1);
        const bool own1 = q1 >= ys && q1 < ye;  // level 1's rate terms count on the chunk's rows
        // level-1 lam^{k+1} row q1 enters level 2's window (with X^k row q1 and the tensor of row q1)
        AdjRow nw;
        nw.u = x0u; nw.v = x0v; nw.w = x0w;
        nw.lv = o1.lv; nw.clv = o1.clv; nw.lw = o1.lw; nw.clw = o1.clw;
        nw.b = P1.b; nw.ay = P1.ay;
        S2w = P2.w; P2 = N2; N2 = nw;
        // level 2: row q2 = r - 2, own fields from level 1's previous output
        const AdjOut o2 = adj_level<KAHAN, EDGE, YEDGE>(k, S2w, P2, N2, lu1prev, clu1prev, axprev, hasW, hasE,
                                                        q2 > 0, q2 + 1 < ny, c2);
        if (own2) {
            const size_t off = (size_t)q2 * pitch + gx;
            sums.add_all(o2);
            if (prev_own) sums.add_all(prev1);
            a.luo[off] = o2.lu; a.lvo[off] = o2.lv; a.lwo[off] = o2.lw;
            if (KAHAN) { a.cluo[off] = o2.clu; a.clvo[off] = o2.clv; a.clwo[off] = o2.clw; }
            a.g11[off] = g11 + (d11c + o2.d11);
            a.g12[off] = g12 + (d12c + o2.d12);
            a.g22[off] = g22 + (d22c + o2.d22);
        }
        // level 1's row q1 becomes level 2's row at the next tick
        lu1prev = o1.lu; clu1prev = o1.clu; axprev = axP;
        d11c = o1.d11; d12c = o1.d12; d22c = o1.d22;
        prev1 = o1;
        prev_own = own1;
    }
    sums.fold(part, lane, k.dt);
}

template <bool KAHAN>
__global__ void __launch_bounds__(128, 4) adjoint2_kernel(const AdjArgs2 a, const Rates32 k, const int H,
                                                          const int nstrips, const int nwarps)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= nwarps) return;
    const int strip = gw % nstrips, chunk = gw / nstrips;
    const int gx0 = strip * 28 - 2;
    double* part = a.partials + (size_t)gw * 4;
    const int ys = chunk * H;
    const bool yin = ys - 3 >= 1 && ys + H + 3 <= a.ny - 1;
    if (gx0 >= 1 && gx0 + 31 <= a.nx - 2) {
        if (yin) adj2_warp<KAHAN, false, false>(a, k, H, strip, chunk, lane, part);
        else adj2_warp<KAHAN, false, true>(a, k, H, strip, chunk, lane, part);
    } else {
        adj2_warp<KAHAN, true, true>(a, k, H, strip, chunk, lane, part);
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
    const int nblocks = std::max(adj_warps(s->nx, s->ny), adj2_warps(s->nx, s->ny));
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
    // recompute depth and chunk height: the simulation's warp plan when it has
    // one, else single steps
    const bool warp_plan = s->plan.kind == 1 || s->plan.kind == 3;
    const int TR = warp_plan ? s->plan.T : 1;
    const int HR = warp_plan ? s->plan.by : default_plan(s->nx, s->ny, 1).by;
    const bool paired = s->plan.kind == 3;
    // Runs nsteps steps from the state `in` (u, v, w, cu, cv, cw) in passes of
    // up to TR steps.  The state after step kk (1 <= kk < nsteps, and nsteps
    // itself when fin is null) is written to slot(kk) (u, v, w); the last
    // state goes to fin (u, v, w and Kahan terms) when fin is given.  Kahan
    // terms between passes alternate between the two scomp buffers.
    auto passes = [&](float* const in[6], int nsteps, auto slot, float* const* fin) -> cudaError_t {
        int kk = 0, pass = 0;
        cudaError_t ee = cudaSuccess;
        while (kk < nsteps && ee == cudaSuccess) {
            const int Tp = std::min(TR, nsteps - kk);
            const bool last = kk + Tp == nsteps && fin;
            Grid32 g;
            if (kk == 0) { g.u = in[0]; g.v = in[1]; g.w = in[2]; }
            else { float* const* x = slot(kk); g.u = x[0]; g.v = x[1]; g.w = x[2]; }
            g.cu = kahan ? (kk == 0 ? in[3] : w->scomp[pass & 1][0]) : nullptr;
            g.cv = kahan ? (kk == 0 ? in[4] : w->scomp[pass & 1][1]) : nullptr;
            g.cw = kahan ? (kk == 0 ? in[5] : w->scomp[pass & 1][2]) : nullptr;
            if (last) {
                g.uo = fin[0]; g.vo = fin[1]; g.wo = fin[2];
                g.cuo = kahan ? fin[3] : nullptr; g.cvo = kahan ? fin[4] : nullptr; g.cwo = kahan ? fin[5] : nullptr;
            } else {
                float* const* x = slot(kk + Tp);
                g.uo = x[0]; g.vo = x[1]; g.wo = x[2];
                g.cuo = kahan ? w->scomp[(pass + 1) & 1][0] : nullptr;
                g.cvo = kahan ? w->scomp[(pass + 1) & 1][1] : nullptr;
                g.cwo = kahan ? w->scomp[(pass + 1) & 1][2] : nullptr;
            }
            g.ax = s->a32[0]; g.b = s->a32[1]; g.ay = s->a32[2];
            g.nx = s->nx; g.ny = s->ny; g.pitch = s->pitch;
            Stash32 sh = {};
            for (int t = 1; t < Tp; ++t) {
                float* const* x = slot(kk + t);
                sh.u[t - 1] = x[0]; sh.v[t - 1] = x[1]; sh.w[t - 1] = x[2];
            }
            ee = paired ? launch_stepw2_stash(g, r, HR, Tp, kahan, sh, st) : launch_stepw_stash(g, r, HR, Tp, kahan, sh, st);
            kk += Tp;
            ++pass;
        }
        return ee;
    };

    // Trailing segments whose states fit in 60 % of the free device memory are
    // kept from the forward pass and need no recomputation.
    int ns = 0;
    {
        size_t freeb = 0, totalb = 0;
        if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) { cudaGetLastError(); freeb = 0; }
        const size_t per_seg = (size_t)K * 3 * ((fbytes + 255) / 256 * 256);
        const size_t have = w->big_bytes;
        // 60 % of (what this workspace already holds + what is free): the same
        // budget on every call, so a second call reuses the first call's buffer
        const size_t budget = (have + freeb) / 10 * 6;
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
    auto big_slot = [&](int seg, int kk, float** out3) {
        char* b = (char*)w->big + ((size_t)(seg - seg_kept) * K + kk) * 3 * fstride;
        out3[0] = (float*)b; out3[1] = (float*)(b + fstride); out3[2] = (float*)(b + 2 * fstride);
    };

    // 1. forward pass, storing the state (with Kahan terms) at the start of every
    // segment and every state of the trailing segments
    for (int seg = 0; seg < nseg && e == cudaSuccess; ++seg) {
        for (int f = 0; f < nstate && e == cudaSuccess; ++f)
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

    const int aH = adj_chunk(s->nx, s->ny), astrips = adj_strips(s->nx), awarps = adj_warps(s->nx, s->ny);
    const int ablocks = (awarps + 3) / 4;
    const int a2H = adj2_chunk(s->nx, s->ny), a2strips = adj2_strips(s->nx), a2warps = adj2_warps(s->nx, s->ny);
    const int a2blocks = (a2warps + 3) / 4;
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
        const bool kept = seg >= seg_kept;
        auto state = [&](int kk, int f) -> float* {  // u, v, w of X^{seg*K + kk}
            if (kk == 0) return w->ckpt[(size_t)seg * nstate + f];
            if (kept) {
                float* x[3];
                big_slot(seg, kk, x);
                return x[f];
            }
            return w->stash[(size_t)kk * 3 + f];
        };
        if (!kept && len > 1) {
            // recompute X^{seg K + 1 .. seg K + len - 1} into the stash
            float* in[6] = {state(0, 0), state(0, 1), state(0, 2),
                            kahan ? w->ckpt[(size_t)seg * nstate + 3] : nullptr,
                            kahan ? w->ckpt[(size_t)seg * nstate + 4] : nullptr,
                            kahan ? w->ckpt[(size_t)seg * nstate + 5] : nullptr};
            float* tmp[3];
            auto slot = [&](int kk) -> float* const* {
                tmp[0] = w->stash[(size_t)kk * 3 + 0];
                tmp[1] = w->stash[(size_t)kk * 3 + 1];
                tmp[2] = w->stash[(size_t)kk * 3 + 2];
                return tmp;
            };
            e = passes(in, len - 1, slot, nullptr);
        }
        // reverse sweep of the segment: an odd first step alone, then pairs of
        // steps (kk, kk - 1) in one two-level pass
        int kr = len - 1;
        auto single = [&](int k1) {
            AdjArgs a;
            a.u = state(k1, 0); a.v = state(k1, 1); a.w = state(k1, 2);
            a.lu = w->lam[lb][0]; a.lv = w->lam[lb][1]; a.lw = w->lam[lb][2];
            a.clu = w->lam[lb][3]; a.clv = w->lam[lb][4]; a.clw = w->lam[lb][5];
            a.luo = w->lam[lb ^ 1][0]; a.lvo = w->lam[lb ^ 1][1]; a.lwo = w->lam[lb ^ 1][2];
            a.cluo = w->lam[lb ^ 1][3]; a.clvo = w->lam[lb ^ 1][4]; a.clwo = w->lam[lb ^ 1][5];
            a.ax = s->a32[0]; a.b = s->a32[1]; a.ay = s->a32[2];
            a.g11 = w->g32[0]; a.g12 = w->g32[1]; a.g22 = w->g32[2];
            a.partials = w->partials;
            a.nx = s->nx; a.ny = s->ny; a.pitch = s->pitch;
            if (kahan) adjoint_step_kernel<true><<<ablocks, 128, 0, st>>>(a, r, aH, astrips, awarps);
            else adjoint_step_kernel<false><<<ablocks, 128, 0, st>>>(a, r, aH, astrips, awarps);
            lb ^= 1;
            since_flush += 1;
            return cudaGetLastError();
        };
        auto pair = [&](int k1) {  // steps k1 and k1 - 1
            AdjArgs2 a;
            a.u1 = state(k1, 0); a.v1 = state(k1, 1); a.w1 = state(k1, 2);
            a.u0 = state(k1 - 1, 0); a.v0 = state(k1 - 1, 1); a.w0 = state(k1 - 1, 2);
            a.lu = w->lam[lb][0]; a.lv = w->lam[lb][1]; a.lw = w->lam[lb][2];
            a.clu = w->lam[lb][3]; a.clv = w->lam[lb][4]; a.clw = w->lam[lb][5];
            a.luo = w->lam[lb ^ 1][0]; a.lvo = w->lam[lb ^ 1][1]; a.lwo = w->lam[lb ^ 1][2];
            a.cluo = w->lam[lb ^ 1][3]; a.clvo = w->lam[lb ^ 1][4]; a.clwo = w->lam[lb ^ 1][5];
            a.ax = s->a32[0]; a.b = s->a32[1]; a.ay = s->a32[2];
            a.g11 = w->g32[0]; a.g12 = w->g32[1]; a.g22 = w->g32[2];
            a.partials = w->partials;
            a.nx = s->nx; a.ny = s->ny; a.pitch = s->pitch;
            if (kahan) adjoint2_kernel<true><<<a2blocks, 128, 0, st>>>(a, r, a2H, a2strips, a2warps);
            else adjoint2_kernel<false><<<a2blocks, 128, 0, st>>>(a, r, a2H, a2strips, a2warps);
            lb ^= 1;
            since_flush += 2;
            return cudaGetLastError();
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
