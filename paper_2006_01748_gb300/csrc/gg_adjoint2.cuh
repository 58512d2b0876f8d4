#pragma once
// Adjoint step of eq. (3) in paired columns: lane l of a warp owns the
// column pair (a, b) = (x0 + 2l, x0 + 2l + 1) of a 64-column strip and every
// quantity is a float2 over that pair (one packed FP32 instruction for two
// cells; one shuffle per pair for an east or west neighbour).  Per cell it
// evaluates the reverse step written out at the top of gg_adjoint.cu: the
// gather form of J(X)^T from the face fluxes of Tables 1 and 2, the
// transposed mirrored central differences of the a12 cross terms, the
// per-cell tensor-gradient increments and the four rate terms.  It is
// written with explicit packed round-to-nearest intrinsics throughout, so
// that the one-step and two-step marches below give the same bits per cell.
//
// Rows stream through a per-warp shared-memory ring filled with cp.async,
// one row ahead, each lane copying and reading back only its own pair (no
// barrier).  A ring slot holds one input row (the stored state X^k, the
// incoming lambda with its Kahan terms, the tensor weights) and the per-cell
// gradient sums of the row written at the tick that consumes the slot.  A level reads its own and
// north rows from the ring instead of keeping them in registers.
#include "gg_stepw2.cuh"

namespace gg {
namespace adjw {

using stepw2::add2;
using stepw2::dup;
using stepw2::east_of;
using stepw2::fma2;
using stepw2::mul2;
using stepw2::sub2;
using stepw2::west_of;

__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }

// Fields of one row that a level reads on its own row and its north row.
struct Row {
    float2 u, v, w, lv, lw, clv, clw, b, ay;
};
// What one level passes from row q-1 to row q.  The level reads row q+1 as
// its north row when it processes row q; at the next tick that row is its
// own row.  So the x-face differences of lamW and the cross sums of a row are
// computed once, when it is the north row, and every south-face term of row q
// is the north-face term of row q-1 (of equal value, or of opposite sign where
// the difference changes direction: it is kept with the sign of the north
// face and subtracted).
struct Carry {
    float2 LxE, LxW;  // lamW differences across the east / west faces of row q
    float2 Sx, SxS;   // b (LxE + LxW) of rows q and q-1
    float2 Ly;        // lamW difference across the north face of row q-1
    float2 f, e, g, qq;  // north-face terms of row q-1 (adj_level2)
};
// Result of one level at one pair: lambda at step k with Kahan terms, the
// tensor-gradient increments (dt included) and the four rate terms.
struct Out {
    float2 lu, clu, lv, clv, lw, clw;
    float2 d11, d12, d22;
    float2 s_delta, s_rho, s_D, s_c;
};
// Boundary flags of the pair's two columns (EDGE variants).
struct Mask {
    bool wa, wb, ea, eb;
};
// Scalars of the reverse step as pairs.
struct K2 {
    float2 dt, D, ndelta, rho, c, nc, ihx2, ihy2, dtkx, dtky, dtkc;
    int no_reaction;
};
__device__ __forceinline__ K2 make_k2(const Rates32& k)
{
    K2 r;
    r.dt = dup(k.dt);
    r.D = dup(k.D);
    r.ndelta = dup(-k.delta);
    r.rho = dup(k.rho);
    r.c = dup(k.c);
    r.nc = dup(-k.c);
    r.ihx2 = dup(k.ihx2);
    r.ihy2 = dup(k.ihy2);
    r.dtkx = dup(__fmul_rn(k.dt, k.kx));
    r.dtky = dup(__fmul_rn(k.dt, k.ky));
    r.dtkc = dup(__fmul_rn(k.dt, k.kc));
    r.no_reaction = k.no_reaction;
    return r;
}

template <bool EDGE>
__device__ __forceinline__ void mask_e(float2& x, float2 y, const Mask& m)
{
    if (EDGE) {
        if (!m.ea) x.x = y.x;
        if (!m.eb) x.y = y.y;
    }
}
template <bool EDGE>
__device__ __forceinline__ void mask_w(float2& x, float2 y, const Mask& m)
{
    if (EDGE) {
        if (!m.wa) x.x = y.x;
        if (!m.wb) x.y = y.y;
    }
}

// One reverse step at row q of a pair, from the rows P (q) and N (q+1), w of
// row q-1, the own-row lamU (with Kahan term) and east-face weight ax, and
// the carry of row q-1 (updated for row q+1).  All lanes call it.  Face
// terms, each with the factor 1/h^2 of its direction: with
// m = 1 - (U_P + U_nb)/2, dv = V_nb - V_P and dl the compensated difference
// of lamV (neighbour minus own),
//   f = m dl (D1^T of lamV),  e = dv dl (dD1/dU);
// the east / north terms are computed here, the west ones are the west
// neighbour's east ones and the south ones the carried north ones of row
// q-1:  D1^T = (fE - fW) + (fN - fS),  dD1/dU = (eE + eW + eN + eS) / 2.
// The rate term of D, sum_cells lamV D1(V; U), is taken in its transposed
// form sum_cells V D1^T(lamV; U): D1(.; U) is a symmetric matrix (Table 1's
// face fluxes with zero flux through boundary faces), so the two sums are
// equal, and the second needs no second difference of the FP32 state V but
// only the compensated differences of lamV.
template <bool KAHAN, bool EDGE, bool YEDGE>
__device__ __forceinline__ Out adj_level2(const K2& k, float2 Sw, const Row& P, const Row& N, float2 lu, float2 clu,
                                          float2 ax, const Mask& m, bool hasS_, bool hasN_, Carry& c)
{
    const bool hasS = YEDGE ? hasS_ : true, hasN = YEDGE ? hasN_ : true;
    const float2 z = make_float2(0.0f, 0.0f), one = dup(1.0f);
    // compensated difference of lambda between two (value, Kahan term) pairs
    auto dW = [](float2 la, float2 ca, float2 lb, float2 cb) { return sub2(sub2(la, lb), sub2(ca, cb)); };
    // x-face differences of lamW on the north row (0 on boundary faces)
    float2 LxE_N = dW(N.lw, N.clw, east_of(N.lw), east_of(N.clw));
    mask_e<EDGE>(LxE_N, z, m);
    float2 LxW_N = west_of(LxE_N);
    mask_w<EDGE>(LxW_N, z, m);
    const float2 LxE_P = c.LxE, LxW_P = c.LxW;
    const float2 LyN = hasN ? dW(P.lw, P.clw, N.lw, N.clw) : z;
    const float2 LyS = hasS ? c.Ly : z;
    // transpose of the a12 cross terms (b carries 1/(4 dx dy))
    const float2 SxN = mul2(N.b, add2(LxE_N, LxW_N)), SxP = c.Sx, SxS = c.SxS;
    const float2 SyP = mul2(P.b, add2(LyN, LyS));
    const float2 SyE = east_of(SyP), SyW = west_of(SyP);
    // Ty = S_{q-1}[q>=1] - S_{q+1}[q<=ny-2] + S_q([q=ny-1] - [q=0]), Tx likewise
    float2 Ty = sub2(hasS ? SxS : z, hasN ? SxN : z);
    if (YEDGE) {
        if (!hasN) Ty = add2(Ty, SxP);
        if (!hasS) Ty = sub2(Ty, SxP);
    }
    float2 Tx;
    if (EDGE) {
        Tx.x = __fsub_rn(m.wa ? SyW.x : 0.0f, m.ea ? SyE.x : 0.0f);
        if (!m.ea) Tx.x = __fadd_rn(Tx.x, SyP.x);
        if (!m.wa) Tx.x = __fsub_rn(Tx.x, SyP.x);
        Tx.y = __fsub_rn(m.wb ? SyW.y : 0.0f, m.eb ? SyE.y : 0.0f);
        if (!m.eb) Tx.y = __fadd_rn(Tx.y, SyP.y);
        if (!m.wb) Tx.y = __fsub_rn(Tx.y, SyP.y);
    } else {
        Tx = sub2(SyW, SyE);
    }
    // face weights: east ax, west the west neighbour's ax, north P.ay, south
    // the carried product of row q-1 (a boundary face has L = 0)
    const float2 axW = west_of(ax);
    const float2 gN = mul2(P.ay, LyN);
    const float2 D2T = add2(add2(fma2(axW, LxW_P, mul2(ax, neg2(LxE_P))), sub2(hasS ? c.g : z, gN)), add2(Tx, Ty));

    // state and lamV neighbourhood (mirrored at the boundary)
    float2 uE = east_of(P.u), vE = east_of(P.v), wE = east_of(P.w), wW = west_of(P.w);
    float2 lvE = east_of(P.lv), cvE = east_of(P.clv);
    mask_e<EDGE>(uE, P.u, m);
    mask_e<EDGE>(vE, P.v, m);
    mask_e<EDGE>(wE, P.w, m);
    mask_e<EDGE>(lvE, P.lv, m);
    mask_e<EDGE>(cvE, P.clv, m);
    mask_w<EDGE>(wW, P.w, m);
    const float2 uN = hasN ? N.u : P.u, vN = hasN ? N.v : P.v, wN = hasN ? N.w : P.w;
    const float2 wS = hasS ? Sw : P.w;
    const float2 nhalf = dup(-0.5f);
    const float2 mE = fma2(nhalf, add2(P.u, uE), one), mN = fma2(nhalf, add2(P.u, uN), one);
    const float2 dvE = mul2(sub2(vE, P.v), k.ihx2), dvN = mul2(sub2(vN, P.v), k.ihy2);
    const float2 dlE = dW(lvE, cvE, P.lv, P.clv), dlN = hasN ? dW(N.lv, N.clv, P.lv, P.clv) : z;
    const float2 fE = mul2(mul2(mE, dlE), k.ihx2), eE = mul2(dvE, dlE);
    const float2 fN = mul2(mul2(mN, dlN), k.ihy2), eN = mul2(dvN, dlN);
    float2 fW = west_of(fE), eW = west_of(eE);
    mask_w<EDGE>(fW, z, m);
    mask_w<EDGE>(eW, z, m);
    const float2 fS = hasS ? c.f : z, eS = hasS ? c.e : z;
    const float2 d1T = add2(sub2(fE, fW), sub2(fN, fS));
    const float2 dU = mul2(dup(0.5f), add2(add2(eE, eW), add2(eN, eS)));

    float2 fu, fvv, fw;
    Out o;
    if (k.no_reaction) {
        fu = mul2(k.D, dU);
        fvv = mul2(k.D, d1T);
        fw = D2T;
        o.s_delta = o.s_rho = o.s_c = z;
    } else {
        const float2 m2 = dup(-2.0f);
        // (1 - 2U - delta W) lamU + D dU
        fu = fma2(fma2(k.ndelta, P.w, fma2(m2, P.u, one)), lu, mul2(k.D, dU));
        // rho (1 - 2V) lamV + D D1^T + c lamW
        fvv = fma2(mul2(k.rho, fma2(m2, P.v, one)), P.lv, fma2(k.D, d1T, mul2(k.c, P.lw)));
        // -delta U lamU - c lamW + D2^T
        fw = fma2(mul2(k.ndelta, P.u), lu, fma2(k.nc, P.lw, D2T));
        o.s_delta = mul2(mul2(neg2(lu), P.u), P.w);
        o.s_rho = mul2(mul2(P.lv, P.v), sub2(one, P.v));
        o.s_c = mul2(P.lw, sub2(P.v, P.w));
    }
    // the rate term of D in its transposed form V D1^T(lamV)
    o.s_D = mul2(P.v, d1T);
    if (KAHAN) {
        // x' = x + y, comp' = (x' - x) - y with y = dt f - comp
        auto kadd = [&](float2 x, float2 f, float2 cx, float2& xo, float2& co) {
            const float2 y = fma2(k.dt, f, neg2(cx));
            const float2 t = add2(x, y);
            co = sub2(sub2(t, x), y);
            xo = t;
        };
        kadd(lu, fu, clu, o.lu, o.clu);
        kadd(P.lv, fvv, P.clv, o.lv, o.clv);
        kadd(P.lw, fw, P.clw, o.lw, o.clw);
    } else {
        o.lu = fma2(k.dt, fu, lu);
        o.lv = fma2(k.dt, fvv, P.lv);
        o.lw = fma2(k.dt, fw, P.lw);
        o.clu = o.clv = o.clw = z;
    }
    const float2 qN = mul2(sub2(wN, P.w), LyN);
    o.d11 = mul2(k.dtkx, fma2(sub2(wE, P.w), LxE_P, mul2(sub2(P.w, wW), LxW_P)));
    o.d22 = mul2(k.dtky, add2(qN, hasS ? c.qq : z));
    o.d12 = mul2(k.dtkc, fma2(add2(LxE_P, LxW_P), sub2(wN, wS), mul2(add2(LyN, LyS), sub2(wE, wW))));
    // row q becomes row q-1 of the next tick
    c.LxE = LxE_N;
    c.LxW = LxW_N;
    c.SxS = SxP;
    c.Sx = SxN;
    c.Ly = LyN;
    c.f = fN;
    c.e = eN;
    c.g = gN;
    c.qq = qN;
    return o;
}

// Per-lane FP32 compensated sums of the four rate terms over the lane's
// pairs (the two columns kept apart until the fold), folded into one FP64
// record per warp in a fixed order.  delta, rho and c use Kahan's update;
// the D term, V D1^T(lamV), sums to a small fraction of the sum of its
// magnitudes (D1^T(lamV) sums to zero over the domain), so it keeps the exact
// rounding error of every addition (TwoSum) in the second accumulator (as
// -accc, so that the fold acc - accc serves both kinds of sum).
struct RateSums2 {
    float2 acc[4], accc[4];
    __device__ __forceinline__ RateSums2()
    {
        for (int q = 0; q < 4; ++q) acc[q] = accc[q] = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void add(int q, float2 x)
    {
        const float2 y = sub2(x, accc[q]);
        const float2 t = add2(acc[q], y);
        accc[q] = sub2(sub2(t, acc[q]), y);
        acc[q] = t;
    }
    __device__ __forceinline__ void add_two_sum(int q, float2 x)
    {
        const float2 s = add2(acc[q], x);
        const float2 z = sub2(s, acc[q]);
        const float2 e = add2(sub2(acc[q], sub2(s, z)), sub2(x, z));
        accc[q] = sub2(accc[q], e);
        acc[q] = s;
    }
    // a lane outside the chunk's columns adds zeros: an exact no-op for the D
    // sum; for the others it folds the running compensation in, which leaves
    // the sum within its rounding.  Unlike a branch around add_all it keeps
    // the four terms from staying live across the code that follows.
    __device__ __forceinline__ void add_all_masked(const Out& o, bool on)
    {
        const float2 z = make_float2(0.0f, 0.0f);
        add(0, on ? o.s_delta : z);
        add(1, on ? o.s_rho : z);
        add_two_sum(2, on ? o.s_D : z);
        add(3, on ? o.s_c : z);
    }
    __device__ __forceinline__ void add_all(const Out& o)
    {
        add(0, o.s_delta);
        add(1, o.s_rho);
        add_two_sum(2, o.s_D);
        add(3, o.s_c);
    }
    // one FP64 record per warp: part[q] += dt * sum over lanes (fixed order)
    __device__ __forceinline__ void fold(double* part, int lane, float dt)
    {
        double s4[4];
        for (int q = 0; q < 4; ++q) {
            s4[q] = ((double)acc[q].x - (double)accc[q].x) + ((double)acc[q].y - (double)accc[q].y);
            for (int off = 16; off > 0; off >>= 1) s4[q] += __shfl_xor_sync(0xffffffffu, s4[q], off);
        }
        if (lane == 0)
            for (int q = 0; q < 4; ++q) part[q] += (double)dt * s4[q];
    }
};

// Ring geometry: row r of the march in slot r & (kSlots - 1); rows r - 2 ..
// r + kAhead are live at tick r.
constexpr int kAhead = 1;
constexpr int kSlots = 4;
// Fields of a slot (float2 rows of 32 lanes): the input row (state, incoming
// lambda with its Kahan terms, tensor weights), then the gradient sums of the
// row written when the slot is consumed.
enum : int {
    F_U = 0, F_V, F_W, F_LU, F_LV, F_LW, F_CLU, F_CLV, F_CLW, F_AX, F_B, F_AY,
    F_G11, F_G12, F_G22,
    F_COUNT
};
constexpr int kRingBytes = kSlots * F_COUNT * 32 * 8;

__device__ __forceinline__ void cp_async8(uint32_t dst, const float* src, int bytes)
{
    stepw2::cp_async8(dst, src, bytes);
}

// Pointers of one reverse pass: the stored state X^k in (u, v, w), the
// incoming lambda (lambda^{k+1} for one step, lambda^{k+2} for two) in
// (lu ... clw), the outgoing lambda^k in (luo ...).
struct PassArgs {
    const float *u, *v, *w;
    const float *lu, *lv, *lw, *clu, *clv, *clw;
    float *luo, *lvo, *lwo, *cluo, *clvo, *clwo;
    const float *ax, *b, *ay;
    float *g11, *g12, *g22;
    double* partials;
    int nx, ny, pitch;
};

// Strip geometry of the marches: STEPS = 1 reverse level (halo 1, rounded up
// to a pair), STEPS = 2 the forward level and two reverse levels (halo 3).
template <int STEPS> struct Geom {
    static constexpr int HLP = STEPS == 1 ? 2 : 4;
    static constexpr int OUT = 64 - 2 * HLP;
};

// What the forward level passes from one row to the next (the carries of
// gg_stepw2.cuh's march): the north faces of the previous row and the east w
// and y cross term of the own row.
struct FwdCarry {
    float2 G, H, WE, Z;
};

// One explicit Euler step of eq. (3) at row q of a pair, without Kahan terms:
// the face fluxes of Tables 1 and 2 from rows q (P) and q+1 (N) and w of row
// q-1, as in gg_stepw2.cuh.  It rebuilds the state X^{k+1} of the step the
// two-level reverse march needs from the stored X^k; the rebuilt state
// differs from the forward pass's compensated one by the last rounding only.
template <bool EDGE, bool YEDGE>
__device__ __forceinline__ void fwd_level(const Rates32& k, float2 bP, float2 bN, float2 ax, float2 ay, float2 u,
                                          float2 v, float2 w, float2 un, float2 vn, float2 wn, float2 wS,
                                          FwdCarry& c, const Mask& m, bool hasS_, bool hasN_, float2& uo,
                                          float2& vo, float2& wo)
{
    const bool hasS = YEDGE ? hasS_ : true, hasN = YEDGE ? hasN_ : true;
    const float2 z = make_float2(0.0f, 0.0f), one = dup(1.0f);
    // x cross term of the own row (tangential difference mirrored at the south / north boundary)
    const float2 zxP = mul2(bP, sub2(hasN ? wn : w, hasS ? wS : w));
    float2 uE = east_of(u), vE = east_of(v), wNE = east_of(wn), wNW = west_of(wn);
    const float2 zxE = east_of(zxP);
    mask_e<EDGE>(uE, u, m);
    mask_e<EDGE>(vE, v, m);
    mask_e<EDGE>(wNE, wn, m);
    mask_w<EDGE>(wNW, wn, m);
    const float2 wE = c.WE;
    c.WE = wNE;
    const float2 zyP = c.Z, zyN = mul2(bN, sub2(wNE, wNW));
    c.Z = zyN;
    // east and north faces: acid a (W_R - W_L) + (z_L + z_R), tumour (K - K/2 (U_L + U_R)) (V_R - V_L)
    float2 gE = fma2(ax, sub2(wE, w), add2(zxP, zxE));
    float2 hE = mul2(fma2(dup(-k.hKx), add2(u, uE), dup(k.Kx)), sub2(vE, v));
    float2 gN = fma2(ay, sub2(wn, w), add2(zyP, zyN));
    float2 hN = mul2(fma2(dup(-k.hKy), add2(u, un), dup(k.Ky)), sub2(vn, v));
    mask_e<EDGE>(gE, z, m);
    mask_e<EDGE>(hE, z, m);
    if (!hasN) { gN = z; hN = z; }
    float2 gW = west_of(gE), hW = west_of(hE);
    mask_w<EDGE>(gW, z, m);
    mask_w<EDGE>(hW, z, m);
    const float2 gS = hasS ? c.G : z, hS = hasS ? c.H : z;
    c.G = gN;
    c.H = hN;
    const float2 d1 = add2(sub2(hE, hW), sub2(hN, hS));
    const float2 d2 = add2(sub2(gE, gW), sub2(gN, gS));
    float2 fu, fv, fw;
    if (k.no_reaction) {
        fu = z;
        fv = d1;
        fw = d2;
    } else {
        fu = mul2(u, fma2(dup(-k.delta), w, sub2(one, u)));
        fv = fma2(mul2(dup(k.rho), v), sub2(one, v), d1);
        fw = fma2(dup(k.c), sub2(v, w), d2);
    }
    const float2 dt = dup(k.dt);
    uo = fma2(dt, fu, u);
    vo = fma2(dt, fv, v);
    wo = fma2(dt, fw, w);
}

// Shared helpers of the marches: the slot of row r, the copy of one input
// row (and of the gradient sums of output row qg) into it, and the store of
// an output row.
struct RingIO {
    float2* rl;  // this lane's entry of slot 0
    const float* src[12];
    int cpb;
    size_t coff;
    __device__ __forceinline__ float2* slot(int r) const { return rl + (r & (kSlots - 1)) * F_COUNT * 32; }
};

template <bool KAHAN>
__device__ __forceinline__ void fetch_row(const RingIO& io, const PassArgs& a, int r, int qg, bool copy_in,
                                          bool copy_g, int ny, int pitch, int ca)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(io.slot(r));
    if (copy_in) {
        const bool in = r >= 0 && r < ny;  // zeros outside the domain
        const size_t o = (size_t)(in ? r : 0) * pitch + io.coff;
#pragma unroll
        for (int f = 0; f < 12; ++f) {
            if (!KAHAN && (f == F_CLU || f == F_CLV || f == F_CLW)) continue;
            cp_async8(d + f * 256, io.src[f] + o, in ? io.cpb : 0);
        }
    }
    if (copy_g) {
        const size_t og = (size_t)qg * pitch + ca;
        cp_async8(d + F_G11 * 256, a.g11 + og, io.cpb);
        cp_async8(d + F_G12 * 256, a.g12 + og, io.cpb);
        cp_async8(d + F_G22 * 256, a.g22 + og, io.cpb);
    }
    stepw2::cp_async_commit();
}

template <bool KAHAN, bool EDGE>
__device__ __forceinline__ void store_row(const PassArgs& a, const Out& o, float2 g11, float2 g12, float2 g22,
                                          size_t off, bool b_in)
{
    if (!EDGE || b_in) {
        *reinterpret_cast<float2*>(a.luo + off) = o.lu;
        *reinterpret_cast<float2*>(a.lvo + off) = o.lv;
        *reinterpret_cast<float2*>(a.lwo + off) = o.lw;
        if (KAHAN) {
            *reinterpret_cast<float2*>(a.cluo + off) = o.clu;
            *reinterpret_cast<float2*>(a.clvo + off) = o.clv;
            *reinterpret_cast<float2*>(a.clwo + off) = o.clw;
        }
        *reinterpret_cast<float2*>(a.g11 + off) = g11;
        *reinterpret_cast<float2*>(a.g12 + off) = g12;
        *reinterpret_cast<float2*>(a.g22 + off) = g22;
    } else {
        a.luo[off] = o.lu.x; a.lvo[off] = o.lv.x; a.lwo[off] = o.lw.x;
        if (KAHAN) { a.cluo[off] = o.clu.x; a.clvo[off] = o.clv.x; a.clwo[off] = o.clw.x; }
        a.g11[off] = g11.x; a.g12[off] = g12.x; a.g22[off] = g22.x;
    }
}

__device__ __forceinline__ Row ring_row(const float2* s, bool kahan)
{
    Row x;
    x.u = s[F_U * 32]; x.v = s[F_V * 32]; x.w = s[F_W * 32];
    x.lv = s[F_LV * 32]; x.lw = s[F_LW * 32];
    if (kahan) { x.clv = s[F_CLV * 32]; x.clw = s[F_CLW * 32]; }
    else { x.clv = x.clw = make_float2(0.0f, 0.0f); }
    x.b = s[F_B * 32]; x.ay = s[F_AY * 32];
    return x;
}

// One reverse step as a warp march (STEPS = 1): the level computes row r - 1
// at tick r from input rows r - 1 and r of the ring (lambda^{k+1}, the stored
// X^k, the tensor); the march starts two rows above its first written row so
// that the carries of that row are complete.
//
// Two reverse steps (STEPS = 2, steps k + 1 and k from the stored X^k and
// lambda^{k+2}): at tick r the forward level F rebuilds row r - 1 of X^{k+1}
// from rows r - 2 .. r of X^k, level A1 computes row r - 2 of lambda^{k+1}
// from X^{k+1} (rows r - 3 .. r - 1, kept in registers) and lambda^{k+2}
// (rows r - 2, r - 1 of the ring), level A2 row r - 3 of lambda^k from X^k
// (rows r - 4 .. r - 2) and A1's lambda^{k+1}; so only every other state is
// stored, and of the two states of the step pair only X^k crosses HBM.  Rows
// that a level has moved past stay in registers (the tensor and X^k rows of
// A2, the X^{k+1} rows of A1), so the ring holds rows r - 2 .. r + 1 only.
template <int STEPS, bool KAHAN, bool EDGE, bool YEDGE>
__device__ __forceinline__ void march(const PassArgs& a, const Rates32& kr, const int H, const int strip,
                                      const int chunk, const int lane, float2* ring, double* part)
{
    static_assert(STEPS == 1 || STEPS == 2, "one or two reverse steps");
    const K2 k = make_k2(kr);
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    constexpr int HLP = Geom<STEPS>::HLP, OUT = Geom<STEPS>::OUT;
    const int ca = strip * OUT - HLP + 2 * lane;
    const int cb = ca + 1;
    const bool ld_ok = EDGE ? (ca >= 0 && ca < nx) : true;
    const bool b_in = EDGE ? (ca >= 0 && cb < nx) : true;
    const Mask m{EDGE ? ca > 0 : true, EDGE ? cb > 0 : true, EDGE ? ca + 1 < nx : true, EDGE ? cb + 1 < nx : true};
    const bool outc = lane >= HLP / 2 && lane < 32 - HLP / 2 && ld_ok;
    const int ys = chunk * H;
    const int ye = min(ny, ys + H);
    // the written row of tick r is r - STEPS - (STEPS == 2): r - 1 or r - 3
    constexpr int LAG = STEPS == 1 ? 1 : 3;
    const int r0 = STEPS == 1 ? max(0, ys - 1) : max(0, ys - 2);
    const int r1 = ye + LAG;  // one past the last tick

    RingIO io;
    io.rl = ring + lane;
    io.cpb = !EDGE ? 8 : (!ld_ok ? 0 : (b_in ? 8 : 4));
    io.coff = ld_ok ? (size_t)ca : 0;
    const float* src[12] = {a.u, a.v, a.w, a.lu, a.lv, a.lw, a.clu, a.clv, a.clw, a.ax, a.b, a.ay};
#pragma unroll
    for (int f = 0; f < 12; ++f) io.src[f] = src[f];
    auto fetch = [&](int r) {
        const int qg = r - LAG;
        fetch_row<KAHAN>(io, a, r, qg, r < r1, r < r1 && qg >= ys && qg < ye && outc, ny, pitch, ca);
    };

    const float2 z = make_float2(0.0f, 0.0f);
    RateSums2 sums;
    Carry c1{z, z, z, z, z, z, z, z, z}, c2{z, z, z, z, z, z, z, z, z};
    FwdCarry cf{z, z, z, z};
    float2 S1w = z;  // STEPS 1: w of row r - 2; STEPS 2: X^{k+1} w of row r - 3
    // STEPS 2: X^{k+1} of row r - 2 (F's last output), X^k of rows r - 3 and
    // w of r - 4, lambda^{k+1} of row r - 3, tensor rows of A1 (r - 2) and A2
    // (r - 3), A1's increments of row r - 3
    float2 xuP = z, xvP = z, xwP = z;
    float2 u0P = z, v0P = z, w0P = z, S2w = z;
    float2 lvP = z, lwP = z, clvP = z, clwP = z, luP = z, cluP = z;
    float2 ax2 = z, b2 = z, ay2 = z;
    float2 d11c = z, d12c = z, d22c = z;

    // rows r0 - 2 .. r0 + kAhead - 1 in flight before the first tick
#pragma unroll
    for (int i = -2; i < kAhead; ++i) fetch(r0 + i);
    for (int r = r0; r < r1; ++r) {
        fetch(r + kAhead);
        stepw2::cp_async_wait<kAhead>();  // rows up to r have landed
        const float2* s0 = io.slot(r);
        const float2* s1 = io.slot(r - 1);
        Out o;
        int qw;
        float2 dc1 = z, dc2 = z, dc3 = z;
        if constexpr (STEPS == 1) {
            const Row P = ring_row(s1, KAHAN), N = ring_row(s0, KAHAN);
            const float2 lu = s1[F_LU * 32], clu = KAHAN ? s1[F_CLU * 32] : z, ax = s1[F_AX * 32];
            const int q = r - 1;
            o = adj_level2<KAHAN, EDGE, YEDGE>(k, S1w, P, N, lu, clu, ax, m, q > 0, q + 1 < ny, c1);
            S1w = P.w;
            qw = q;
        } else {
            const float2* s2 = io.slot(r - 2);
            // F: row r - 1 of X^{k+1} from X^k rows r - 2 (w), r - 1, r
            const float2 axF = s1[F_AX * 32], bF = s1[F_B * 32], ayF = s1[F_AY * 32], bNF = s0[F_B * 32];
            float2 xu, xv, xw;
            const int qf = r - 1;
            fwd_level<EDGE, YEDGE>(kr, bF, bNF, axF, ayF, s1[F_U * 32], s1[F_V * 32], s1[F_W * 32], s0[F_U * 32],
                                   s0[F_V * 32], s0[F_W * 32], s2[F_W * 32], cf, m, qf > 0, qf + 1 < ny, xu, xv,
                                   xw);
            // A1: row r - 2 of lambda^{k+1} (step k + 1, state X^{k+1})
            const int q1 = r - 2;
            Row P1, N1;
            P1.u = xuP; P1.v = xvP; P1.w = xwP;
            P1.lv = s2[F_LV * 32]; P1.lw = s2[F_LW * 32];
            if (KAHAN) { P1.clv = s2[F_CLV * 32]; P1.clw = s2[F_CLW * 32]; }
            else { P1.clv = P1.clw = z; }
            const float2 ax1 = s2[F_AX * 32], b1 = s2[F_B * 32], ay1 = s2[F_AY * 32];
            P1.b = b1; P1.ay = ay1;
            N1.u = xu; N1.v = xv; N1.w = xw;
            N1.lv = s1[F_LV * 32]; N1.lw = s1[F_LW * 32];
            if (KAHAN) { N1.clv = s1[F_CLV * 32]; N1.clw = s1[F_CLW * 32]; }
            else { N1.clv = N1.clw = z; }
            N1.b = bF; N1.ay = ayF;
            const float2 lu1 = s2[F_LU * 32], clu1 = KAHAN ? s2[F_CLU * 32] : z;
            const Out o1 = adj_level2<KAHAN, EDGE, YEDGE>(k, S1w, P1, N1, lu1, clu1, ax1, m, q1 > 0, q1 + 1 < ny, c1);
            // A1's rate terms count where its row is the chunk's
            if (q1 >= ys && q1 < ye) sums.add_all_masked(o1, outc);
            // A2: row r - 3 of lambda^k (step k, state X^k)
            const int q2 = r - 3;
            Row P2, N2;
            P2.u = u0P; P2.v = v0P; P2.w = w0P;
            P2.lv = lvP; P2.lw = lwP; P2.clv = clvP; P2.clw = clwP;
            P2.b = b2; P2.ay = ay2;
            N2.u = s2[F_U * 32]; N2.v = s2[F_V * 32]; N2.w = s2[F_W * 32];
            N2.lv = o1.lv; N2.lw = o1.lw; N2.clv = o1.clv; N2.clw = o1.clw;
            N2.b = b1; N2.ay = ay1;
            o = adj_level2<KAHAN, EDGE, YEDGE>(k, S2w, P2, N2, luP, cluP, ax2, m, q2 > 0, q2 + 1 < ny, c2);
            qw = q2;
            dc1 = d11c; dc2 = d12c; dc3 = d22c;
            // rows move on: F's row r - 1 becomes A1's own row, X^k row r - 2
            // and A1's lambda row r - 2 become A2's own row
            S1w = xwP; xuP = xu; xvP = xv; xwP = xw;
            S2w = w0P; u0P = N2.u; v0P = N2.v; w0P = N2.w;
            lvP = o1.lv; lwP = o1.lw; clvP = o1.clv; clwP = o1.clw; luP = o1.lu; cluP = o1.clu;
            ax2 = ax1; b2 = b1; ay2 = ay1;
            d11c = o1.d11; d12c = o1.d12; d22c = o1.d22;
        }
        if (qw >= ys && qw < ye && outc) {
            sums.add_all(o);
            const size_t off = (size_t)qw * pitch + ca;
            const float2 g11 = add2(s0[F_G11 * 32], add2(dc1, o.d11));
            const float2 g12 = add2(s0[F_G12 * 32], add2(dc2, o.d12));
            const float2 g22 = add2(s0[F_G22 * 32], add2(dc3, o.d22));
            store_row<KAHAN, EDGE>(a, o, g11, g12, g22, off, b_in);
        }
    }
    stepw2::cp_async_wait<0>();  // nothing in flight when the warp leaves
    sums.fold(part, lane, kr.dt);
}

}  // namespace adjw
}  // namespace gg
