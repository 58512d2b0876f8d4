#pragma once
// FP32 step of eq. (3) as a warp-register wavefront (T = 1..4 steps per pass).
//
// Each warp owns a strip of 32 consecutive columns and a chunk of rows.  Lane
// l holds column x0 + l; east / west values come from the adjacent lanes with
// warp shuffles, so there is no shared memory and no block barrier.  The warp
// streams the rows of its chunk (plus T halo rows on each side) from HBM once
// per pass, two rows ahead of use, and keeps in registers, per time level
// t < T, the rows q-1 (w only), q and q+1 of (u, v, w) and two rows of Kahan
// terms; the tensor entries keep the last T+1 input rows.  At tick k the
// input row R = lo0 + k enters level 0 and level t = 1..T computes row R - t
// from level t-1 (a wavefront lagging one row per level).
//
// Each lane computes the east and north face fluxes of its cell once
// (gg_math.cuh); the west face is the east face of the lane to the west (one
// shuffle) and the south face is the north face the same level computed one
// tick earlier (a register).  Row q + 1, which level t reads as its north
// row at tick k, is its own row at tick k + 1: the east / west neighbours of
// w and the y cross term of that row are kept from one tick to the next
// instead of being exchanged again.  Level t is valid on lanes [t, 32 - t), so a
// warp writes its 32 - 2T middle columns and neighbouring strips overlap by
// 2T columns.  Warps that touch the west or east domain boundary run a
// variant with the boundary conditions; interior warps skip them.
#include <type_traits>

#include "gg_math.cuh"

namespace gg {
namespace stepw {

constexpr unsigned kFull = 0xffffffffu;

// Two floats without the pair alignment of float2: the one-step pass keeps
// its (u, v) windows in this form, so that the compiler allocates them as
// independent scalars.
struct F2 {
    float x, y;
};
template <typename V> __device__ __forceinline__ V mk2(float a, float b) { return V{a, b}; }

__device__ __forceinline__ float from_west(float x) { return __shfl_up_sync(kFull, x, 1); }
__device__ __forceinline__ float from_east(float x) { return __shfl_down_sync(kFull, x, 1); }

// State loads: COHERENT = false reads through the read-only cache (state
// written by an earlier launch); COHERENT = true bypasses L1, for the
// persistent ensemble kernel that reads state written by other CTAs of the
// same launch.
template <bool COHERENT>
__device__ __forceinline__ float ld_state(const float* p)
{
    if constexpr (COHERENT) return __ldcg(p);
    else return __ldg(p);
}

// EDGE: the strip touches the west or east domain boundary.  YEDGE: the
// chunk's rows (with their halo of T rows) touch the south or north boundary;
// interior chunks take every south / north face as present.
template <int T, bool KAHAN, bool EDGE, bool COHERENT = false, bool YEDGE = true>
__device__ __forceinline__ void warp_pass(const Grid32& g, const Rates32& k, const int H, const int strip,
                                          const int chunk, const int lane)
{
    constexpr int OUT = 32 - 2 * T;
    // packed FP32 pairs for T >= 2 (issue-bound); the one-step pass is
    // HBM-bound and keeps scalar code, which needs fewer registers
    constexpr bool PK = T >= 2;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const int gx = strip * OUT - T + lane;
    const bool ind = EDGE ? (gx >= 0 && gx < nx) : true;
    const bool hasW = EDGE ? gx > 0 : true;
    const bool hasE = EDGE ? gx + 1 < nx : true;
    const bool outc = ind && lane >= T && lane < 32 - T;
    const int ys = chunk * H;
    const int lo0 = max(0, ys - T);
    const int hi0 = min(ny, ys + H + T);
    const int hiT = min(ny, ys + H);
    const int nticks = hiT - lo0 + T;

    // windows of level t-1 used by level t, index t-1; u and v (and their
    // Kahan terms) as pairs for the packed arithmetic
    using V2 = typename std::conditional<PK, float2, F2>::type;
    V2 pUV[T], nUV[T], cPuv[T], cNuv[T];
    float sW[T], pW[T], nW[T], cPw[T], cNw[T];
    V2 cfA[T + 1];       // [age] (ax, ay); age a holds input row R - a
    float cfB[T + 1];    // [age] b
    float carG[T + 1], carH[T + 1];           // north faces of the previous tick
    float carWE[T + 1], carZ[T + 1];          // east w and y cross term of the own row
    const float2 dt2 = make_float2(k.dt, k.dt);  // used by the packed body only
#pragma unroll
    for (int t = 0; t < T; ++t) {
        pUV[t] = nUV[t] = cPuv[t] = cNuv[t] = mk2<V2>(0.0f, 0.0f);
        sW[t] = pW[t] = nW[t] = cPw[t] = cNw[t] = 0.0f;
    }
#pragma unroll
    for (int a = 0; a <= T; ++a) {
        cfA[a] = mk2<V2>(0.0f, 0.0f);
        cfB[a] = 0.0f;
        carG[a] = carH[a] = carWE[a] = carZ[a] = 0.0f;
    }

    auto fetch = [&](int r, float* in) {
        if (ind) {
            const size_t o = (size_t)r * pitch + gx;
            in[0] = ld_state<COHERENT>(g.u + o);
            in[1] = ld_state<COHERENT>(g.v + o);
            in[2] = ld_state<COHERENT>(g.w + o);
            in[3] = __ldg(g.ax + o);
            in[4] = __ldg(g.b + o);
            in[5] = __ldg(g.ay + o);
            if constexpr (KAHAN) {
                in[6] = ld_state<COHERENT>(g.cu + o);
                in[7] = ld_state<COHERENT>(g.cv + o);
                in[8] = ld_state<COHERENT>(g.cw + o);
            }
        } else {
#pragma unroll
            for (int f = 0; f < 9; ++f) in[f] = 0.0f;
        }
    };

    auto tick = [&](int tk, float* in) {
        const int R = lo0 + tk;
        // input row R enters the tensor window and level 0
#pragma unroll
        for (int a = T; a > 0; --a) {
            cfA[a] = cfA[a - 1];
            cfB[a] = cfB[a - 1];
        }
        cfA[0] = mk2<V2>(in[3], in[5]);
        cfB[0] = in[4];
        sW[0] = pW[0]; pUV[0] = nUV[0]; pW[0] = nW[0];
        nUV[0] = mk2<V2>(in[0], in[1]); nW[0] = in[2];
        if constexpr (KAHAN) {
            cPuv[0] = cNuv[0]; cPw[0] = cNw[0];
            cNuv[0] = mk2<V2>(in[6], in[7]); cNw[0] = in[8];
        }
        if (R + 2 < hi0) fetch(R + 2, in);  // two rows ahead

#pragma unroll
        for (int t = 1; t <= T; ++t) {
            const int q = R - t;
            const bool valid = q >= max(0, ys - T + t) && q < min(ny, ys + H + T - t);  // warp-uniform
            const bool hasS = YEDGE ? q > 0 : true, hasN = YEDGE ? q + 1 < ny : true;
            const V2 uvP = pUV[t - 1], uvN = nUV[t - 1];
            const float wP = pW[t - 1], wN = nW[t - 1];
            const V2 axy = cfA[t];
            const float bP = cfB[t], bN = cfB[t - 1];
            // x cross term of the own row (tangential difference mirrored at
            // the south / north boundary), shared with the west neighbour
            const float zxP = fvm::cross(bP, __fsub_rn(hasN ? wN : wP, hasS ? sW[t - 1] : wP));
            V2 uvE = mk2<V2>(from_east(uvP.x), from_east(uvP.y));
            float zxE = from_east(zxP);
            float wNE = from_east(wN), wNW = from_west(wN);
            if constexpr (EDGE) {
                if (!hasE) { uvE = uvP; wNE = wN; }
                if (!hasW) wNW = wN;
            }
            // east w of the own row: the north row's of the last tick
            const float wE = carWE[t];
            carWE[t] = wNE;
            // y cross terms of the own row (last tick's north row) and the north row
            const float zyP = carZ[t], zyN = fvm::cross(bN, __fsub_rn(wNE, wNW));
            carZ[t] = zyN;
            // east and north faces as (x, y) pairs: the acid flux
            // a (W_R - W_L) + (z_L + z_R) and the tumour flux
            // (K - K/2 (U_L + U_R)) (V_R - V_L) of gg_math.cuh
            V2 gf, hf;
            if constexpr (PK) {
                const float2 dw = make_float2(__fsub_rn(wE, wP), __fsub_rn(wN, wP));
                const float2 zs = make_float2(__fadd_rn(zxP, zxE), __fadd_rn(zyP, zyN));
                gf = __ffma2_rn(axy, dw, zs);
                const float2 su = make_float2(__fadd_rn(uvP.x, uvE.x), __fadd_rn(uvP.x, uvN.x));
                const float2 dv = make_float2(__fsub_rn(uvE.y, uvP.y), __fsub_rn(uvN.y, uvP.y));
                hf = __fmul2_rn(__ffma2_rn(k.nhK2, su, k.K2), dv);
            } else {
                gf = mk2<V2>(fvm::g_face(axy.x, wP, wE, zxP, zxE), fvm::g_face(axy.y, wP, wN, zyP, zyN));
                hf = mk2<V2>(fvm::h_face(uvP.x, uvE.x, uvP.y, uvE.y, k.Kx, k.hKx),
                             fvm::h_face(uvP.x, uvN.x, uvP.y, uvN.y, k.Ky, k.hKy));
            }
            if constexpr (EDGE) {
                if (!hasE) { gf.x = 0.0f; hf.x = 0.0f; }
            }
            if (!hasN) { gf.y = 0.0f; hf.y = 0.0f; }
            float gW = from_west(gf.x), hW = from_west(hf.x);
            if constexpr (EDGE) {
                if (!hasW) { gW = 0.0f; hW = 0.0f; }
            }
            const float gS = hasS ? carG[t] : 0.0f, hS = hasS ? carH[t] : 0.0f;
            carG[t] = gf.y;
            carH[t] = hf.y;
            float fu, fv, fw;
            if constexpr (PK) {
                // D D1 = (hE - hW) + (hN - hS), D2 = (gE - gW) + (gN - gS)
                const float2 eh = fvm::sub2(hf, make_float2(hW, hS));
                const float2 eg = fvm::sub2(gf, make_float2(gW, gS));
                const float d1 = __fadd_rn(eh.x, eh.y), d2 = __fadd_rn(eg.x, eg.y);
                if (k.no_reaction) {
                    fu = 0.0f;
                    fv = d1;
                    fw = d2;
                } else {
                    // U((1-U) - delta W),  rho V (1-V) + D D1,  c (V-W) + D2
                    const float2 om = fvm::sub2(make_float2(1.0f, 1.0f), uvP);
                    fu = __fmul_rn(uvP.x, __fmaf_rn(-k.delta, wP, om.x));
                    fv = __fmaf_rn(__fmul_rn(k.rho, uvP.y), om.y, d1);
                    fw = __fmaf_rn(k.c, __fsub_rn(uvP.y, wP), d2);
                }
            } else {
                fvm::rates_faces(k, uvP.x, uvP.y, wP, hf.x, hW, hf.y, hS, gf.x, gW, gf.y, gS, fu, fv, fw);
            }
            V2 uvn, cuvn = mk2<V2>(0.0f, 0.0f);
            float wn, cwn = 0.0f;
            if constexpr (KAHAN && PK) {
                // kahan_step of gg_math.cuh on the (u, v) pair and on w
                const float2 c0 = cPuv[t - 1];
                const float2 y = __ffma2_rn(dt2, make_float2(fu, fv), make_float2(-c0.x, -c0.y));
                uvn = __fadd2_rn(uvP, y);
                cuvn = fvm::sub2(fvm::sub2(uvn, uvP), y);
                fvm::kahan_step(wP, k.dt, fw, cPw[t - 1], wn, cwn);
            } else if constexpr (KAHAN) {
                fvm::kahan_step(uvP.x, k.dt, fu, cPuv[t - 1].x, uvn.x, cuvn.x);
                fvm::kahan_step(uvP.y, k.dt, fv, cPuv[t - 1].y, uvn.y, cuvn.y);
                fvm::kahan_step(wP, k.dt, fw, cPw[t - 1], wn, cwn);
            } else if constexpr (PK) {
                uvn = __ffma2_rn(dt2, make_float2(fu, fv), uvP);
                wn = fvm::euler_step(wP, k.dt, fw);
            } else {
                uvn = mk2<V2>(fvm::euler_step(uvP.x, k.dt, fu), fvm::euler_step(uvP.y, k.dt, fv));
                wn = fvm::euler_step(wP, k.dt, fw);
            }
            if (t == T) {
                if (valid && outc) {
                    const size_t o = (size_t)q * pitch + gx;
                    g.uo[o] = uvn.x;
                    g.vo[o] = uvn.y;
                    g.wo[o] = wn;
                    if constexpr (KAHAN) {
                        g.cuo[o] = cuvn.x;
                        g.cvo[o] = cuvn.y;
                        g.cwo[o] = cwn;
                    }
                }
            } else {
                const int tt = (t < T) ? t : 0;  // level t passes row q on
                sW[tt] = pW[tt]; pUV[tt] = nUV[tt]; pW[tt] = nW[tt];
                nUV[tt] = uvn; nW[tt] = wn;
                if constexpr (KAHAN) {
                    cPuv[tt] = cNuv[tt]; cPw[tt] = cNw[tt];
                    cNuv[tt] = cuvn; cNw[tt] = cwn;
                }
            }
        }
    };

    float inA[9], inB[9];
    fetch(lo0, inA);
    if (lo0 + 1 < hi0) fetch(lo0 + 1, inB);
    for (int tk = 0; tk < nticks; tk += 2) {
        tick(tk, inA);
        if (tk + 1 < nticks) tick(tk + 1, inB);
    }
}

// Runs warp_pass with the variant that matches the warp's position: interior
// strips skip the east / west boundary handling, interior chunks the south /
// north one.
template <int T, bool KAHAN, bool COHERENT = false>
__device__ __forceinline__ void warp_pass_any(const Grid32& g, const Rates32& k, const int H, const int strip,
                                              const int chunk, const int lane)
{
    constexpr int OUT = 32 - 2 * T;
    const int gx0 = strip * OUT - T;
    const bool xin = gx0 >= 1 && gx0 + 31 <= g.nx - 2;
    const int ys = chunk * H;
    const bool yin = ys - T >= 1 && ys + H + T <= g.ny - 1;
    if (xin) {
        if (yin) warp_pass<T, KAHAN, false, COHERENT, false>(g, k, H, strip, chunk, lane);
        else warp_pass<T, KAHAN, false, COHERENT, true>(g, k, H, strip, chunk, lane);
    } else {
        warp_pass<T, KAHAN, true, COHERENT, true>(g, k, H, strip, chunk, lane);
    }
}

}  // namespace stepw
}  // namespace gg
