// Per-cell arithmetic of the FP32 forward step, shared by every kernel.
//
// eq. (3) is evaluated from face fluxes (the flux form of Tables 1 and 2):
//
//   D1(V;U)_P = (h(P,E) - h(W,P)) + (h(P,N) - h(S,P)),
//       h(L,R) = (1 - (U_L + U_R)/2) (V_R - V_L) / h^2           (Table 1)
//   D2(W;A)_P = (Gx(P,E) - Gx(W,P)) + (Gy(P,N) - Gy(S,P)),
//       Gx(L,R) = (a11_L + a11_R)/(2 dx^2) (W_R - W_L)
//               + (a12_L ty_L + a12_R ty_R) / (4 dx dy)          (Table 2)
//       ty = W_north - W_south at the same column, tx = W_east - W_west
//       (mirror ghosts at the domain boundary), Gy likewise.
//
// A face on the domain boundary carries zero flux (Section 2): callers pass
// 0 for it.  Every operation uses an explicit round-to-nearest intrinsic, so
// that the compiler cannot contract or reorder it differently in different
// kernels: a face computed once and shared (warp kernel) and the same face
// computed from both sides (shared-memory kernel) give the same bits, and
// every launch plan produces the same result.
#pragma once

#include "gg_internal.cuh"

namespace gg {
namespace fvm {

__device__ __forceinline__ float gx_face(const Rates32& k, float a11L, float a11R, float wL, float wR, float bL,
                                         float tyL, float bR, float tyR)
{
    const float n = __fmul_rn(__fmul_rn(__fadd_rn(a11L, a11R), __fsub_rn(wR, wL)), k.kx);
    const float c = __fmaf_rn(bL, tyL, __fmul_rn(bR, tyR));
    return __fmaf_rn(k.kc, c, n);
}

__device__ __forceinline__ float gy_face(const Rates32& k, float a22S, float a22N, float wS, float wN, float bS,
                                         float txS, float bN, float txN)
{
    const float n = __fmul_rn(__fmul_rn(__fadd_rn(a22S, a22N), __fsub_rn(wN, wS)), k.ky);
    const float c = __fmaf_rn(bS, txS, __fmul_rn(bN, txN));
    return __fmaf_rn(k.kc, c, n);
}

__device__ __forceinline__ float h_face(float uL, float uR, float vL, float vR, float ih2)
{
    const float m = __fmaf_rn(-0.5f, __fadd_rn(uL, uR), 1.0f);
    return __fmul_rn(__fmul_rn(m, __fsub_rn(vR, vL)), ih2);
}

// Rates of eq. (3) from the four face fluxes of each operator.
__device__ __forceinline__ void rates_faces(const Rates32& k, float up, float vp, float wp, float hE, float hW,
                                            float hN, float hS, float gE, float gW, float gN, float gS, float& fu,
                                            float& fv, float& fw)
{
    const float d1 = __fadd_rn(__fsub_rn(hE, hW), __fsub_rn(hN, hS));
    const float d2 = __fadd_rn(__fsub_rn(gE, gW), __fsub_rn(gN, gS));
    if (k.no_reaction) {
        fu = 0.0f;
        fv = __fmul_rn(k.D, d1);
        fw = d2;
    } else {
        // U(1-U) - delta U W,  rho V(1-V) + D D1,  c (V-W) + D2
        fu = __fmaf_rn(-k.delta, __fmul_rn(up, wp), __fmul_rn(up, __fsub_rn(1.0f, up)));
        fv = __fmaf_rn(k.D, d1, __fmul_rn(__fmul_rn(k.rho, vp), __fsub_rn(1.0f, vp)));
        fw = __fmaf_rn(k.c, __fsub_rn(vp, wp), d2);
    }
}

// x' = x + dt f with the Kahan compensation comp (x - comp is the value the
// compensated sum represents): y = dt f - comp, t = x + y,
// comp' = (t - x) - y.
__device__ __forceinline__ void kahan_step(float x, float dt, float f, float comp, float& xo, float& compo)
{
    const float y = __fmaf_rn(dt, f, -comp);
    const float t = __fadd_rn(x, y);
    compo = __fsub_rn(__fsub_rn(t, x), y);
    xo = t;
}

__device__ __forceinline__ float euler_step(float x, float dt, float f) { return __fmaf_rn(dt, f, x); }

}  // namespace fvm
}  // namespace gg
