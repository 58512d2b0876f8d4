// Per-cell arithmetic of the FP32 forward step, shared by every kernel.
//
// eq. (3) is evaluated from face fluxes (the flux form of Tables 1 and 2):
//
//   D D1(V;U)_P = (h(P,E) - h(W,P)) + (h(P,N) - h(S,P)),
//       h(L,R) = D/h^2 (1 - (U_L + U_R)/2) (V_R - V_L)              (Table 1)
//   D2(W;A)_P = (G(P,E) - G(W,P)) + (G(P,N) - G(S,P)),
//       G(L,R) = a_f (W_R - W_L) + (z_L + z_R)                      (Table 2)
//       a_f = (a11_L + a11_R)/(2 dx^2) on x-faces, (a22_L + a22_R)/(2 dy^2)
//       on y-faces (built once per tissue, Grid32::ax / ay), and
//       z = a12/(4 dx dy) * t per cell with t the tangential difference:
//       t = W_north - W_south on x-faces, W_east - W_west on y-faces
//       (mirror ghosts at the domain boundary).
//
// D is folded into the tumour face weight, so h already carries the factor
// D of eq. (3).  A face on the domain boundary carries zero flux (Section 2):
// callers pass 0 for it.  Every operation uses an explicit round-to-nearest
// intrinsic, so that the compiler cannot contract or reorder it differently
// in different kernels: a face computed once and shared (warp kernel) and the
// same face computed from both sides (shared-memory kernel) give the same
// bits, and every launch plan produces the same result.
#pragma once

#include "gg_internal.cuh"

namespace gg {
namespace fvm {

// Acid flux through a face from its weight a, the two cell values (west /
// south first) and the two cells' cross terms.
__device__ __forceinline__ float g_face(float a, float wL, float wR, float zL, float zR)
{
    return __fmaf_rn(a, __fsub_rn(wR, wL), __fadd_rn(zL, zR));
}

// Cross term of one cell: b = a12/(4 dx dy) times its tangential difference.
__device__ __forceinline__ float cross(float b, float t) { return __fmul_rn(b, t); }

// Tumour flux through a face: (K - K/2 (U_L + U_R)) (V_R - V_L), K = D/h^2.
__device__ __forceinline__ float h_face(float uL, float uR, float vL, float vR, float K, float hK)
{
    return __fmul_rn(__fmaf_rn(-hK, __fadd_rn(uL, uR), K), __fsub_rn(vR, vL));
}

// Rates of eq. (3) from the four face fluxes of each operator.
__device__ __forceinline__ void rates_faces(const Rates32& k, float up, float vp, float wp, float hE, float hW,
                                            float hN, float hS, float gE, float gW, float gN, float gS, float& fu,
                                            float& fv, float& fw)
{
    const float d1 = __fadd_rn(__fsub_rn(hE, hW), __fsub_rn(hN, hS));  // D D1
    const float d2 = __fadd_rn(__fsub_rn(gE, gW), __fsub_rn(gN, gS));
    if (k.no_reaction) {
        fu = 0.0f;
        fv = d1;
        fw = d2;
    } else {
        // U((1-U) - delta W),  rho V (1-V) + D D1,  c (V-W) + D2
        fu = __fmul_rn(up, __fmaf_rn(-k.delta, wp, __fsub_rn(1.0f, up)));
        fv = __fmaf_rn(__fmul_rn(k.rho, vp), __fsub_rn(1.0f, vp), d1);
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

// Packed pairs (sm_100 family): each lane is the same IEEE round-to-nearest
// operation as the scalar intrinsic, so packed and scalar code give the same
// bits.  a - b is formed as fma(b, -1, a), one rounding of a - b.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

}  // namespace fvm
}  // namespace gg
