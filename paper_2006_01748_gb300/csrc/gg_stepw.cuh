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
#include "gg_math.cuh"

namespace gg {
namespace stepw {

constexpr unsigned kFull = 0xffffffffu;

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
template <int T, bool KAHAN, bool EDGE, bool COHERENT = false, bool STASH = false, bool YEDGE = true>
__device__ __forceinline__ void warp_pass(const Grid32& g, const Rates32& k, const int H, const int strip,
                                          const int chunk, const int lane, const Stash32* stash = nullptr)
{
    constexpr int OUT = 32 - 2 * T;
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

    // windows of level t-1 used by level t, index t-1
    float sW[T], pU[T], pV[T], pW[T], nU[T], nV[T], nW[T];
    float cP[T][3], cN[T][3];
    float cf[T + 1][3];  // [age][ax, b, ay]; age a holds input row R - a
    float carG[T + 1], carH[T + 1];           // north faces of the previous tick
    float carWE[T + 1], carZ[T + 1];          // east w and y cross term of the own row
#pragma unroll
    for (int t = 0; t < T; ++t) {
        sW[t] = pU[t] = pV[t] = pW[t] = nU[t] = nV[t] = nW[t] = 0.0f;
#pragma unroll
        for (int f = 0; f < 3; ++f) cP[t][f] = cN[t][f] = 0.0f;
    }
#pragma unroll
    for (int a = 0; a <= T; ++a) {
        cf[a][0] = cf[a][1] = cf[a][2] = 0.0f;
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
            cf[a][0] = cf[a - 1][0];
            cf[a][1] = cf[a - 1][1];
            cf[a][2] = cf[a - 1][2];
        }
        cf[0][0] = in[3]; cf[0][1] = in[4]; cf[0][2] = in[5];
        sW[0] = pW[0]; pU[0] = nU[0]; pV[0] = nV[0]; pW[0] = nW[0];
        nU[0] = in[0]; nV[0] = in[1]; nW[0] = in[2];
        if constexpr (KAHAN) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                cP[0][f] = cN[0][f];
                cN[0][f] = in[6 + f];
            }
        }
        if (R + 2 < hi0) fetch(R + 2, in);  // two rows ahead

#pragma unroll
        for (int t = 1; t <= T; ++t) {
            const int q = R - t;
            const bool valid = q >= max(0, ys - T + t) && q < min(ny, ys + H + T - t);  // warp-uniform
            const bool hasS = YEDGE ? q > 0 : true, hasN = YEDGE ? q + 1 < ny : true;
            const float uP = pU[t - 1], vP = pV[t - 1], wP = pW[t - 1];
            const float uN = nU[t - 1], vN = nV[t - 1], wN = nW[t - 1];
            const float axP = cf[t][0], bP = cf[t][1], ayP = cf[t][2];
            const float bN = cf[t - 1][1];
            // x cross term of the own row (tangential difference mirrored at
            // the south / north boundary), shared with the west neighbour
            const float zxP = fvm::cross(bP, __fsub_rn(hasN ? wN : wP, hasS ? sW[t - 1] : wP));
            float uE = from_east(uP), vE = from_east(vP), zxE = from_east(zxP);
            float wNE = from_east(wN), wNW = from_west(wN);
            if constexpr (EDGE) {
                if (!hasE) { uE = uP; vE = vP; wNE = wN; }
                if (!hasW) wNW = wN;
            }
            // east w of the own row: the north row's of the last tick
            const float wE = carWE[t];
            carWE[t] = wNE;
            // y cross terms of the own row (last tick's north row) and the north row
            const float zyP = carZ[t], zyN = fvm::cross(bN, __fsub_rn(wNE, wNW));
            carZ[t] = zyN;
            float gE = fvm::g_face(axP, wP, wE, zxP, zxE);
            float hE = fvm::h_face(uP, uE, vP, vE, k.Kx, k.hKx);
            if constexpr (EDGE) {
                if (!hasE) { gE = 0.0f; hE = 0.0f; }
            }
            const float gN = hasN ? fvm::g_face(ayP, wP, wN, zyP, zyN) : 0.0f;
            const float hN = hasN ? fvm::h_face(uP, uN, vP, vN, k.Ky, k.hKy) : 0.0f;
            float gW = from_west(gE), hW = from_west(hE);
            if constexpr (EDGE) {
                if (!hasW) { gW = 0.0f; hW = 0.0f; }
            }
            const float gS = hasS ? carG[t] : 0.0f, hS = hasS ? carH[t] : 0.0f;
            carG[t] = gN;
            carH[t] = hN;
            float fu, fv, fw;
            fvm::rates_faces(k, uP, vP, wP, hE, hW, hN, hS, gE, gW, gN, gS, fu, fv, fw);
            float un, vn, wn, cun = 0.0f, cvn = 0.0f, cwn = 0.0f;
            if constexpr (KAHAN) {
                fvm::kahan_step(uP, k.dt, fu, cP[t - 1][0], un, cun);
                fvm::kahan_step(vP, k.dt, fv, cP[t - 1][1], vn, cvn);
                fvm::kahan_step(wP, k.dt, fw, cP[t - 1][2], wn, cwn);
            } else {
                un = fvm::euler_step(uP, k.dt, fu);
                vn = fvm::euler_step(vP, k.dt, fv);
                wn = fvm::euler_step(wP, k.dt, fw);
            }
            if (t == T) {
                if (valid && outc) {
                    const size_t o = (size_t)q * pitch + gx;
                    g.uo[o] = un;
                    g.vo[o] = vn;
                    g.wo[o] = wn;
                    if constexpr (KAHAN) {
                        g.cuo[o] = cun;
                        g.cvo[o] = cvn;
                        g.cwo[o] = cwn;
                    }
                }
            } else {
                if constexpr (STASH) {
                    // intermediate level: also write the own rows and columns of step s0 + t
                    if (q >= ys && q < hiT && outc) {
                        const size_t o = (size_t)q * pitch + gx;
                        const int li = (t < T) ? t - 1 : 0;
                        stash->u[li][o] = un;
                        stash->v[li][o] = vn;
                        stash->w[li][o] = wn;
                    }
                }
                const int tt = (t < T) ? t : 0;  // level t passes row q on
                sW[tt] = pW[tt]; pU[tt] = nU[tt]; pV[tt] = nV[tt]; pW[tt] = nW[tt];
                nU[tt] = un; nV[tt] = vn; nW[tt] = wn;
                if constexpr (KAHAN) {
                    cP[tt][0] = cN[tt][0]; cP[tt][1] = cN[tt][1]; cP[tt][2] = cN[tt][2];
                    cN[tt][0] = cun; cN[tt][1] = cvn; cN[tt][2] = cwn;
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
template <int T, bool KAHAN, bool COHERENT = false, bool STASH = false>
__device__ __forceinline__ void warp_pass_any(const Grid32& g, const Rates32& k, const int H, const int strip,
                                              const int chunk, const int lane, const Stash32* stash = nullptr)
{
    constexpr int OUT = 32 - 2 * T;
    const int gx0 = strip * OUT - T;
    const bool xin = gx0 >= 1 && gx0 + 31 <= g.nx - 2;
    const int ys = chunk * H;
    const bool yin = ys - T >= 1 && ys + H + T <= g.ny - 1;
    if (xin) {
        if (yin) warp_pass<T, KAHAN, false, COHERENT, STASH, false>(g, k, H, strip, chunk, lane, stash);
        else warp_pass<T, KAHAN, false, COHERENT, STASH, true>(g, k, H, strip, chunk, lane, stash);
    } else {
        warp_pass<T, KAHAN, true, COHERENT, STASH, true>(g, k, H, strip, chunk, lane, stash);
    }
}

}  // namespace stepw
}  // namespace gg
