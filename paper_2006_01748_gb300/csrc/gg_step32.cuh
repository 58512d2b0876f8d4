// FP32 fused u/v/w step of eq. (3) with optional Kahan-compensated state and
// temporal blocking (T explicit Euler steps per pass over HBM).
//
// Decomposition.  A CTA owns a strip of `bx` output columns and a chunk of
// `by` output rows.  It streams the rows of its strip (plus a halo of T
// columns on each side and T rows above and below) from HBM once, and keeps
// T+1 time levels in flight in shared memory: at tick k it stores row
// lo0 + k of level 0 (the loaded state), then level t = 1..T computes row
// lo0 + k - t from the three rows r-1, r, r+1 of level t-1 (a wavefront that
// lags one row per level).  Level T is written back to HBM.  Each level keeps
// a ring of 3 state rows and 2 compensation rows; the tensor entries keep a
// ring of T+2 rows shared by all levels.  The next row of level 0 is fetched
// into registers while the levels of the current tick are computed.
//
// Cells outside the domain are never read by cells inside it: a missing
// neighbour is replaced by the cell itself (mirror ghost), which zeroes every
// normal difference at a boundary face, and the a12 cross flux through a
// boundary face is masked to zero (Section 2, zero flux).  Cells of the halo
// that lose validity level by level compute throw-away values; they are never
// stored.
#pragma once

#include "gg_internal.cuh"
#include "gg_math.cuh"

namespace gg {
namespace step32 {

struct Rows {
    const float *uS, *uP, *uN, *vS, *vP, *vN, *wS, *wP, *wN;
    const float *axP, *bS, *bP, *bN, *ayS, *ayP;
};

// Rates (fu, fv, fw) of eq. (3) at one cell from shared-memory rows.  lxW /
// lxE are the west / east neighbours, equal to lx at a domain boundary
// (mirror ghost); the row pointers S / N are mirrored in the same way.  The
// four faces are computed with the shared face functions of gg_math.cuh,
// each with its two cells in west-east / south-north order, and a boundary
// face carries zero flux.
__device__ __forceinline__ void cell_rates(const Rows& R, const Rates32& k, int lx, int lxW, int lxE, bool hasW,
                                           bool hasE, bool hasS, bool hasN, float& up, float& vp, float& wp,
                                           float& fu, float& fv, float& fw)
{
    up = R.uP[lx];
    vp = R.vP[lx];
    wp = R.wP[lx];
    const float wE = R.wP[lxE], wW = R.wP[lxW], wN = R.wN[lx], wS = R.wS[lx];
    const float wNE = R.wN[lxE], wNW = R.wN[lxW], wSE = R.wS[lxE], wSW = R.wS[lxW];
    // cross terms: x faces use t = W_N - W_S, y faces t = W_E - W_W
    const float bP = R.bP[lx];
    const float zxP = fvm::cross(bP, __fsub_rn(wN, wS));
    const float zxE = fvm::cross(R.bP[lxE], __fsub_rn(wNE, wSE));
    const float zxW = fvm::cross(R.bP[lxW], __fsub_rn(wNW, wSW));
    const float zyP = fvm::cross(bP, __fsub_rn(wE, wW));
    const float zyN = fvm::cross(R.bN[lx], __fsub_rn(wNE, wNW));
    const float zyS = fvm::cross(R.bS[lx], __fsub_rn(wSE, wSW));
    const float gE = hasE ? fvm::g_face(R.axP[lx], wp, wE, zxP, zxE) : 0.0f;
    const float gW = hasW ? fvm::g_face(R.axP[lxW], wW, wp, zxW, zxP) : 0.0f;
    const float gN = hasN ? fvm::g_face(R.ayP[lx], wp, wN, zyP, zyN) : 0.0f;
    const float gS = hasS ? fvm::g_face(R.ayS[lx], wS, wp, zyS, zyP) : 0.0f;
    const float hE = hasE ? fvm::h_face(up, R.uP[lxE], vp, R.vP[lxE], k.Kx, k.hKx) : 0.0f;
    const float hW = hasW ? fvm::h_face(R.uP[lxW], up, R.vP[lxW], vp, k.Kx, k.hKx) : 0.0f;
    const float hN = hasN ? fvm::h_face(up, R.uN[lx], vp, R.vN[lx], k.Ky, k.hKy) : 0.0f;
    const float hS = hasS ? fvm::h_face(R.uS[lx], up, R.vS[lx], vp, k.Ky, k.hKy) : 0.0f;
    fvm::rates_faces(k, up, vp, wp, hE, hW, hN, hS, gE, gW, gN, gS, fu, fv, fw);
}

// One pass of T steps over the tile (strip sx, chunk sy) of one grid; smem
// holds the rings described above.  Called by every thread of the CTA.
// State loads: COHERENT = false reads through the read-only cache (the state
// was written by an earlier launch); COHERENT = true bypasses L1 (__ldcg),
// for a persistent kernel that reads state written by other CTAs of the
// same launch.
template <bool COHERENT>
__device__ __forceinline__ float ld_state(const float* p)
{
    if constexpr (COHERENT) return __ldcg(p);
    else return __ldg(p);
}

template <int T, bool KAHAN, int MAXM, bool COHERENT = false>
__device__ __forceinline__ void tile_pass(const Grid32& g, const Rates32& k, const int bx, const int by,
                                          const int halo, const int sw, const int sx, const int sy, float* smem)
{
    float* const st = smem;                             // [T][3 fields][3 slots][sw]
    float* const cp = st + T * 9 * sw;                  // [T][3 fields][2 slots][sw]
    float* const cf = cp + (KAHAN ? T * 6 * sw : 0);    // [3 fields][T+2 slots][sw]
#define ST(lev, f, slot) (st + (((lev) * 3 + (f)) * 3 + (slot)) * sw)
#define CP(lev, f, slot) (cp + (((lev) * 3 + (f)) * 2 + (slot)) * sw)
#define CF(f, slot) (cf + ((f) * (T + 2) + (slot)) * sw)

    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const int xs = sx * bx;
    const int ys = sy * by;
    const int x0 = xs - halo;  // global column of shared-memory column 0
    const int lo0 = max(0, ys - T);
    const int hi0 = min(ny, ys + by + T);
    const int hiT = min(ny, ys + by);
    const int nticks = hiT - lo0 + T;

    // Columns owned by this thread.
    int lxs[MAXM], lxw[MAXM], lxe[MAXM], gxs[MAXM];
    bool hWs[MAXM], hEs[MAXM];
    bool act[MAXM], ind[MAXM], outc[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
        const int lx = threadIdx.x + m * blockDim.x;
        const int gx = x0 + lx;
        lxs[m] = lx;
        gxs[m] = gx;
        act[m] = lx < sw;
        ind[m] = act[m] && gx >= 0 && gx < nx;
        const bool hasW = gx > 0, hasE = gx + 1 < nx;
        lxw[m] = hasW ? max(lx - 1, 0) : lx;
        lxe[m] = hasE ? min(lx + 1, sw - 1) : lx;
        hWs[m] = hasW;
        hEs[m] = hasE;
        outc[m] = ind[m] && lx >= halo && lx < halo + bx;
    }

    // Prefetch registers for the next level-0 row.
    constexpr int NF = KAHAN ? 9 : 6;
    float pre[MAXM][NF];
    auto fetch = [&](int r) {
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
            if (ind[m]) {
                const size_t o = (size_t)r * pitch + gxs[m];
                pre[m][0] = ld_state<COHERENT>(g.u + o);
                pre[m][1] = ld_state<COHERENT>(g.v + o);
                pre[m][2] = ld_state<COHERENT>(g.w + o);
                pre[m][3] = __ldg(g.ax + o);
                pre[m][4] = __ldg(g.b + o);
                pre[m][5] = __ldg(g.ay + o);
                if constexpr (KAHAN) {
                    pre[m][6] = ld_state<COHERENT>(g.cu + o);
                    pre[m][7] = ld_state<COHERENT>(g.cv + o);
                    pre[m][8] = ld_state<COHERENT>(g.cw + o);
                }
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) pre[m][f] = 0.0f;
            }
        }
    };
    fetch(lo0);

    for (int tick = 0; tick < nticks; ++tick) {
        const int r0 = lo0 + tick;
        if (r0 < hi0) {
            const int s3 = r0 % 3, s2 = r0 % 2, sc = r0 % (T + 2);
#pragma unroll
            for (int m = 0; m < MAXM; ++m) {
                if (act[m]) {
                    const int lx = lxs[m];
                    ST(0, 0, s3)[lx] = pre[m][0];
                    ST(0, 1, s3)[lx] = pre[m][1];
                    ST(0, 2, s3)[lx] = pre[m][2];
                    CF(0, sc)[lx] = pre[m][3];
                    CF(1, sc)[lx] = pre[m][4];
                    CF(2, sc)[lx] = pre[m][5];
                    if constexpr (KAHAN) {
                        CP(0, 0, s2)[lx] = pre[m][6];
                        CP(0, 1, s2)[lx] = pre[m][7];
                        CP(0, 2, s2)[lx] = pre[m][8];
                    }
                }
            }
            if (r0 + 1 < hi0) fetch(r0 + 1);
        }
        __syncthreads();

#pragma unroll
        for (int t = 1; t <= T; ++t) {
            const int r = r0 - t;
            const int lo_t = max(0, ys - T + t);
            const int hi_t = min(ny, ys + by + T - t);
            if (r >= lo_t && r < hi_t) {
                const bool hasS = r > 0, hasN = r + 1 < ny;
                const int rs = hasS ? r - 1 : r, rn = hasN ? r + 1 : r;
                const int pS = rs % 3, pP = r % 3, pN = rn % 3;
                const int cS = rs % (T + 2), cPs = r % (T + 2), cN = rn % (T + 2);
                Rows R;
                R.uS = ST(t - 1, 0, pS); R.uP = ST(t - 1, 0, pP); R.uN = ST(t - 1, 0, pN);
                R.vS = ST(t - 1, 1, pS); R.vP = ST(t - 1, 1, pP); R.vN = ST(t - 1, 1, pN);
                R.wS = ST(t - 1, 2, pS); R.wP = ST(t - 1, 2, pP); R.wN = ST(t - 1, 2, pN);
                R.axP = CF(0, cPs);
                R.bS = CF(1, cS); R.bP = CF(1, cPs); R.bN = CF(1, cN);
                R.ayS = CF(2, cS); R.ayP = CF(2, cPs);
                const int s2 = r % 2;
#pragma unroll
                for (int m = 0; m < MAXM; ++m) {
                    if (!act[m]) continue;
                    if (t == T && !outc[m]) continue;
                    const int lx = lxs[m];
                    float up, vp, wp, fu, fv, fw;
                    cell_rates(R, k, lx, lxw[m], lxe[m], hWs[m], hEs[m], hasS, hasN, up, vp, wp, fu, fv, fw);
                    float un, vn, wn, cun = 0.f, cvn = 0.f, cwn = 0.f;
                    if constexpr (KAHAN) {
                        fvm::kahan_step(up, k.dt, fu, CP(t - 1, 0, s2)[lx], un, cun);
                        fvm::kahan_step(vp, k.dt, fv, CP(t - 1, 1, s2)[lx], vn, cvn);
                        fvm::kahan_step(wp, k.dt, fw, CP(t - 1, 2, s2)[lx], wn, cwn);
                    } else {
                        un = fvm::euler_step(up, k.dt, fu);
                        vn = fvm::euler_step(vp, k.dt, fv);
                        wn = fvm::euler_step(wp, k.dt, fw);
                    }
                    if (t == T) {
                        const size_t o = (size_t)r * pitch + gxs[m];
                        g.uo[o] = un;
                        g.vo[o] = vn;
                        g.wo[o] = wn;
                        if (KAHAN) {
                            g.cuo[o] = cun;
                            g.cvo[o] = cvn;
                            g.cwo[o] = cwn;
                        }
                    } else {
                        const int tt = (t < T) ? t : 0;  // level index of the ring written (t < T here)
                        ST(tt, 0, pP)[lx] = un;
                        ST(tt, 1, pP)[lx] = vn;
                        ST(tt, 2, pP)[lx] = wn;
                        if (KAHAN) {
                            CP(tt, 0, s2)[lx] = cun;
                            CP(tt, 1, s2)[lx] = cvn;
                            CP(tt, 2, s2)[lx] = cwn;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
#undef ST
#undef CP
#undef CF
}

template <int T, bool KAHAN, int MAXM>
__global__ void __launch_bounds__(256) step32_kernel(const Grid32 g, const Rates32 k, const int bx, const int by,
                                                     const int halo, const int sw)
{
    extern __shared__ float smem[];
    tile_pass<T, KAHAN, MAXM>(g, live_rates(k), bx, by, halo, sw, blockIdx.x, blockIdx.y, smem);
}

template <int T, bool KAHAN>
cudaError_t launch_T(const Grid32& g, const Rates32& r, const Plan32& p, cudaStream_t s)
{
    const int sw = p.bx + 2 * p.halo;
    const int maxm = (sw + p.threads - 1) / p.threads;
    const dim3 grid((g.nx + p.bx - 1) / p.bx, (g.ny + p.by - 1) / p.by);
    const size_t smem = (size_t)sw * sizeof(float) * (T * 9 + (KAHAN ? T * 6 : 0) + 3 * (T + 2));
    if (maxm > 3) return cudaErrorInvalidConfiguration;
    auto run = [&](auto kern) -> cudaError_t {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, p.threads, smem, s>>>(g, r, p.bx, p.by, p.halo, sw);
        return cudaGetLastError();
    };
    switch (maxm) {
        case 1: return run(step32_kernel<T, KAHAN, 1>);
        case 2: return run(step32_kernel<T, KAHAN, 2>);
        default: return run(step32_kernel<T, KAHAN, 3>);
    }
}

}  // namespace step32
}  // namespace gg
