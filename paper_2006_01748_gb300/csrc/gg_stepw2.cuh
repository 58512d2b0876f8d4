#pragma once
// FP32 step of eq. (3) as a warp-register wavefront over 64-column strips,
// two adjacent columns per lane (T = 1..4 steps per pass).
//
// The same march as gg_stepw.cuh (rows streamed from HBM once per pass, two
// rows ahead; level t computes row R - t at tick R from level t - 1; south
// faces carried from the previous tick, the north row's east w and y cross
// term carried to the next), but lane l holds the column pair
// (a, b) = (x0 + 2l, x0 + 2l + 1) and every quantity is a float2 over that
// pair.  So:
//   * every arithmetic step is one packed FP32 instruction for two cells
//     (__ffma2_rn, __fadd2_rn, __fmul2_rn; each lane of a packed instruction
//     is the same IEEE round-to-nearest operation as the scalar intrinsic, so
//     the bits are those of every other plan);
//   * an east / west neighbour costs one shuffle per pair: the east
//     neighbour of b is a of the next lane, that of a is the own b;
//   * rows move as 8-byte copies: each lane streams its own pair of every
//     input row into a per-warp shared-memory ring with cp.async, three rows
//     ahead of use, and reads it back when the row enters the march (state)
//     or when a level needs it (tensor weights: the ring keeps the last
//     T + 1 rows).  No lane reads another lane's ring entries, so no barrier
//     is needed: cp.async.wait_group makes a lane's own copies visible to it.
//     The prefetched rows and the tensor rows of the levels cost no
//     registers, which keeps T = 3, 4 inside the register file;
//   * a strip keeps 2 HL halo columns of its 64 (HL = T rounded up to even,
//     so that every pair starts on an even, 8-byte aligned column): 56 of 64
//     columns are written for T = 3, 4 and 60 for T = 1, 2, against 24 of 32
//     for T = 4 with one column per lane.
// Level t is valid on columns [x0 + t, x0 + 64 - t), which holds the written
// columns [x0 + HL, x0 + 64 - HL).  Warps whose strip touches the west or
// east domain boundary run the variant with the boundary conditions; the
// pair (nx - 1, nx) of an odd nx reads its second column from the row
// padding (pitch > nx) and never lets it reach a written cell.
#include "gg_math.cuh"

namespace gg {
namespace stepw2 {

constexpr unsigned kFull = 0xffffffffu;

template <int T> struct Geom {
    static constexpr int HL = (T + 1) / 2 * 2;  // halo columns on each side (even)
    static constexpr int OUT = 64 - 2 * HL;      // written columns per strip
};

// The pair one column east / west: (b, a of the next lane), (b of the
// previous lane, a).
__device__ __forceinline__ float2 east_of(float2 x) { return make_float2(x.y, __shfl_down_sync(kFull, x.x, 1)); }
__device__ __forceinline__ float2 west_of(float2 x) { return make_float2(__shfl_up_sync(kFull, x.y, 1), x.x); }
__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fvm::sub2(a, b); }

// Shared-memory ring of one warp: kRingS rows of the state fields, kRingT
// rows of the tensor weights, each row a [field][lane] array of float2.
constexpr int kAhead = 3;   // rows in flight ahead of the row entering the march
constexpr int kRingS = 4;   // >= kAhead + 1, a power of two
constexpr int kRingT = 8;   // >= T + kAhead + 1 for T <= 4, a power of two
template <bool KAHAN> struct Ring {
    static constexpr int NSF = KAHAN ? 6 : 3;  // state fields: u, v, w (, cu, cv, cw)
    static constexpr int bytes = (kRingS * NSF + kRingT * 3) * 32 * 8;
};

__device__ __forceinline__ void cp_async8(uint32_t dst, const float* src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// EDGE: the strip touches the west or east domain boundary.  YEDGE: the
// chunk's rows (with their halo of T rows) touch the south or north
// boundary.  SMASK: level t (1 <= t < T) with bit t - 1 set also writes u, v,
// w of its own rows to the stash (a compile-time set: no test per tick).
// ring: this warp's Ring<KAHAN>::bytes of shared memory.  The ring is read
// with ordinary shared-memory loads, which the compiler keeps in program order
// with the cp.async copies (their asm statements clobber memory); a slot is
// refilled only after the loads of the row it held were issued.
template <int T, bool KAHAN, bool EDGE, int SMASK = 0, bool YEDGE = true>
__device__ __forceinline__ void warp_pass2(const Grid32& g, const Rates32& k, const int H, const int strip,
                                           const int chunk, const int lane, float2* ring,
                                           const Stash32* stash = nullptr)
{
    static_assert(T >= 1 && T <= 4, "T = 1..4");
    constexpr int HL = Geom<T>::HL, OUT = Geom<T>::OUT;
    constexpr int NSF = Ring<KAHAN>::NSF;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const int ca = strip * OUT - HL + 2 * lane;  // column a of the pair (even)
    const int cb = ca + 1;
    const bool ld_ok = EDGE ? (ca >= 0 && ca < nx) : true;  // the pair starts inside the row
    const bool b_in = EDGE ? (ca >= 0 && cb < nx) : true;
    const bool hasWa = EDGE ? ca > 0 : true, hasWb = EDGE ? cb > 0 : true;
    const bool hasEa = EDGE ? ca + 1 < nx : true, hasEb = EDGE ? cb + 1 < nx : true;
    const bool outp = lane >= HL / 2 && lane < 32 - HL / 2 && ld_ok;
    const int ys = chunk * H;
    const int lo0 = max(0, ys - T);
    const int hi0 = min(ny, ys + H + T);
    const int hiT = min(ny, ys + H);
    const int nticks = hiT - lo0 + T;
    // bytes a lane copies per row and field: both columns, column a only (the
    // pair (nx - 1, nx) of an odd nx), or none (zero fill outside the domain)
    const int cpb = !EDGE ? 8 : (!ld_ok ? 0 : (b_in ? 8 : 4));
    const size_t coff = ld_ok ? (size_t)ca : 0;  // a valid source address when nothing is copied

    // this lane's entries: state row slot s, field f at rs[(s * NSF + f) * 32];
    // tensor row slot s, field f (ax, b, ay) at rt[(s * 3 + f) * 32]
    float2* const rs = ring + lane;
    float2* const rt = ring + kRingS * NSF * 32 + lane;
    const float* const src_s[6] = {g.u, g.v, g.w, g.cu, g.cv, g.cw};
    const float* const src_t[3] = {g.ax, g.b, g.ay};

    auto fetch = [&](int r) {
        if (r < hi0) {
            const size_t o = (size_t)r * pitch + coff;
            const uint32_t ds = (uint32_t)__cvta_generic_to_shared(rs + (r & (kRingS - 1)) * NSF * 32);
            const uint32_t dt = (uint32_t)__cvta_generic_to_shared(rt + (r & (kRingT - 1)) * 3 * 32);
#pragma unroll
            for (int f = 0; f < NSF; ++f) cp_async8(ds + f * 256, src_s[f] + o, cpb);
#pragma unroll
            for (int f = 0; f < 3; ++f) cp_async8(dt + f * 256, src_t[f] + o, cpb);
        }
        cp_async_commit();  // one group per row (empty past the chunk)
    };
    // tensor row r: ax at [0], b at [32], ay at [64]
    auto trow = [&](int r) { return rt + (r & (kRingT - 1)) * 3 * 32; };

    const float2 zero = make_float2(0.0f, 0.0f);
    // windows of level t - 1 read by level t, index t - 1
    float2 uP[T], vP[T], wP[T], uN[T], vN[T], wN[T], wS[T];
    float2 cuP[T], cvP[T], cwP[T], cuN[T], cvN[T], cwN[T];
    float2 carG[T + 1], carH[T + 1];   // north faces of the previous tick
    float2 carWE[T + 1], carZ[T + 1];  // east w and y cross term of the own row
#pragma unroll
    for (int t = 0; t < T; ++t) {
        uP[t] = vP[t] = wP[t] = uN[t] = vN[t] = wN[t] = wS[t] = zero;
        cuP[t] = cvP[t] = cwP[t] = cuN[t] = cvN[t] = cwN[t] = zero;
    }
#pragma unroll
    for (int a = 0; a <= T; ++a) carG[a] = carH[a] = carWE[a] = carZ[a] = zero;
    const float2 dt2 = dup(k.dt), K2x = dup(k.Kx), K2y = dup(k.Ky), nhx = dup(-k.hKx), nhy = dup(-k.hKy);
    const float2 one2 = dup(1.0f), ndelta = dup(-k.delta), rho2 = dup(k.rho), c2 = dup(k.c);

    auto tick = [&](int tk) {
        const int R = lo0 + tk;
        fetch(R + kAhead);
        cp_async_wait<kAhead>();  // row R has landed
        {
            const float2* ds = rs + (R & (kRingS - 1)) * NSF * 32;
            wS[0] = wP[0]; uP[0] = uN[0]; vP[0] = vN[0]; wP[0] = wN[0];
            uN[0] = ds[0]; vN[0] = ds[32]; wN[0] = ds[64];
            if constexpr (KAHAN) {
                cuP[0] = cuN[0]; cvP[0] = cvN[0]; cwP[0] = cwN[0];
                cuN[0] = ds[96]; cvN[0] = ds[128]; cwN[0] = ds[160];
            }
        }
        float2 bN = trow(R)[32];  // b of the north row of level 1

#pragma unroll
        for (int t = 1; t <= T; ++t) {
            const int q = R - t;
            const bool valid = q >= max(0, ys - T + t) && q < min(ny, ys + H + T - t);  // warp-uniform
            const bool hasS = YEDGE ? q > 0 : true, hasN = YEDGE ? q + 1 < ny : true;
            const int i = t - 1;
            const float2* tq = trow(q);
            const float2 ax = tq[0], bP = tq[32], ay = tq[64];
            const float2 u = uP[i], v = vP[i], w = wP[i], un = uN[i], vn = vN[i], wn = wN[i];
            // x cross term of the own row (tangential difference mirrored at
            // the south / north boundary)
            const float2 zxP = mul2(bP, sub2(hasN ? wn : w, hasS ? wS[i] : w));
            float2 uE = east_of(u), vE = east_of(v), zxE = east_of(zxP);
            float2 wNE = east_of(wn), wNW = west_of(wn);
            if constexpr (EDGE) {
                if (!hasEa) { uE.x = u.x; vE.x = v.x; wNE.x = wn.x; }
                if (!hasEb) { uE.y = u.y; vE.y = v.y; wNE.y = wn.y; }
                if (!hasWa) wNW.x = wn.x;
                if (!hasWb) wNW.y = wn.y;
            }
            const float2 wE = carWE[t];
            carWE[t] = wNE;
            const float2 zyP = carZ[t], zyN = mul2(bN, sub2(wNE, wNW));
            carZ[t] = zyN;
            bN = bP;  // the own row is the north row of the next level
            // east and north faces: acid a (W_R - W_L) + (z_L + z_R), tumour
            // (K - K/2 (U_L + U_R)) (V_R - V_L)
            float2 gE = fma2(ax, sub2(wE, w), add2(zxP, zxE));
            float2 hE = mul2(fma2(nhx, add2(u, uE), K2x), sub2(vE, v));
            float2 gN = fma2(ay, sub2(wn, w), add2(zyP, zyN));
            float2 hN = mul2(fma2(nhy, add2(u, un), K2y), sub2(vn, v));
            if constexpr (EDGE) {
                if (!hasEa) { gE.x = 0.0f; hE.x = 0.0f; }
                if (!hasEb) { gE.y = 0.0f; hE.y = 0.0f; }
            }
            if (!hasN) { gN = zero; hN = zero; }
            float2 gW = west_of(gE), hW = west_of(hE);
            if constexpr (EDGE) {
                if (!hasWa) { gW.x = 0.0f; hW.x = 0.0f; }
                if (!hasWb) { gW.y = 0.0f; hW.y = 0.0f; }
            }
            const float2 gS = hasS ? carG[t] : zero, hS = hasS ? carH[t] : zero;
            carG[t] = gN;
            carH[t] = hN;
            // D D1 = (hE - hW) + (hN - hS), D2 = (gE - gW) + (gN - gS)
            const float2 d1 = add2(sub2(hE, hW), sub2(hN, hS));
            const float2 d2 = add2(sub2(gE, gW), sub2(gN, gS));
            float2 fu, fv, fw;
            if (k.no_reaction) {
                fu = zero;
                fv = d1;
                fw = d2;
            } else {
                // U((1-U) - delta W),  rho V (1-V) + D D1,  c (V-W) + D2
                fu = mul2(u, fma2(ndelta, w, sub2(one2, u)));
                fv = fma2(mul2(rho2, v), sub2(one2, v), d1);
                fw = fma2(c2, sub2(v, w), d2);
            }
            float2 uo, vo, wo, cuo = zero, cvo = zero, cwo = zero;
            if constexpr (KAHAN) {
                // x' = x + y, comp' = (x' - x) - y with y = dt f - comp
                const float2 yu = fma2(dt2, fu, make_float2(-cuP[i].x, -cuP[i].y));
                const float2 yv = fma2(dt2, fv, make_float2(-cvP[i].x, -cvP[i].y));
                const float2 yw = fma2(dt2, fw, make_float2(-cwP[i].x, -cwP[i].y));
                uo = add2(u, yu);
                vo = add2(v, yv);
                wo = add2(w, yw);
                cuo = sub2(sub2(uo, u), yu);
                cvo = sub2(sub2(vo, v), yv);
                cwo = sub2(sub2(wo, w), yw);
            } else {
                uo = fma2(dt2, fu, u);
                vo = fma2(dt2, fv, v);
                wo = fma2(dt2, fw, w);
            }
            if (t == T) {
                if (valid && outp) {
                    const size_t o = (size_t)q * pitch + ca;
                    if (!EDGE || b_in) {
                        *reinterpret_cast<float2*>(g.uo + o) = uo;
                        *reinterpret_cast<float2*>(g.vo + o) = vo;
                        *reinterpret_cast<float2*>(g.wo + o) = wo;
                        if constexpr (KAHAN) {
                            *reinterpret_cast<float2*>(g.cuo + o) = cuo;
                            *reinterpret_cast<float2*>(g.cvo + o) = cvo;
                            *reinterpret_cast<float2*>(g.cwo + o) = cwo;
                        }
                    } else {
                        g.uo[o] = uo.x;
                        g.vo[o] = vo.x;
                        g.wo[o] = wo.x;
                        if constexpr (KAHAN) {
                            g.cuo[o] = cuo.x;
                            g.cvo[o] = cvo.x;
                            g.cwo[o] = cwo.x;
                        }
                    }
                }
            } else {
                if constexpr (SMASK != 0) {
                    // intermediate level in the stash set: also write the own
                    // rows of step s0 + t (streaming stores: the stash is read
                    // back only by the reverse sweep, long after the pass, so
                    // it is written evict-first and leaves the pass's own rows
                    // in L2)
                    const int li = (t < T) ? t - 1 : 0;
                    if (((SMASK >> li) & 1) && q >= ys && q < hiT && outp) {
                        const size_t o = (size_t)q * pitch + ca;
                        if (!EDGE || b_in) {
                            __stcs(reinterpret_cast<float2*>(stash->u[li] + o), uo);
                            __stcs(reinterpret_cast<float2*>(stash->v[li] + o), vo);
                            __stcs(reinterpret_cast<float2*>(stash->w[li] + o), wo);
                        } else {
                            __stcs(stash->u[li] + o, uo.x);
                            __stcs(stash->v[li] + o, vo.x);
                            __stcs(stash->w[li] + o, wo.x);
                        }
                    }
                }
                const int tt = (t < T) ? t : 0;  // level t passes row q on
                wS[tt] = wP[tt]; uP[tt] = uN[tt]; vP[tt] = vN[tt]; wP[tt] = wN[tt];
                uN[tt] = uo; vN[tt] = vo; wN[tt] = wo;
                if constexpr (KAHAN) {
                    cuP[tt] = cuN[tt]; cvP[tt] = cvN[tt]; cwP[tt] = cwN[tt];
                    cuN[tt] = cuo; cvN[tt] = cvo; cwN[tt] = cwo;
                }
            }
        }
    };

#pragma unroll
    for (int r = 0; r < kAhead; ++r) fetch(lo0 + r);
    for (int tk = 0; tk < nticks; tk += 2) {
        tick(tk);
        if (tk + 1 < nticks) tick(tk + 1);
    }
    cp_async_wait<0>();  // nothing in flight when the warp leaves
}

// Runs warp_pass2 with the variant that matches the warp's position.
template <int T, bool KAHAN, int SMASK = 0>
__device__ __forceinline__ void warp_pass2_any(const Grid32& g, const Rates32& k, const int H, const int strip,
                                               const int chunk, const int lane, float2* ring,
                                               const Stash32* stash = nullptr)
{
    constexpr int HL = Geom<T>::HL, OUT = Geom<T>::OUT;
    const int x0 = strip * OUT - HL;
    const bool xin = x0 >= 1 && x0 + 63 <= g.nx - 2;
    const int ys = chunk * H;
    const bool yin = ys - T >= 1 && ys + H + T <= g.ny - 1;
    if (xin) {
        if (yin) warp_pass2<T, KAHAN, false, SMASK, false>(g, k, H, strip, chunk, lane, ring, stash);
        else warp_pass2<T, KAHAN, false, SMASK, true>(g, k, H, strip, chunk, lane, ring, stash);
    } else {
        warp_pass2<T, KAHAN, true, SMASK, true>(g, k, H, strip, chunk, lane, ring, stash);
    }
}

}  // namespace stepw2
}  // namespace gg
