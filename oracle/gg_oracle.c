/*
 * FP64 serial oracle for the explicit finite-volume step of the anisotropic,
 * heterogeneous Gatenby-Gawlinski system (Mascia, Pera, Simeoni,
 * arXiv 2006.01748).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Plain, slow and literal on purpose: one loop over cells, double precision,
 * every operation in the order of the formula it restates.
 *
 *   Model              eq. (1):  U_t = U(1-U) - d U W
 *                                V_t = r V(1-V) + alpha div[(1-U) grad V]
 *                                W_t = c (V-W) + div(A grad W)
 *   Tensor             eq. (2):  A = [[a, b], [b, c]]; here a11=a, a12=b, a22=c
 *                                of the paper's Table 2 (the scalar acid rate
 *                                keeps the letter c).  A = R(theta) diag(l1,l2)
 *                                R(theta)^T with R = [[cos,-sin],[sin,cos]].
 *   Scheme             eq. (3):  explicit Euler, cell-centred unknowns on the
 *                                dual cells C_ij of Section 2.
 *   Tumour stencil     Table 1:  five-point, face mobility 1-(U_P+U_nb)/2.
 *   Acid stencil       Table 2:  nine-point, written here as face fluxes that
 *                                telescope to Table 2 in the interior.
 *   Boundary           Section 2 ("Neumann-type"): zero flux through every
 *                                boundary face; a tangential central difference
 *                                that reaches outside the domain uses the mirror
 *                                ghost (W_{-1,j} = W_{0,j}, corners mirrored in
 *                                both directions).
 *
 * The row loop of ggo_step carries an OpenMP pragma; only the multi-core
 * CPU-baseline build (-fopenmp) enables it, every other build ignores it.
 * Each cell is computed by the same arithmetic either way.
 *
 * Parity pins of each function are listed in tests/test_oracle_pins.py.
 * Parity unpinned: none of the functions below is unpinned, but the paper
 * prints no numerical result, so agreement with the authors' own code cannot
 * be checked.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the step runs on: omp_get_max_threads() in the OpenMP build, else 1. */
int ggo_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    int32_t nx, ny;      /* cells in x and y */
    int32_t no_reaction; /* 1: drop U(1-U)-dUW, rV(1-V) and c(V-W) */
    int32_t pad;
    double dx, dy;       /* cell sizes */
    double delta;        /* d     (eq. 1) */
    double rho;          /* r     (eq. 1) */
    double D;            /* alpha (eq. 1) */
    double c;            /* c     (eq. 1) */
    double dt;           /* Delta t_k, held fixed */
} ggo_problem;

#define AT(f, i, j) ((f)[(size_t)(j) * (size_t)nx + (size_t)(i)])

static int clampi(int k, int lo, int hi) { return k < lo ? lo : (k > hi ? hi : k); }

/* ---------------------------------------------------------------- eq. (2) */

/* A = R(theta) diag(l1, l2) R(theta)^T, written as two 2x2 products. */
void ggo_coefficients(int64_t n, const double* theta, const double* l1, const double* l2,
                      double* a11, double* a12, double* a22)
{
    for (int64_t k = 0; k < n; ++k) {
        double cs = cos(theta[k]), sn = sin(theta[k]);
        double R[2][2] = {{cs, -sn}, {sn, cs}};
        double L[2] = {l1[k], l2[k]};
        double RL[2][2];
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) RL[r][q] = R[r][q] * L[q];
        double A[2][2];
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) A[r][q] = RL[r][0] * R[q][0] + RL[r][1] * R[q][1];
        a11[k] = A[0][0];
        a12[k] = A[0][1];
        a22[k] = A[1][1];
    }
}

/* Largest eigenvalue of the symmetric 2x2 matrix [[a11,a12],[a12,a22]]. */
double ggo_lambda_max(int64_t n, const double* a11, const double* a12, const double* a22)
{
    double m = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double h = 0.5 * (a11[k] - a22[k]);
        double e = 0.5 * (a11[k] + a22[k]) + sqrt(h * h + a12[k] * a12[k]);
        if (e > m) m = e;
    }
    return m;
}

/* Largest stable step of the explicit scheme.  Section 2 recomputes
 * Delta t_k so that the scheme stays stable but gives no formula; the reading
 * used here bounds every diagonal coefficient of eq. (3) at once:
 *   dt_max = 1 / ( 2 Lambda (1/dx^2 + 1/dy^2) + c + rho + 1 + delta ),
 *   Lambda = max( max_ij lambda_max(A_ij), D ).
 * It is always below h^2 / (4 Lambda) when dx = dy = h. */
double ggo_dt_max(double dx, double dy, double Lambda, double delta, double rho, double D, double c)
{
    double L = Lambda > D ? Lambda : D;
    return 1.0 / (2.0 * L * (1.0 / (dx * dx) + 1.0 / (dy * dy)) + (c + rho + 1.0 + delta));
}

/* ------------------------------------------------------------ Table 1 */

/* D1(V;U)_P = sum over the interior faces of P of
 *             (1 - (U_P + U_nb)/2) (V_nb - V_P) / h^2.
 * x part (east + west) and y part (north + south) are summed separately and
 * then added, so that transposing the problem maps the evaluation onto itself. */
static double tumour_at(int nx, int ny, double dx, double dy, const double* U, const double* V, int i, int j)
{
    double up = AT(U, i, j), vp = AT(V, i, j);
    double hx2 = dx * dx, hy2 = dy * dy;
    double e = 0.0, w = 0.0, n = 0.0, s = 0.0;
    if (i + 1 < nx) e = (1.0 - 0.5 * (up + AT(U, i + 1, j))) * (AT(V, i + 1, j) - vp) / hx2;
    if (i - 1 >= 0) w = (1.0 - 0.5 * (up + AT(U, i - 1, j))) * (AT(V, i - 1, j) - vp) / hx2;
    if (j + 1 < ny) n = (1.0 - 0.5 * (up + AT(U, i, j + 1))) * (AT(V, i, j + 1) - vp) / hy2;
    if (j - 1 >= 0) s = (1.0 - 0.5 * (up + AT(U, i, j - 1))) * (AT(V, i, j - 1) - vp) / hy2;
    return (e + w) + (n + s);
}

void ggo_tumour_operator(int32_t nx, int32_t ny, double dx, double dy,
                         const double* U, const double* V, double* out)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) AT(out, i, j) = tumour_at(nx, ny, dx, dy, U, V, i, j);
}

/* ------------------------------------------------------------ Table 2 */

/* Flux of A grad W through the x-face between (i,j) and (i+1,j), 0 <= i < nx-1:
 *   (a11_ij + a11_{i+1,j}) / (2 dx^2) (W_{i+1,j} - W_ij)
 * + [ a12_ij (W_{i,j+1} - W_{i,j-1}) + a12_{i+1,j} (W_{i+1,j+1} - W_{i+1,j-1}) ] / (4 dx dy)
 * with mirror ghosts in j.  Summing these fluxes over the four faces of an
 * interior cell gives exactly the nine coefficients of Table 2. */
static double flux_x(int nx, int ny, double dx, double dy, const double* a11, const double* a12,
                     const double* W, int i, int j)
{
    int jn = clampi(j + 1, 0, ny - 1), js = clampi(j - 1, 0, ny - 1);
    double normal = (AT(a11, i, j) + AT(a11, i + 1, j)) * (0.5 / (dx * dx)) * (AT(W, i + 1, j) - AT(W, i, j));
    double cross = (AT(a12, i, j) * (AT(W, i, jn) - AT(W, i, js))
                    + AT(a12, i + 1, j) * (AT(W, i + 1, jn) - AT(W, i + 1, js))) * (0.25 / (dx * dy));
    return normal + cross;
}

/* Flux through the y-face between (i,j) and (i,j+1), 0 <= j < ny-1 (the
 * mirror image of flux_x). */
static double flux_y(int nx, int ny, double dx, double dy, const double* a22, const double* a12,
                     const double* W, int i, int j)
{
    int ie = clampi(i + 1, 0, nx - 1), iw = clampi(i - 1, 0, nx - 1);
    double normal = (AT(a22, i, j) + AT(a22, i, j + 1)) * (0.5 / (dy * dy)) * (AT(W, i, j + 1) - AT(W, i, j));
    double cross = (AT(a12, i, j) * (AT(W, ie, j) - AT(W, iw, j))
                    + AT(a12, i, j + 1) * (AT(W, ie, j + 1) - AT(W, iw, j + 1))) * (0.25 / (dy * dx));
    return normal + cross;
}

static double acid_at(int nx, int ny, double dx, double dy, const double* a11, const double* a12,
                      const double* a22, const double* W, int i, int j)
{
    double ge = (i + 1 < nx) ? flux_x(nx, ny, dx, dy, a11, a12, W, i, j) : 0.0;
    double gw = (i - 1 >= 0) ? flux_x(nx, ny, dx, dy, a11, a12, W, i - 1, j) : 0.0;
    double gn = (j + 1 < ny) ? flux_y(nx, ny, dx, dy, a22, a12, W, i, j) : 0.0;
    double gs = (j - 1 >= 0) ? flux_y(nx, ny, dx, dy, a22, a12, W, i, j - 1) : 0.0;
    return (ge - gw) + (gn - gs);
}

void ggo_acid_operator(int32_t nx, int32_t ny, double dx, double dy,
                       const double* a11, const double* a12, const double* a22,
                       const double* W, double* out)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) AT(out, i, j) = acid_at(nx, ny, dx, dy, a11, a12, a22, W, i, j);
}

/* ------------------------------------------------------------ eq. (3) */

/* One explicit Euler step from (U,V,W) at t_k to (Uo,Vo,Wo) at t_{k+1}:
 *   U' = U + dt (U(1-U) - d U W)
 *   V' = V + dt (r V(1-V) + alpha D1(V;U))
 *   W' = W + dt (c (V-W) + D2(W;A))
 * The rate is summed before it is scaled by dt (the grouping of eq. (3) with
 * dt factored out), so a state whose rate is exactly zero stays bitwise fixed. */
void ggo_step(const ggo_problem* p, const double* a11, const double* a12, const double* a22,
              const double* U, const double* V, const double* W,
              double* Uo, double* Vo, double* Wo)
{
    int nx = p->nx, ny = p->ny;
    double dt = p->dt;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double u = AT(U, i, j), v = AT(V, i, j), w = AT(W, i, j);
            double d1 = tumour_at(nx, ny, p->dx, p->dy, U, V, i, j);
            double d2 = acid_at(nx, ny, p->dx, p->dy, a11, a12, a22, W, i, j);
            double fu, fv, fw;
            if (p->no_reaction) {
                fu = 0.0;
                fv = p->D * d1;
                fw = d2;
            } else {
                fu = u * (1.0 - u) - p->delta * u * w;
                fv = p->rho * v * (1.0 - v) + p->D * d1;
                fw = p->c * (v - w) + d2;
            }
            AT(Uo, i, j) = u + dt * fu;
            AT(Vo, i, j) = v + dt * fv;
            AT(Wo, i, j) = w + dt * fw;
        }
    }
}

/* nsteps steps in place (U, V, W hold t_0 on entry and t_n on exit).
 * Returns 0, or -1 if scratch memory could not be allocated. */
int ggo_run(const ggo_problem* p, const double* a11, const double* a12, const double* a22,
            double* U, double* V, double* W, int64_t nsteps)
{
    size_t n = (size_t)p->nx * (size_t)p->ny;
    double* buf = (double*)malloc(3 * n * sizeof(double));
    if (!buf) return -1;
    double *u2 = buf, *v2 = buf + n, *w2 = buf + 2 * n;
    for (int64_t k = 0; k < nsteps; ++k) {
        ggo_step(p, a11, a12, a22, U, V, W, u2, v2, w2);
        memcpy(U, u2, n * sizeof(double));
        memcpy(V, v2, n * sizeof(double));
        memcpy(W, w2, n * sizeof(double));
    }
    free(buf);
    return 0;
}

/* ------------------------------------------------------------ adaptive Delta t_k */

/* The step of Section 2 recomputed from the state, Delta t_k.  The paper
 * recomputes Delta t_k after each iteration "to ensure numerical stability"
 * and gives no formula.  Reading: Delta t_k is the largest step for which the
 * coefficient of each unknown's own old value in eq. (3) stays at least
 * 1 - cfl, evaluated on the current state X^k:
 *   U' = U (1 + dt (1 - U - d W))                      -> kU = U + d W - 1
 *   V' = V (1 + dt (r (1 - V) - alpha S)) + (neighbours),
 *        S = sum over the interior faces f of (1 - (U_P + U_nb)/2) / h_f^2
 *                                                      -> kV = alpha S - r (1 - V)
 *   W: the acid operator's stable bound, static since A is:
 *        kW = c + 2 Lambda_A (1/dx^2 + 1/dy^2), Lambda_A = max lambda_max(A)
 *   Delta t_k = cfl / max(kW, max_cells kU, max_cells kV).
 * Without reactions the reaction parts (1, d, r, c) are left out.  For
 * states in [0, 1] it is never below the fixed step of ggo_dt_max. */
double ggo_adaptive_dt(const ggo_problem* p, double Lambda_A, double cfl, const double* U, const double* V,
                       const double* W)
{
    int nx = p->nx, ny = p->ny;
    double hx2 = p->dx * p->dx, hy2 = p->dy * p->dy;
    double kW = 2.0 * Lambda_A * (1.0 / hx2 + 1.0 / hy2) + (p->no_reaction ? 0.0 : p->c);
    double kU = 0.0, kV = 0.0;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double u = AT(U, i, j), v = AT(V, i, j), w = AT(W, i, j);
            double S = 0.0;
            if (i + 1 < nx) S += (1.0 - 0.5 * (u + AT(U, i + 1, j))) / hx2;
            if (i - 1 >= 0) S += (1.0 - 0.5 * (u + AT(U, i - 1, j))) / hx2;
            if (j + 1 < ny) S += (1.0 - 0.5 * (u + AT(U, i, j + 1))) / hy2;
            if (j - 1 >= 0) S += (1.0 - 0.5 * (u + AT(U, i, j - 1))) / hy2;
            double ku = p->no_reaction ? 0.0 : u + p->delta * w - 1.0;
            double kv = p->D * S - (p->no_reaction ? 0.0 : p->rho * (1.0 - v));
            if (ku > kU) kU = ku;
            if (kv > kV) kV = kv;
        }
    }
    double k = kW;
    if (kU > k) k = kU;
    if (kV > k) k = kV;
    return cfl / k;
}

/* nsteps steps in place with the adaptive step: Delta t_k is recomputed
 * (ggo_adaptive_dt) at every step k = 0, every, 2 every, ... of this call and
 * held in between.  *t_out (may be NULL) receives the time advanced,
 * sum_k Delta t_k, and *dt_out (may be NULL) the last Delta t_k.  p->dt is not
 * used.  Returns 0, or -1 if scratch memory could not be allocated. */
int ggo_run_adaptive(const ggo_problem* p, const double* a11, const double* a12, const double* a22,
                     double Lambda_A, double cfl, int64_t every, double* U, double* V, double* W, int64_t nsteps,
                     double* t_out, double* dt_out)
{
    size_t n = (size_t)p->nx * (size_t)p->ny;
    double* buf = (double*)malloc(3 * n * sizeof(double));
    if (!buf) return -1;
    double *u2 = buf, *v2 = buf + n, *w2 = buf + 2 * n;
    ggo_problem q = *p;
    double t = 0.0;
    if (every < 1) every = 1;
    for (int64_t k = 0; k < nsteps; ++k) {
        if (k % every == 0) q.dt = ggo_adaptive_dt(p, Lambda_A, cfl, U, V, W);
        ggo_step(&q, a11, a12, a22, U, V, W, u2, v2, w2);
        memcpy(U, u2, n * sizeof(double));
        memcpy(V, v2, n * sizeof(double));
        memcpy(W, w2, n * sizeof(double));
        t += q.dt;
    }
    if (t_out) *t_out = t;
    if (dt_out) *dt_out = q.dt;
    free(buf);
    return 0;
}

/* ------------------------------------------------------------ diagnostics */

/* out[0..2]  integrals dx dy sum F of U, V, W
 * out[3..5]  minima, out[6..8] maxima of U, V, W
 * out[9]     number of non-finite values over the three fields
 * out[10]    tumour area dx dy #{V > 1/2}
 * out[11]    gap area dx dy #{U < eps and V < eps} */
void ggo_diagnostics(int32_t nx, int32_t ny, double dx, double dy, const double* U, const double* V,
                     const double* W, double eps, double* out)
{
    const double* F[3] = {U, V, W};
    size_t n = (size_t)nx * (size_t)ny;
    double nonfinite = 0.0, tumour = 0.0, gap = 0.0;
    for (int f = 0; f < 3; ++f) {
        double s = 0.0, lo = INFINITY, hi = -INFINITY;
        for (size_t k = 0; k < n; ++k) {
            double x = F[f][k];
            if (!isfinite(x)) { nonfinite += 1.0; continue; }
            s += x;
            if (x < lo) lo = x;
            if (x > hi) hi = x;
        }
        out[f] = s * dx * dy;
        out[3 + f] = lo;
        out[6 + f] = hi;
    }
    for (size_t k = 0; k < n; ++k) {
        if (V[k] > 0.5) tumour += 1.0;
        if (U[k] < eps && V[k] < eps) gap += 1.0;
    }
    out[9] = nonfinite;
    out[10] = tumour * dx * dy;
    out[11] = gap * dx * dy;
}

/* ------------------------------------------------------------ front diagnostics */

/* Propagating fronts and the interstitial gap of Section 2, measured along the
 * four axis rays from the cell (i0, j0) (the centre of the initial tumour).
 * Ray d = 0 east, 1 west, 2 north, 3 south holds the cells k = 0 .. L-1 at
 * k cells from (i0, j0) (k = 0 is (i0, j0) itself); h = dx on the east and
 * west rays, dy on the others; distances are from the centre of cell k = 0.
 *   kT         the farthest cell with V > v_front (-1 if none)
 *   kH         the first cell beyond kT with U > u_edge (L if none)
 *   front[d]   (kT + 1/2) h, the outer face of the tumour (0 if kT = -1)
 *   edge[d]    (kH - 1/2) h, the inner face of the healthy tissue
 *   gap[d]     h #{k : kT < k < kH, U_k < eps and V_k < eps}
 *   mass_v[d]  h sum_k V_k,  mass_u[d] = h sum_k U_k
 * out[0..3] front, [4..7] edge, [8..11] gap, [12..15] mass_v, [16..19] mass_u. */
void ggo_front_rays(int32_t nx, int32_t ny, double dx, double dy, const double* U, const double* V, int32_t i0,
                    int32_t j0, double v_front, double u_edge, double eps, double* out)
{
    for (int d = 0; d < 4; ++d) {
        int L, di = 0, dj = 0;
        double h;
        if (d == 0) { L = nx - i0; di = 1; h = dx; }
        else if (d == 1) { L = i0 + 1; di = -1; h = dx; }
        else if (d == 2) { L = ny - j0; dj = 1; h = dy; }
        else { L = j0 + 1; dj = -1; h = dy; }
        int kT = -1;
        double sv = 0.0, su = 0.0;
        for (int k = 0; k < L; ++k) {
            double u = AT(U, i0 + di * k, j0 + dj * k), v = AT(V, i0 + di * k, j0 + dj * k);
            if (v > v_front) kT = k;
            sv += v;
            su += u;
        }
        int kH = L;
        for (int k = kT + 1; k < L; ++k)
            if (AT(U, i0 + di * k, j0 + dj * k) > u_edge) { kH = k; break; }
        int gap = 0;
        for (int k = kT + 1; k < kH; ++k) {
            double u = AT(U, i0 + di * k, j0 + dj * k), v = AT(V, i0 + di * k, j0 + dj * k);
            if (u < eps && v < eps) ++gap;
        }
        out[d] = kT >= 0 ? (kT + 0.5) * h : 0.0;
        out[4 + d] = (kH - 0.5) * h;
        out[8 + d] = gap * h;
        out[12 + d] = sv * h;
        out[16 + d] = su * h;
    }
}

/* Space-averaged front speed along each ray (the LeVeque-Yee formula): the
 * rate of change of the ray integral of V divided by the jump of V across
 * the front, from the state behind it (V = 1, both invasion regimes of
 * Section 2) to the state ahead of it (V = 0):
 *   speed[d] = (mass_v_after[d] - mass_v_before[d]) / (elapsed (1 - 0)).
 * before / after are ggo_front_rays outputs. */
void ggo_front_speed(const double* before, const double* after, double elapsed, double* speed)
{
    for (int d = 0; d < 4; ++d) speed[d] = (after[12 + d] - before[12 + d]) / (elapsed * (1.0 - 0.0));
}

/* ------------------------------------------------------------ discrete adjoint */

/* Reverse-mode derivative of one step (ggo_step) at the state (U,V,W):
 * given lamU/lamV/lamW = dL/d(U',V',W'), it overwrites them with
 * dL/d(U,V,W) and adds dL/d(a11,a12,a22) into ga11/ga12/ga22 and
 * dL/d(delta, rho, D, c) into gs[0..3].  It is the transpose of each term of
 * ggo_step taken one term at a time (scatter form), in the order the forward
 * computes them; the derivative of dt is not taken (dt is a fixed input). */
int ggo_step_vjp(const ggo_problem* p, const double* a11, const double* a12, const double* a22,
                 const double* U, const double* V, const double* W,
                 double* lamU, double* lamV, double* lamW,
                 double* ga11, double* ga12, double* ga22, double* gs)
{
    int nx = p->nx, ny = p->ny;
    size_t n = (size_t)nx * (size_t)ny;
    double dt = p->dt, dx = p->dx, dy = p->dy;
    double* nu = (double*)malloc(3 * n * sizeof(double));
    if (!nu) return -1;
    double *nU = nu, *nV = nu + n, *nW = nu + 2 * n;
    /* identity part of U' = U + dt f */
    memcpy(nU, lamU, n * sizeof(double));
    memcpy(nV, lamV, n * sizeof(double));
    memcpy(nW, lamW, n * sizeof(double));

    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t P = (size_t)j * nx + i;
            double u = U[P], v = V[P], w = W[P];
            double bu = dt * lamU[P], bv = dt * lamV[P], bw = dt * lamW[P]; /* dL/df at P */
            if (!p->no_reaction) {
                /* fu = u(1-u) - delta u w */
                nU[P] += bu * (1.0 - 2.0 * u - p->delta * w);
                nW[P] += bu * (-p->delta * u);
                gs[0] += bu * (-u * w);
                /* fv = rho v(1-v) + D d1 */
                nV[P] += bv * p->rho * (1.0 - 2.0 * v);
                gs[1] += bv * v * (1.0 - v);
                /* fw = c(v-w) + d2 */
                nV[P] += bw * p->c;
                nW[P] += bw * (-p->c);
                gs[3] += bw * (v - w);
            }
            /* fv += D d1,  d1 = sum_faces (1 - (U_P+U_nb)/2) (V_nb - V_P) / h^2 */
            double d1 = tumour_at(nx, ny, dx, dy, U, V, i, j);
            gs[2] += bv * d1;
            double bd1 = bv * p->D;
            int nbi[4] = {i + 1, i - 1, i, i};
            int nbj[4] = {j, j, j + 1, j - 1};
            double h2[4] = {dx * dx, dx * dx, dy * dy, dy * dy};
            for (int f = 0; f < 4; ++f) {
                if (nbi[f] < 0 || nbi[f] >= nx || nbj[f] < 0 || nbj[f] >= ny) continue;
                size_t Q = (size_t)nbj[f] * nx + nbi[f];
                double mob = 1.0 - 0.5 * (U[P] + U[Q]);
                double dv = V[Q] - V[P];
                nU[P] += bd1 * (-0.5) * dv / h2[f];
                nU[Q] += bd1 * (-0.5) * dv / h2[f];
                nV[Q] += bd1 * mob / h2[f];
                nV[P] -= bd1 * mob / h2[f];
            }
            /* fw += d2 = (Gx(i+1/2) - Gx(i-1/2)) + (Gy(j+1/2) - Gy(j-1/2)) */
            for (int f = 0; f < 4; ++f) {
                double sgn;
                int fi, fj, isx;
                if (f == 0) { if (i + 1 >= nx) continue; fi = i; fj = j; isx = 1; sgn = 1.0; }
                else if (f == 1) { if (i - 1 < 0) continue; fi = i - 1; fj = j; isx = 1; sgn = -1.0; }
                else if (f == 2) { if (j + 1 >= ny) continue; fi = i; fj = j; isx = 0; sgn = 1.0; }
                else { if (j - 1 < 0) continue; fi = i; fj = j - 1; isx = 0; sgn = -1.0; }
                double g = sgn * bw; /* dL/dG for this face, seen from cell P */
                if (isx) {
                    int L = fi, R = fi + 1;
                    int jn = clampi(fj + 1, 0, ny - 1), js = clampi(fj - 1, 0, ny - 1);
                    double kn = 0.5 / (dx * dx), kc = 0.25 / (dx * dy);
                    double dW = AT(W, R, fj) - AT(W, L, fj);
                    double sa = AT(a11, L, fj) + AT(a11, R, fj);
                    AT(ga11, L, fj) += g * kn * dW;
                    AT(ga11, R, fj) += g * kn * dW;
                    AT(nW, R, fj) += g * sa * kn;
                    AT(nW, L, fj) -= g * sa * kn;
                    AT(ga12, L, fj) += g * kc * (AT(W, L, jn) - AT(W, L, js));
                    AT(ga12, R, fj) += g * kc * (AT(W, R, jn) - AT(W, R, js));
                    AT(nW, L, jn) += g * kc * AT(a12, L, fj);
                    AT(nW, L, js) -= g * kc * AT(a12, L, fj);
                    AT(nW, R, jn) += g * kc * AT(a12, R, fj);
                    AT(nW, R, js) -= g * kc * AT(a12, R, fj);
                } else {
                    int S = fj, N = fj + 1;
                    int ie = clampi(fi + 1, 0, nx - 1), iw = clampi(fi - 1, 0, nx - 1);
                    double kn = 0.5 / (dy * dy), kc = 0.25 / (dy * dx);
                    double dW = AT(W, fi, N) - AT(W, fi, S);
                    double sa = AT(a22, fi, S) + AT(a22, fi, N);
                    AT(ga22, fi, S) += g * kn * dW;
                    AT(ga22, fi, N) += g * kn * dW;
                    AT(nW, fi, N) += g * sa * kn;
                    AT(nW, fi, S) -= g * sa * kn;
                    AT(ga12, fi, S) += g * kc * (AT(W, ie, S) - AT(W, iw, S));
                    AT(ga12, fi, N) += g * kc * (AT(W, ie, N) - AT(W, iw, N));
                    AT(nW, ie, S) += g * kc * AT(a12, fi, S);
                    AT(nW, iw, S) -= g * kc * AT(a12, fi, S);
                    AT(nW, ie, N) += g * kc * AT(a12, fi, N);
                    AT(nW, iw, N) -= g * kc * AT(a12, fi, N);
                }
            }
        }
    }
    memcpy(lamU, nU, n * sizeof(double));
    memcpy(lamV, nV, n * sizeof(double));
    memcpy(lamW, nW, n * sizeof(double));
    free(nu);
    return 0;
}

/* Discrete adjoint of nsteps steps from (U0,V0,W0), all states stored.
 * On entry lamU/lamV/lamW hold dL/d(U,V,W) at t_n; on exit dL/d(U,V,W) at t_0.
 * ga11/ga12/ga22 (n cells) and gs[4] are overwritten with dL/d(a11,a12,a22)
 * and dL/d(delta, rho, D, c).  Returns 0 or -1 on allocation failure. */
int ggo_adjoint(const ggo_problem* p, const double* a11, const double* a12, const double* a22,
                const double* U0, const double* V0, const double* W0, int64_t nsteps,
                double* lamU, double* lamV, double* lamW,
                double* ga11, double* ga12, double* ga22, double* gs)
{
    size_t n = (size_t)p->nx * (size_t)p->ny;
    size_t states = (size_t)nsteps + 1;
    double* X = (double*)malloc(3 * n * states * sizeof(double));
    if (!X) return -1;
    memcpy(X, U0, n * sizeof(double));
    memcpy(X + n, V0, n * sizeof(double));
    memcpy(X + 2 * n, W0, n * sizeof(double));
    for (int64_t k = 0; k < nsteps; ++k) {
        double* a = X + 3 * n * (size_t)k;
        double* b = a + 3 * n;
        ggo_step(p, a11, a12, a22, a, a + n, a + 2 * n, b, b + n, b + 2 * n);
    }
    memset(ga11, 0, n * sizeof(double));
    memset(ga12, 0, n * sizeof(double));
    memset(ga22, 0, n * sizeof(double));
    gs[0] = gs[1] = gs[2] = gs[3] = 0.0;
    for (int64_t k = nsteps - 1; k >= 0; --k) {
        double* a = X + 3 * n * (size_t)k;
        if (ggo_step_vjp(p, a11, a12, a22, a, a + n, a + 2 * n, lamU, lamV, lamW, ga11, ga12, ga22, gs)) {
            free(X);
            return -1;
        }
    }
    free(X);
    return 0;
}

/* Chain rule from dL/d(a11,a12,a22) to dL/d(theta, l1, l2) through
 * a11 = l1 cos^2 + l2 sin^2, a12 = (l1 - l2) sin cos, a22 = l1 sin^2 + l2 cos^2. */
void ggo_coefficients_vjp(int64_t n, const double* theta, const double* l1, const double* l2,
                          const double* ga11, const double* ga12, const double* ga22,
                          double* gtheta, double* gl1, double* gl2)
{
    for (int64_t k = 0; k < n; ++k) {
        double cs = cos(theta[k]), sn = sin(theta[k]);
        double d = l1[k] - l2[k];
        double da11 = -2.0 * d * sn * cs;           /* (l2 - l1) sin 2theta */
        double da12 = d * (cs * cs - sn * sn);      /* (l1 - l2) cos 2theta */
        double da22 = 2.0 * d * sn * cs;            /* (l1 - l2) sin 2theta */
        gtheta[k] = ga11[k] * da11 + ga12[k] * da12 + ga22[k] * da22;
        gl1[k] = ga11[k] * cs * cs + ga12[k] * sn * cs + ga22[k] * sn * sn;
        gl2[k] = ga11[k] * sn * sn - ga12[k] * sn * cs + ga22[k] * cs * cs;
    }
}
