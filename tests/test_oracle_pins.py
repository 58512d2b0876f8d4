"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
paper's printed stencils (Tables 1 and 2, transcribed under tests/golden/),
closed forms (Neumann cosine modes, polynomial exactness), exact invariants
(equilibria of eq. (1), conservation, transpose symmetry, 1D reduction), the
qualitative regimes of Section 2, and finite differences of the forward map
for the discrete adjoint.  None needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- eq. (2)

def test_tensor_is_rotated_diagonal():
    """A = R(theta) diag(l1, l2) R^T: eigenvalues l1, l2 and the eigenvector of
    l1 along (cos theta, sin theta)."""
    th = inputs.white_noise(7, 5, 11, 0.0, math.pi)
    l1 = inputs.white_noise(7, 5, 12, 0.1, 1.0)
    l2 = inputs.white_noise(7, 5, 13, 0.01, 0.09)   # l2 < l1 everywhere
    a11, a12, a22 = oracle.coefficients(th, l1, l2)
    for k in range(th.size):
        A = np.array([[a11.flat[k], a12.flat[k]], [a12.flat[k], a22.flat[k]]])
        w, v = np.linalg.eigh(A)
        assert np.allclose(w, [l2.flat[k], l1.flat[k]], rtol=0, atol=1e-15)
        e1 = np.array([math.cos(th.flat[k]), math.sin(th.flat[k])])
        assert abs(abs(e1 @ v[:, 1]) - 1.0) < 1e-14


def test_lambda_max_matches_eigvalsh():
    a11 = inputs.white_noise(9, 4, 21, 0.1, 1.0)
    a22 = inputs.white_noise(9, 4, 22, 0.1, 1.0)
    a12 = inputs.white_noise(9, 4, 23, -0.3, 0.3)
    ref = max(np.linalg.eigvalsh(np.array([[a, b], [b, c]])).max()
              for a, b, c in zip(a11.flat, a12.flat, a22.flat))
    assert abs(oracle.lambda_max(a11, a12, a22) - ref) < 1e-15


def test_dt_rule_below_diffusion_bound():
    """dt_max never exceeds h^2 / (4 Lambda) on a square grid; with
    c = rho = delta = 0 only the logistic rate 1 of U remains beside it."""
    h = 1.0 / 128
    assert oracle.dt_max(h, h, 1.0, 0.0, 0.0, 0.0, 0.0) == pytest.approx(1.0 / (4.0 / (h * h) + 1.0), rel=1e-15)
    for lam, delta, c in [(1.0, 12.5, 70.0), (0.01, 0.5, 70.0), (0.3, 20.0, 5.0)]:
        assert oracle.dt_max(h, h, lam, delta, 1.0, 4e-5, c) < h * h / (4.0 * lam)
    # Lambda is at least D
    assert oracle.dt_max(h, h, 1e-6, 0, 0, 1e-3, 0) == pytest.approx(1.0 / (4e-3 / (h * h) + 1.0), rel=1e-15)


def test_dt_rule_keeps_diagonals_nonnegative():
    """Under CFL <= 1 every diagonal coefficient of eq. (3) is >= 0 for a12 = 0:
    the counterexample that rules out min(diffusion, reaction) bounds."""
    for (h, lam, delta, rho, D, c) in [(1 / 100, 0.003, 0.5, 1, 4e-5, 70), (1 / 128, 1.0, 12.5, 1, 4e-5, 70),
                                       (1 / 16, 0.01, 20, 1, 1e-3, 70)]:
        dt = oracle.dt_max(h, h, lam, delta, rho, D, c)
        assert 1 - dt * (c + 4 * lam / h ** 2) >= 0        # W centre
        assert 1 - dt * (1 + delta) >= 0                   # U (U, W <= 1)
        assert 1 - dt * 4 * max(lam, D) / h ** 2 >= 0      # V centre


# --------------------------------------------------------------- adaptive Delta t_k

def _setup(nx, ny, delta=12.5, rho=1.0, D=4e-5, c=70.0, lx=1.0, ly=1.0, no_reaction=False):
    return oracle.Setup(nx, ny, delta, rho, D, c, 0.0, no_reaction, lx, ly)


def test_adaptive_dt_closed_forms():
    """Uniform and single-cell states where the rule's maxima are known by
    hand: the V bound with every face of an interior cell at mobility 1, the
    U bound of healthy tissue with acid, the static acid bound, and a corner
    cell (two faces) as the only cell with mobility 1/2."""
    nx, ny, lx, ly = 7, 5, 1.0, 0.6
    dx, dy = lx / nx, ly / ny
    lam, cfl = 0.2, 0.9
    kW = 70.0 + 2 * lam * (1 / dx ** 2 + 1 / dy ** 2)
    z, one = np.zeros((ny, nx)), np.ones((ny, nx))
    # U = V = W = 0, D = 3 lam: interior cells have four faces of mobility 1
    s = _setup(nx, ny, D=3 * lam, lx=lx, ly=ly)
    kV = 3 * lam * (2 / dx ** 2 + 2 / dy ** 2) - 1.0
    assert kV > kW
    assert oracle.adaptive_dt(s, lam, cfl, z, z, z) == pytest.approx(cfl / kV, rel=1e-15)
    # healthy tissue full of acid (U = V = W = 1): mobility 0, U bound delta
    s = _setup(nx, ny, delta=1e7, lx=lx, ly=ly)
    assert oracle.adaptive_dt(s, lam, cfl, one, one, one) == pytest.approx(cfl / 1e7, rel=1e-15)
    # U = 1, V = W = 0: only the acid bound is positive
    s = _setup(nx, ny, lx=lx, ly=ly)
    assert oracle.adaptive_dt(s, lam, cfl, one, z, z) == pytest.approx(cfl / kW, rel=1e-15)
    # without reactions the acid bound loses c
    s = _setup(nx, ny, lx=lx, ly=ly, no_reaction=True)
    assert oracle.adaptive_dt(s, lam, cfl, one, z, z) == pytest.approx(cfl / (kW - 70.0), rel=1e-15)
    # a tumour corner cell (U = 0) in healthy tissue, V = 1: its two faces
    # have mobility 1/2, every other face 0 or 1/2 on one side only
    U = one.copy()
    U[0, 0] = 0.0
    s = _setup(nx, ny, D=1e3, lx=lx, ly=ly)
    expect = 1e3 * 0.5 * (1 / dx ** 2 + 1 / dy ** 2)
    assert expect > kW
    assert oracle.adaptive_dt(s, lam, cfl, U, one, z) == pytest.approx(cfl / expect, rel=1e-15)


def _own_coefficients(s, a, U, V, W, dt):
    """d(U', V', W')_P / d(U, V, W)_P of one oracle step, by central
    differences with the cells perturbed three apart in x and y (so that no
    perturbed cell sees another in its nine-point stencil); exact for the
    quadratic step up to rounding."""
    st = oracle.Setup(s.nx, s.ny, s.delta, s.rho, s.D, s.c, dt, s.no_reaction, s.lx, s.ly)
    out = [np.zeros_like(U) for _ in range(3)]
    eps = 1e-4
    for f in range(3):
        for oy in range(3):
            for ox in range(3):
                m = np.zeros_like(U)
                m[oy::3, ox::3] = 1.0
                X = [U.copy(), V.copy(), W.copy()]
                Xp, Xm = [x.copy() for x in X], [x.copy() for x in X]
                Xp[f] += eps * m
                Xm[f] -= eps * m
                yp = oracle.step(st, *a, *Xp)[f]
                ym = oracle.step(st, *a, *Xm)[f]
                out[f] += m * (yp - ym) / (2 * eps)
    return out


def test_adaptive_dt_is_the_largest_step_keeping_own_coefficients():
    """On states where the logistic factors are frozen (V = 0 for V, U = 0
    for U), d V'_P / d V_P = 1 - dt kV_P and d U'_P / d U_P = 1 - dt kU_P, so
    the step's own derivative (the tumour operator of Table 1, not the
    rule's face sum) shows the rule: with the adaptive dt every such
    coefficient is >= 1 - cfl, and the binding one equals it."""
    nx, ny = 9, 7
    cfl = 0.8
    th = inputs.white_noise(nx, ny, 31, 0.0, math.pi)
    l1 = inputs.white_noise(nx, ny, 32, 0.1, 0.3)
    l2 = inputs.white_noise(nx, ny, 33, 0.05, 0.1)
    a = oracle.coefficients(th, l1, l2)
    lam = oracle.lambda_max(*a)
    z = np.zeros((ny, nx))
    # V bound binding: large D, rough mobility
    s = _setup(nx, ny, D=2.0, lx=1.0, ly=0.8)
    U = inputs.white_noise(nx, ny, 34, 0.0, 1.0)
    W = inputs.white_noise(nx, ny, 35, 0.0, 1.0)
    dt = oracle.adaptive_dt(s, lam, cfl, U, z, W)
    cV = _own_coefficients(s, a, U, z, W, dt)[1]
    assert cV.min() >= 1 - cfl - 1e-12
    assert cV.min() == pytest.approx(1 - cfl, abs=1e-9)
    # U bound binding: huge delta on U = 0 with acid
    s = _setup(nx, ny, delta=5e3)
    dt = oracle.adaptive_dt(s, lam, cfl, z, z, W)
    cU = _own_coefficients(s, a, z, z, W, dt)[0]
    assert cU.min() >= 1 - cfl - 1e-12
    assert cU.min() == pytest.approx(1 - cfl, abs=1e-9)


def test_adaptive_dt_never_below_the_fixed_step_and_runs():
    """For states in [0, 1] the adaptive step is at least the fixed step of
    the static rule; held for a whole run it reproduces the fixed-step run
    with that dt bit for bit; and on a tissue whose tumour region grows (large
    D, U -> 0 inside the disk) it shrinks over time while U, V, W stay in
    [0, 1] (a12 = 0)."""
    nx, ny = 24, 20
    p = inputs.plain_128(nx, ny, steps=0)
    a = oracle.coefficients(p.theta, p.lambda1, p.lambda2)
    lam = oracle.lambda_max(*a)
    s = _setup(nx, ny)
    for seed in range(3):
        U, V, W = inputs.random_state(nx, ny, 40 + seed)
        fixed = 0.9 * oracle.dt_max(s.dx, s.dy, lam, s.delta, s.rho, s.D, s.c)
        assert oracle.adaptive_dt(s, lam, 0.9, U, V, W) >= fixed
    U0, V0, W0 = inputs.random_state(nx, ny, 44)
    (Ua, Va, Wa), t, dt = oracle.run_adaptive(s, *a, lam, 0.9, 1000, U0, V0, W0, 30)
    assert dt == oracle.adaptive_dt(s, lam, 0.9, U0, V0, W0)
    assert t == pytest.approx(30 * dt, rel=1e-14)
    sf = oracle.Setup(nx, ny, s.delta, s.rho, s.D, s.c, dt)
    for x, y in zip((Ua, Va, Wa), oracle.run(sf, *a, U0, V0, W0, 30)):
        assert np.array_equal(x, y)
    # isotropic tissue, D = 4 lambda: the V bound takes over as U -> 0
    th = np.zeros((ny, nx))
    l = np.full((ny, nx), 0.05)
    a = oracle.coefficients(th, l, l)
    s = _setup(nx, ny, delta=3.0, rho=1.0, D=0.2, c=5.0)
    U0, V0, W0 = inputs.tumour_disk(nx, ny, 0.2)
    U0 = np.ones((ny, nx))  # healthy tissue with tumour cells: mobility 0 at first
    dts = []
    U, V, W = U0, V0, W0
    for _ in range(20):
        (U, V, W), t, dt = oracle.run_adaptive(s, *a, 0.05, 0.9, 25, U, V, W, 25)
        dts.append(dt)
        assert U.min() >= 0 and U.max() <= 1 and V.min() >= 0 and W.min() >= 0
    assert dts[-1] < 0.9 * dts[0]


# --------------------------------------------------------------- Tables 1, 2

def _read_stencil(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            ox, oy, expr = line.split(None, 2)
            rows.append((int(ox), int(oy), expr))
    assert len(rows) == 9
    return rows


def _dense_from_table(rows, nx, ny, dx, dy, fields):
    """Dense operator assembled straight from a table, interior rows only."""
    n = nx * ny
    M = np.zeros((n, n))
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            env = {"dx": dx, "dy": dy}
            for name, F in fields.items():
                env[name] = (lambda F: (lambda p, q: F[j + q, i + p]))(F)
            for ox, oy, expr in rows:
                M[j * nx + i, (j + oy) * nx + (i + ox)] += eval(expr, {"__builtins__": {}}, env)
    return M


def _interior(nx, ny):
    return np.array([j * nx + i for j in range(1, ny - 1) for i in range(1, nx - 1)])


def test_table1_tumour_stencil_literal():
    nx, ny = 7, 6
    dx, dy = 1.0 / nx, 1.3 / ny
    U = inputs.white_noise(nx, ny, 31)
    M = _dense_from_table(_read_stencil("table1_tumour_stencil.txt"), nx, ny, dx, dy, {"U": U})
    rows = _interior(nx, ny)
    for k in range(nx * ny):
        e = np.zeros(nx * ny)
        e[k] = 1.0
        col = oracle.tumour_operator(U, e.reshape(ny, nx), dx, dy).ravel()
        scale = 1.0 / min(dx, dy) ** 2
        assert np.max(np.abs(col[rows] - M[rows, k])) <= 1e-13 * scale


def test_table2_acid_stencil_literal():
    nx, ny = 7, 6
    dx, dy = 1.0 / nx, 1.3 / ny
    a = inputs.white_noise(nx, ny, 41, 0.1, 1.0)
    b = inputs.white_noise(nx, ny, 42, -0.4, 0.4)
    c = inputs.white_noise(nx, ny, 43, 0.1, 1.0)
    M = _dense_from_table(_read_stencil("table2_acid_stencil.txt"), nx, ny, dx, dy, {"a": a, "b": b, "c": c})
    rows = _interior(nx, ny)
    for k in range(nx * ny):
        e = np.zeros(nx * ny)
        e[k] = 1.0
        col = oracle.acid_operator(a, b, c, e.reshape(ny, nx), dx, dy).ravel()
        scale = 1.0 / min(dx, dy) ** 2
        assert np.max(np.abs(col[rows] - M[rows, k])) <= 1e-13 * scale


def test_tables_have_zero_row_sums():
    """Both printed stencils annihilate constants (a property of the tables)."""
    nx, ny = 5, 5
    U = inputs.white_noise(nx, ny, 51)
    a, b, c = (inputs.white_noise(nx, ny, s, 0.1, 1.0) for s in (52, 53, 54))
    for name, fields in [("table1_tumour_stencil.txt", {"U": U}),
                         ("table2_acid_stencil.txt", {"a": a, "b": b, "c": c})]:
        M = _dense_from_table(_read_stencil(name), nx, ny, 0.2, 0.2, fields)
        assert np.max(np.abs(M[_interior(nx, ny)].sum(axis=1))) < 1e-10


# --------------------------------------------------------------- invariants

def _hetero(nx, ny, seed):
    th, l1, l2 = inputs.heterogeneous_tensor(nx, ny, seed, 0.1, 1.0)
    return oracle.coefficients(th, l1, l2)


@pytest.mark.parametrize("state", [(1.0, 0.0, 0.0), (0.0, 1.0, 1.0), (0.0, 0.0, 0.0), (0.5, 1.0, 1.0)])
def test_constant_equilibria_bitwise(state):
    """(1,0,0), (0,1,1), (0,0,0) and (1-delta,1,1) with delta = 1/2 zero every
    rate of eq. (1) and every stencil difference, for any heterogeneous A."""
    nx, ny = 13, 9
    a = _hetero(nx, ny, 61)
    s = oracle.Setup(nx, ny, 0.5, 1.0, 4e-5, 70.0, 1e-4)
    U, V, W = (np.full((ny, nx), v) for v in state)
    U1, V1, W1 = oracle.run(s, *a, U, V, W, 50)
    assert np.array_equal(U1, U) and np.array_equal(V1, V) and np.array_equal(W1, W)


def test_mass_conservation_without_reactions():
    """Zero boundary flux and the flux form conserve sum V and sum W."""
    nx, ny = 24, 20
    p = inputs.plain_128(nx, ny)
    s, a = oracle.setup_for(p, no_reaction=True)
    s.D = 1e-2  # make the tumour flux non-trivial
    U, V, W = inputs.random_state(nx, ny, 71)
    m0 = oracle.diagnostics(U, V, W, s.dx, s.dy)["mass"]
    U1, V1, W1 = oracle.run(s, *a, U, V, W, 2000)
    m1 = oracle.diagnostics(U1, V1, W1, s.dx, s.dy)["mass"]
    assert np.array_equal(U1, U)
    assert abs(m1[1] - m0[1]) <= 1e-13 * m0[1]
    assert abs(m1[2] - m0[2]) <= 1e-13 * m0[2]
    assert np.max(np.abs(W1 - W)) > 1e-3  # it did move


def test_transpose_symmetry_bitwise():
    """Swapping x and y (a11 <-> a22, nx <-> ny, dx <-> dy, fields transposed)
    transposes the result exactly."""
    nx, ny = 11, 7
    a11, a12, a22 = _hetero(nx, ny, 81)
    U, V, W = inputs.random_state(nx, ny, 82)
    s = oracle.Setup(nx, ny, 3.0, 1.0, 3e-3, 70.0, 2e-5, lx=1.0, ly=0.8)
    sT = oracle.Setup(ny, nx, 3.0, 1.0, 3e-3, 70.0, 2e-5, lx=0.8, ly=1.0)
    r = oracle.run(s, a11, a12, a22, U, V, W, 30)
    rT = oracle.run(sT, a22.T, a12.T, a11.T, U.T, V.T, W.T, 30)
    for f, g in zip(r, rT):
        assert np.array_equal(f, g.T)


@pytest.mark.parametrize("k,l", [(1, 0), (2, 3), (5, 1)])
def test_neumann_cosine_closed_form(k, l):
    """Isotropic constant kappa, no reactions: cos(k pi x) cos(l pi y) at cell
    centres is an eigenvector of the zero-flux operator with eigenvalue
    -4 kappa [sin^2(k pi dx / 2)/dx^2 + sin^2(l pi dy / 2)/dy^2]."""
    nx, ny, kappa = 16, 12, 0.7
    s = oracle.Setup(nx, ny, 0.0, 0.0, 0.0, 0.0, 0.0, no_reaction=True)
    s.dt = 0.45 / (2 * kappa * (1 / s.dx ** 2 + 1 / s.dy ** 2))
    x = (np.arange(nx) + 0.5) * s.dx
    y = (np.arange(ny) + 0.5) * s.dy
    W0 = np.outer(np.cos(l * math.pi * y), np.cos(k * math.pi * x))
    g = 1 - 4 * s.dt * kappa * (math.sin(k * math.pi * s.dx / 2) ** 2 / s.dx ** 2
                                + math.sin(l * math.pi * s.dy / 2) ** 2 / s.dy ** 2)
    A = np.full((ny, nx), kappa), np.zeros((ny, nx)), np.full((ny, nx), kappa)
    n = 40
    _, _, Wn = oracle.run(s, *A, np.zeros((ny, nx)), np.zeros((ny, nx)), W0, n)
    assert np.max(np.abs(Wn - g ** n * W0)) < 1e-13


def test_polynomial_exactness_interior():
    """On cells away from the boundary: W = x^2, xy, y^2 with constant A gives
    D2 = 2 a11, 2 a12, 2 a22; W = x^2 with a11 = x gives 4x; V = x^2 with
    U = x gives D1 = 2 - 4x."""
    nx, ny = 10, 8
    dx, dy = 1.0 / nx, 1.0 / ny
    x = ((np.arange(nx) + 0.5) * dx)[None, :] * np.ones((ny, 1))
    y = ((np.arange(ny) + 0.5) * dy)[:, None] * np.ones((1, nx))
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    A = (np.full((ny, nx), 0.8), np.full((ny, nx), -0.3), np.full((ny, nx), 0.5))
    for Wf, expect in [(x * x, 2 * 0.8), (x * y, 2 * -0.3), (y * y, 2 * 0.5)]:
        d2 = oracle.acid_operator(*A, Wf, dx, dy)
        assert np.max(np.abs(d2[inner] - expect)) < 1e-11
    d2 = oracle.acid_operator(x, np.zeros_like(x), np.ones_like(x), x * x, dx, dy)
    assert np.max(np.abs(d2[inner] - 4 * x[inner])) < 1e-11
    d1 = oracle.tumour_operator(x, x * x, dx, dy)
    assert np.max(np.abs(d1[inner] - (2 - 4 * x[inner]))) < 1e-11


def test_positivity_isotropic_and_parity_of_anisotropic_minimum():
    """With a12 = 0 the CFL step keeps U in [0,1] and V, W >= 0 (a monotone
    scheme).  With a12 != 0 the corner coefficients of Table 2 have both signs,
    so W >= 0 is not guaranteed: only U, V bounds are asserted."""
    nx = ny = 48
    p = inputs.plain_128(nx, ny, steps=600)
    th0 = np.zeros_like(p.theta)
    s, a = oracle.setup_for(p)
    a_iso = oracle.coefficients(th0, p.lambda1, p.lambda2)
    for coeffs, check_w in [(a_iso, True), (a, False)]:
        U, V, W = oracle.run(s, *coeffs, p.u0, p.v0, p.w0, p.steps)
        assert U.min() >= 0 and U.max() <= 1 and V.min() >= 0 and V.max() <= 1
        if check_w:
            assert W.min() >= 0


# --------------------------------------------------------------- 1D reduction and regimes

def _oned_reference(U, V, W, a11, dx, dy, delta, rho, D, c, dt, n):
    """Independent three-point 1D scheme (numpy), zero flux at both ends."""
    U, V, W = U.copy(), V.copy(), W.copy()
    for _ in range(n):
        m = 1 - 0.5 * (U[1:] + U[:-1])
        Hv = m * (V[1:] - V[:-1]) / dx ** 2
        d1 = np.zeros_like(V)
        d1[:-1] += Hv
        d1[1:] -= Hv
        Gw = 0.5 * (a11[1:] + a11[:-1]) * (W[1:] - W[:-1]) / dx ** 2
        d2 = np.zeros_like(W)
        d2[:-1] += Gw
        d2[1:] -= Gw
        U, V, W = (U + dt * (U * (1 - U) - delta * U * W),
                   V + dt * (rho * V * (1 - V) + D * d1),
                   W + dt * (c * (V - W) + d2))
    return U, V, W


def test_one_dimensional_reduction():
    """y-uniform data with a y-independent diagonal tensor stays y-uniform
    (exactly) and matches an independent 1D three-point scheme."""
    nx, ny = 40, 6
    x = (np.arange(nx) + 0.5) / nx
    l1 = 0.2 + 0.8 * x ** 2
    a11 = np.tile(l1, (ny, 1))
    a22 = np.tile(0.3 + 0 * x, (ny, 1))
    a12 = np.zeros((ny, nx))
    U0 = np.tile(np.where(x < 0.2, 0.0, 1.0), (ny, 1))
    V0 = 1 - U0
    W0 = np.zeros((ny, nx))
    s = oracle.Setup(nx, ny, 3.0, 1.0, 1e-3, 70.0, 2e-5)
    U, V, W = oracle.run(s, a11, a12, a22, U0, V0, W0, 400)
    for F in (U, V, W):
        assert np.array_equal(F, np.tile(F[0], (ny, 1)))
    Ur, Vr, Wr = _oned_reference(U0[0], V0[0], W0[0], l1, s.dx, s.dy, 3.0, 1.0, 1e-3, 70.0, 2e-5, 400)
    assert np.max(np.abs(U[0] - Ur)) < 1e-13
    assert np.max(np.abs(V[0] - Vr)) < 1e-13
    assert np.max(np.abs(W[0] - Wr)) < 1e-13


def _front_run(delta, nx=100, T=10.0, lam=1.0, D=4e-5, c=70.0, rho=1.0, xt=0.3):
    x = (np.arange(nx) + 0.5) / nx
    a = oracle.coefficients(np.zeros((1, nx)), np.full((1, nx), lam), np.full((1, nx), lam))
    dt = oracle.stable_dt(nx, 1, *a, delta, rho, D, c)
    s = oracle.Setup(nx, 1, delta, rho, D, c, dt)
    U0 = np.ones((1, nx))
    V0 = np.where(x < xt, 1.0, 0.0)[None, :]
    U, V, W = oracle.run(s, *a, U0, V0, np.zeros((1, nx)), int(T / dt))
    return x, U[0], V[0], W[0]


def test_heterogeneous_invasion_regime():
    """d < 1 (Section 2, item 1): tumour and normal cells coexist behind the
    front, with U at the kinetic equilibrium 1 - d W of eq. (1)."""
    x, U, V, W = _front_run(0.5)
    bulk = x < 0.1
    assert np.all(V[bulk] > 0.99)
    assert np.all(U[bulk] > 0.4)
    assert np.max(np.abs(U[bulk] - (1 - 0.5 * W[bulk]))) < 0.01


def test_homogeneous_invasion_gap_regime():
    """d > 1 (Section 2, item 2): healthy tissue is destroyed behind the front
    and an interstitial gap (U and V both negligible) opens ahead of it."""
    x, U, V, W = _front_run(12.5)
    assert np.all(U[V > 0.5] < 1e-6)
    gap = (U < 0.01) & (V < 0.01)
    assert gap.sum() * (x[1] - x[0]) >= 0.05


# --------------------------------------------------------------- diagnostics

def test_diagnostics_definitions():
    nx, ny = 9, 7
    U, V, W = inputs.random_state(nx, ny, 91)
    U[2, 3] = 0.001
    V[2, 3] = 0.002
    U[0, 0], V[0, 0] = 0.003, 0.7   # only U below the gap threshold
    U[1, 1], V[1, 1] = 0.6, 0.004   # only V below it
    W[4, 4] = np.nan
    d = oracle.diagnostics(U, V, W, 0.1, 0.2, eps=0.01)
    assert d["nonfinite"] == 1
    assert d["mass"][0] == pytest.approx(0.02 * U.sum(), rel=1e-14)
    assert d["max"][1] == V.max() and d["min"][0] == U.min()
    assert d["mass"][2] == pytest.approx(0.02 * np.nansum(W), rel=1e-14)
    assert d["tumour_area"] == pytest.approx(0.02 * (V > 0.5).sum())
    assert d["gap_area"] == pytest.approx(0.02 * ((U < 0.01) & (V < 0.01)).sum())
    assert ((U < 0.01) & (V < 0.01)).sum() == 1


# --------------------------------------------------------------- fronts and the interstitial gap

def test_front_rays_measure_a_drawn_disk_and_annulus():
    """Tumour (V = 1) inside radius rT, healthy tissue (U = 1) outside rH,
    nothing between: each ray sees the front at rT, the healthy edge at rH
    and a gap of rH - rT, to within one cell of its direction; the ray
    integral of V is the tumour radius (plus the centre cell's half)."""
    nx, ny, lx, ly = 60, 120, 1.0, 1.0
    dx, dy = lx / nx, ly / ny
    i0, j0 = 30, 60
    xc, yc = (i0 + 0.5) * dx, (j0 + 0.5) * dy
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    r = np.hypot(x[None, :] - xc, y[:, None] - yc)
    rT, rH = 0.2, 0.3
    V = np.where(r < rT, 1.0, 0.0)
    U = np.where(r > rH, 1.0, 0.0)
    f = oracle.front_rays(U, V, dx, dy, i0, j0)
    for d, h in enumerate((dx, dx, dy, dy)):
        assert abs(f["front"][d] - rT) <= h
        assert abs(f["edge"][d] - rH) <= h
        assert abs(f["gap"][d] - (rH - rT)) <= 2 * h
        assert abs(f["mass_v"][d] - (rT + h / 2)) <= h
    # no tumour: front 0, the healthy edge where U first exceeds 1/2
    f0 = oracle.front_rays(U, 0 * V, dx, dy, i0, j0)
    assert np.all(f0["front"] == 0) and np.all(f0["mass_v"] == 0)
    assert abs(f0["edge"][0] - rH) <= dx
    # healthy cells coexisting inside the tumour (U = 0.8 there): the edge is
    # still the first healthy cell beyond the front
    fc = oracle.front_rays(np.where(r < rT, 0.8, U), V, dx, dy, i0, j0)
    for d, h in enumerate((dx, dx, dy, dy)):
        assert abs(fc["edge"][d] - rH) <= h
    # seen from 6 columns west of the disk centre the east front is 6 cells
    # farther and the west front 6 cells nearer
    fo = oracle.front_rays(U, V, dx, dy, i0 - 6, j0)
    assert abs(fo["front"][0] - (rT + 6 * dx)) <= dx
    assert abs(fo["front"][1] - (rT - 6 * dx)) <= dx


def test_front_rays_are_mirror_symmetric():
    """A state mirrored about the centre column gives equal east and west
    results, and mirrored about the centre row equal north and south ones."""
    nx, ny = 41, 33
    i0, j0 = 20, 16
    U, V, W = inputs.random_state(nx, ny, 77)
    U = 0.5 * (U + U[:, ::-1])
    V = 0.5 * (V + V[:, ::-1])
    U = 0.5 * (U + U[::-1, :])
    V = 0.5 * (V + V[::-1, :])
    f = oracle.front_rays(U, V, 1 / nx, 1 / ny, i0, j0, v_front=0.4, u_edge=0.6, eps=0.3)
    for key in ("front", "edge", "gap", "mass_v", "mass_u"):
        assert f[key][0] == pytest.approx(f[key][1], rel=1e-14, abs=1e-15), key
        assert f[key][2] == pytest.approx(f[key][3], rel=1e-14, abs=1e-15), key


def test_front_speed_is_the_fisher_kpp_speed():
    """With U = 0 the V equation of eq. (1) is Fisher-KPP,
    V_t = rho V(1-V) + D V_xx, whose fronts from steep data travel at
    2 sqrt(rho D) less a lag that decays like 3/(2 lambda t), lambda =
    sqrt(rho/D) (Bramson).  The LeVeque-Yee speed of the scheme over
    t in [20, 30] matches that (the lag is 3 % there) to 1.5 %, the size of
    the next, unmodelled term of the expansion at t = 20 (a wrong D or rho
    moves it by tens of percent), and the front position moves at the same
    speed."""
    nx, lx = 1000, 2.0
    rho, D = 1.0, 2.5e-4
    x = (np.arange(nx) + 0.5) * lx / nx
    a = oracle.coefficients(np.zeros((1, nx)), np.full((1, nx), D), np.full((1, nx), D))
    dt = oracle.stable_dt(nx, 1, *a, 0.0, rho, D, 0.0, lx=lx)
    s = oracle.Setup(nx, 1, 0.0, rho, D, 0.0, dt, lx=lx)
    U0 = np.zeros((1, nx))
    V0 = np.where(x < 0.1, 1.0, 0.0)[None, :]
    W0 = np.zeros((1, nx))
    n1, n2 = int(round(20 / dt)), int(round(30 / dt))
    U1, V1, W1 = oracle.run(s, *a, U0, V0, W0, n1)
    U2, V2, W2 = oracle.run(s, *a, U1, V1, W1, n2 - n1)
    assert np.all(U2 == 0)
    f1 = oracle.front_rays(U1, V1, s.dx, s.dy, 0, 0)
    f2 = oracle.front_rays(U2, V2, s.dx, s.dy, 0, 0)
    elapsed = (n2 - n1) * dt
    speed = oracle.front_speed(f1, f2, elapsed)[0]
    cstar = 2 * np.sqrt(rho * D)
    lam = np.sqrt(rho / D)
    expected = cstar - 3 / (2 * lam) * np.log(30 / 20) / 10
    assert speed == pytest.approx(expected, rel=0.015)
    assert (f2["front"][0] - f1["front"][0]) / elapsed == pytest.approx(expected, abs=2 * s.dx / elapsed + 0.015 * cstar)


def test_front_rays_see_the_two_invasion_regimes():
    """Section 2: d > 1 opens an interstitial gap ahead of the tumour front,
    d < 1 leaves none (tumour and healthy cells coexist behind the front)."""
    for delta, has_gap in ((12.5, True), (0.5, False)):
        x, U, V, W = _front_run(delta)
        f = oracle.front_rays(U[None, :], V[None, :], x[1] - x[0], 1.0, 0, 0)
        assert f["front"][0] > 0.3
        assert (f["gap"][0] >= 0.05) == has_gap, delta
        if not has_gap:
            assert f["gap"][0] == 0


# --------------------------------------------------------------- discrete adjoint

def _problem_small(nx=12, ny=10, seed=101):
    th, l1, l2 = inputs.heterogeneous_tensor(nx, ny, seed, 0.1, 1.0)
    U, V, W = inputs.random_state(nx, ny, seed + 1)
    s = oracle.Setup(nx, ny, 2.5, 1.3, 2e-3, 7.0, 0.0, lx=1.0, ly=0.9)
    a = oracle.coefficients(th, l1, l2)
    s.dt = 0.8 * oracle.stable_dt(nx, ny, *a, s.delta, s.rho, s.D, s.c, cfl=1.0, lx=1.0, ly=0.9)
    return s, (th, l1, l2), a, (U, V, W)


def test_one_step_adjoint_is_exact_transpose():
    """One step is quadratic in the state and linear in (a11, a12, a22, delta,
    rho, D, c), so central differences give its Jacobian exactly up to
    rounding: <J dx, lam> must equal <dx, J^T lam> to ~1e-12."""
    s, _, a, X = _problem_small()
    ny, nx = X[0].shape
    lam = [inputs.white_noise(nx, ny, 111 + k, -1, 1) for k in range(3)]
    dX = [inputs.white_noise(nx, ny, 121 + k, -1, 1) for k in range(3)]
    (lu, lv, lw), ga, gs = oracle.step_vjp(s, *a, *X, *lam)
    eps = 1e-3

    def F(Xs, A=a, ss=s):
        return oracle.step(ss, *A, *Xs)

    Fp = F([x + eps * d for x, d in zip(X, dX)])
    Fm = F([x - eps * d for x, d in zip(X, dX)])
    lhs = sum(np.sum((p - m) / (2 * eps) * l) for p, m, l in zip(Fp, Fm, lam))
    rhs = sum(np.sum(d * g) for d, g in zip(dX, (lu, lv, lw)))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))
    # coefficients
    dA = [inputs.white_noise(nx, ny, 131 + k, -1, 1) for k in range(3)]
    Fp = F(X, A=[x + eps * d for x, d in zip(a, dA)])
    Fm = F(X, A=[x - eps * d for x, d in zip(a, dA)])
    lhs = sum(np.sum((p - m) / (2 * eps) * l) for p, m, l in zip(Fp, Fm, lam))
    rhs = sum(np.sum(d * g) for d, g in zip(dA, ga))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))
    # scalars
    for k, name in enumerate(["delta", "rho", "D", "c"]):
        sp = oracle.Setup(**{**s.__dict__})
        sm = oracle.Setup(**{**s.__dict__})
        setattr(sp, name, getattr(s, name) + eps)
        setattr(sm, name, getattr(s, name) - eps)
        lhs = sum(np.sum((p - m) / (2 * eps) * l) for p, m, l in zip(F(X, ss=sp), F(X, ss=sm), lam))
        assert abs(lhs - gs[k]) <= 1e-11 * max(1.0, abs(lhs))


def test_adjoint_matches_finite_differences():
    """Gradient of the final-state misfit over many steps against central
    differences of the forward oracle (dt held fixed)."""
    s, (th, l1, l2), a, X = _problem_small(nx=10, ny=9, seed=141)
    n = 60
    Vstar = inputs.random_state(s.nx, s.ny, 149)[1]

    def loss(th_, l1_, l2_, ss=s):
        A = oracle.coefficients(th_, l1_, l2_)
        _, V, _ = oracle.run(ss, *A, *X, n)
        return oracle.misfit(V, Vstar, ss.dx, ss.dy)

    U, V, W = oracle.run(s, *a, *X, n)
    gV = oracle.misfit_grad(V, Vstar, s.dx, s.dy)
    _, ga, gs = oracle.adjoint(s, *a, *X, n, np.zeros_like(U), gV, np.zeros_like(W))
    gth, gl1, gl2 = oracle.coefficients_vjp(th, l1, l2, *ga)
    # the misfit is O(1e-2) and the tensor gradients O(1e-8): a large step keeps
    # the rounding of the differences (~1e-16 L / eps) well below the tolerance;
    # the O(eps^2) truncation error stays below it too.
    eps = 1e-3
    rng = np.random.default_rng(0)
    cells = rng.choice(s.nx * s.ny, size=8, replace=False)
    for field, grad in [(0, gth), (1, gl1), (2, gl2)]:
        scale = np.max(np.abs(grad))
        for k in cells:
            args_p = [th.copy(), l1.copy(), l2.copy()]
            args_m = [th.copy(), l1.copy(), l2.copy()]
            args_p[field].flat[k] += eps
            args_m[field].flat[k] -= eps
            fd = (loss(*args_p) - loss(*args_m)) / (2 * eps)
            assert abs(fd - grad.flat[k]) <= 1e-5 * scale
    for k, name in enumerate(["delta", "rho", "D", "c"]):
        sp = oracle.Setup(**{**s.__dict__})
        sm = oracle.Setup(**{**s.__dict__})
        h = 1e-4 * max(1.0, abs(getattr(s, name)))
        setattr(sp, name, getattr(s, name) + h)
        setattr(sm, name, getattr(s, name) - h)
        fd = (loss(th, l1, l2, ss=sp) - loss(th, l1, l2, ss=sm)) / (2 * h)
        assert abs(fd - gs[k]) <= 1e-5 * max(abs(fd), 1e-6)


def test_coefficient_chain_rule_matches_finite_differences():
    th = inputs.white_noise(6, 5, 151, 0, math.pi)
    l1 = inputs.white_noise(6, 5, 152, 0.1, 1.0)
    l2 = inputs.white_noise(6, 5, 153, 0.1, 1.0)
    g = [inputs.white_noise(6, 5, 154 + k, -1, 1) for k in range(3)]
    gt, g1, g2 = oracle.coefficients_vjp(th, l1, l2, *g)
    eps = 1e-6
    for which, grad in [(0, gt), (1, g1), (2, g2)]:
        p = [th.copy(), l1.copy(), l2.copy()]
        m = [th.copy(), l1.copy(), l2.copy()]
        p[which] += eps
        m[which] -= eps
        Ap, Am = oracle.coefficients(*p), oracle.coefficients(*m)
        fd = sum((x - y) / (2 * eps) * gg for x, y, gg in zip(Ap, Am, g))
        assert np.max(np.abs(fd - grad)) < 1e-9

