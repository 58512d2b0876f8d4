"""The 8192 x 8192 heterogeneous tissue at full size, in the launch
configuration the benchmark times (the autotuned plan), checked on sampled
cells against the oracle and on properties that hold at any size.

Sampled cells: after n steps a cell depends only on the cells within n cells
of it (the nine-point stencil of Table 2 reaches one cell per step, Table 1
less), so the oracle, run on a window of half-width n + 2 around the cell
(clipped at the domain boundary, where the zero-flux condition is the true
one) with the full grid's time step, reproduces that cell exactly up to
rounding; the window's cut edges are wrong by their mirror ghosts, but that
error travels one cell per step and does not reach the centre."""
import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import gg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_01748_gb300 import build
    build()
    return inputs.hetero_8192()


def window_oracle(p, dt, i, j, n):
    """The oracle's value of cell (i, j) after n steps, from a window."""
    R = n + 2
    i0, i1 = max(0, i - R), min(p.nx, i + R + 1)
    j0, j1 = max(0, j - R), min(p.ny, j + R + 1)
    sl = (slice(j0, j1), slice(i0, i1))
    dx, dy = p.lx / p.nx, p.ly / p.ny
    s = oracle.Setup(i1 - i0, j1 - j0, p.delta, p.rho, p.D, p.c, dt, lx=(i1 - i0) * dx, ly=(j1 - j0) * dy)
    a = oracle.coefficients(p.theta[sl], p.lambda1[sl], p.lambda2[sl])
    U, V, W = oracle.run(s, *a, p.u0[sl], p.v0[sl], p.w0[sl], n)
    return U[j - j0, i - i0], V[j - j0, i - i0], W[j - j0, i - i0]


def test_sampled_cells_of_the_full_grid_match_the_oracle(full):
    p = full
    n = 48  # a multiple of every T the autotuner can pick
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        plan = sim.plan()
        sim.step(n)
        got = sim.state()
        dt = sim.dt
    rng = np.random.default_rng(2006)
    c = p.nx // 2
    r = int(0.1 * p.nx)  # the initial tumour's rim
    cells = [(0, 0), (p.nx - 1, 0), (0, p.ny - 1), (p.nx - 1, p.ny - 1), (c, 0), (0, c), (p.nx - 1, c),
             (c, p.ny - 1), (c, c), (c + r, c), (c, c - r), (c - r + 1, c + 1)]
    cells += [tuple(int(x) for x in rng.integers(0, p.nx, 2)) for _ in range(6)]
    scale = [max(float(np.max(np.abs(f))), 1e-300) for f in got]
    for i, j in cells:
        ref = window_oracle(p, dt, i, j, n)
        for name, g, rv, sc in zip("uvw", got, ref, scale):
            assert abs(g[j, i] - rv) <= 1e-5 * sc, (plan, i, j, name, g[j, i], rv)


def test_full_grid_against_the_fp64_kernel_and_invariants(full):
    """300 steps of the tuned FP32 + Kahan plan against the plain FP64
    kernel over the whole grid (relative max-norm 1e-5), then the rest of
    the benchmark's 5000 steps with the bounds of eq. (1) and no NaN."""
    p = full
    with gg.GGSim.from_problem(p, precision="fp64") as ref:
        ref.step(300)
        r = ref.state()
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        sim.step(300)
        g = sim.state()
        for a, b in zip(g, r):
            assert np.max(np.abs(a - b)) <= 1e-5 * np.max(np.abs(b))
        sim.step(p.steps - 300)
        d = sim.diagnostics()
        assert sim.steps == p.steps
    assert d["nonfinite"] == 0
    assert d["min"][0] >= 0 and d["max"][0] <= 1
    assert d["min"][1] >= 0 and d["max"][1] <= 1 + 1e-6
    assert d["tumour_area"] > np.pi * 0.1 ** 2 * 0.9  # the tumour has not shrunk
