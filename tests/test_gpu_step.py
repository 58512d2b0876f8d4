"""Parity of the CUDA forward step (libgg.so, called through the C ABI) with
the FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative max-norm per field, max|F_gpu - F_orc| / max|F_orc|):
  plain FP64 kernel         1e-12 (only the rounding order differs);
  fused FP32 + Kahan        1e-5 (the target precision of the FP32 path);
  fused FP32, no Kahan      1e-4 (documented drift of uncompensated updates).
"""
import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import build, gg, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32_kahan": 1e-5, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    gg.lib()


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def run_oracle(p, steps, dt=None, no_reaction=False):
    s, a = oracle.setup_for(p, dt=dt, no_reaction=no_reaction)
    return s, oracle.run(s, *a, p.u0, p.v0, p.w0, steps)


def run_gpu(p, steps, precision, **kw):
    with gg.GGSim.from_problem(p, precision=precision, **kw) as sim:
        sim.step(steps)
        return sim.dt, sim.state()


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan", "fp32"])
def test_plain_128_config_full_run(precision):
    """128 x 128, delta=12.5, rho=1, D=4e-5, c=70, 2000 steps at CFL 0.9."""
    p = inputs.plain_128()
    s, ref = run_oracle(p, p.steps)
    dt, got = run_gpu(p, p.steps, precision)
    assert abs(dt - s.dt) <= 1e-14 * s.dt
    for name, g, r in zip("uvw", got, ref):
        err = rel_err(g, r)
        assert err <= TOL[precision], f"{name}: {err:.3e}"


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (9, 1), (2, 2), (3, 5), (37, 29), (300, 173), (257, 130)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_ragged_and_degenerate_grids(nx, ny, precision):
    """Empty-ish, one-row, one-column and ragged grids spanning several strips
    and chunks, on a rectangle (dx != dy)."""
    p = inputs.plain_128(nx, ny, steps=60)
    p.lx, p.ly = 1.0, 0.7
    p.u0, p.v0, p.w0 = inputs.random_state(nx, ny, 7 + nx)
    s, ref = run_oracle(p, p.steps)
    _, got = run_gpu(p, p.steps, precision)
    for name, g, r in zip("uvw", got, ref):
        assert rel_err(g, r) <= TOL[precision], name


PLANS = ([("warp", T) for T in (1, 2, 3, 4)] + [("warp2", T) for T in (1, 2, 3, 4)]
         + [("smem", T) for T in range(1, 9)])


@pytest.mark.parametrize("kind,T", PLANS)
def test_temporal_blocking_matches_oracle(kind, T):
    """T steps per HBM pass with both kernels: 29 steps (not a multiple of T)
    on a grid whose strips and chunks have ragged tails."""
    p = inputs.plain_128(300, 173, steps=29)
    p.u0, p.v0, p.w0 = inputs.random_state(300, 173, 5)
    s, ref = run_oracle(p, p.steps)
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        sim.set_plan(kind, T, chunk=40)
        sim.step(p.steps)
        got = sim.state()
    for name, g, r in zip("uvw", got, ref):
        assert rel_err(g, r) <= 1e-5, name


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp32"])
def test_every_plan_is_bitwise_identical(precision):
    """Each level of a temporally blocked pass, in either kernel, runs the
    same per-cell arithmetic (rates_v) as a single step, so every plan gives
    the same bits."""
    p = inputs.plain_128(200, 150, steps=24)
    p.u0, p.v0, p.w0 = inputs.random_state(200, 150, 9)
    base = None
    for kind, T in PLANS:
        for chunk in (0, 17):
            with gg.GGSim.from_problem(p, precision=precision) as sim:
                sim.set_plan(kind, T, chunk=chunk)
                sim.step(p.steps)
                got = sim.state(fp64=False)
            if base is None:
                base = got
            else:
                for g, b in zip(got, base):
                    assert np.array_equal(g, b), (kind, T, chunk)


@pytest.mark.parametrize("nx,ny", [(1, 6), (5, 1), (3, 5), (77, 45), (131, 29), (64, 33)])
def test_paired_column_plans_on_ragged_grids(nx, ny):
    """The paired-column kernel on odd widths (its last pair reads one column
    of the row only), widths below one strip and single rows or columns:
    every T and chunk height gives the bits of the one-column kernel."""
    p = inputs.plain_128(nx, ny, steps=13)
    p.u0, p.v0, p.w0 = inputs.random_state(nx, ny, 3 + nx + ny)
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        sim.set_plan("warp", 1)
        sim.step(p.steps)
        base = sim.state(fp64=False)
    for T in (1, 2, 3, 4):
        for chunk in (0, 7):
            with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
                sim.set_plan("warp2", T, chunk=chunk)
                assert sim.plan()["kind"] == "warp2"
                sim.step(p.steps)
                for g, b in zip(sim.state(fp64=False), base):
                    assert np.array_equal(g, b), (T, chunk)


def test_autotuner_keeps_the_state_and_the_bits():
    p = inputs.plain_128(700, 520, steps=40)
    p.u0, p.v0, p.w0 = inputs.random_state(700, 520, 19)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", steps_per_pass=1) as a:
        before = a.state(fp64=False)
        chosen = a.autotune(trial_steps=24)
        assert chosen["T"] >= 1
        for x, y in zip(before, a.state(fp64=False)):
            assert np.array_equal(x, y)
        a.step(40)
        tuned = a.state(fp64=False)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", steps_per_pass=1) as b:
        b.step(40)
        for x, y in zip(tuned, b.state(fp64=False)):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("state", [(1.0, 0.0, 0.0), (0.0, 1.0, 1.0), (0.0, 0.0, 0.0), (0.5, 1.0, 1.0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan", "fp32"])
def test_constant_equilibria_bitwise(state, precision):
    nx, ny = 70, 45
    p = inputs.plain_128(nx, ny, steps=40)
    p.delta = 0.5
    p.u0, p.v0, p.w0 = (np.full((ny, nx), v) for v in state)
    _, got = run_gpu(p, p.steps, precision, steps_per_pass=3 if precision != "fp64" else 0)
    for g, v in zip(got, state):
        assert np.all(g == v)


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_mass_conservation_without_reactions(precision):
    nx, ny = 160, 120
    p = inputs.plain_128(nx, ny)
    p.D = 1e-2
    p.u0, p.v0, p.w0 = inputs.random_state(nx, ny, 71)
    with gg.GGSim.from_problem(p, precision=precision, no_reaction=True) as sim:
        m0 = sim.diagnostics()["mass"]
        sim.step(2000)
        m1 = sim.diagnostics()["mass"]
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert abs(m1[1] - m0[1]) <= tol * m0[1]
    assert abs(m1[2] - m0[2]) <= tol * m0[2]


def test_diagnostics_match_oracle():
    p = inputs.plain_128(130, 97, steps=300)
    s, ref = run_oracle(p, p.steps)
    with gg.GGSim.from_problem(p, precision="fp64") as sim:
        sim.step(p.steps)
        d = sim.diagnostics(eps=0.05)
    o = oracle.diagnostics(*ref, s.dx, s.dy, eps=0.05)
    assert np.allclose(d["mass"], o["mass"], rtol=1e-12, atol=0)
    assert np.allclose(d["min"], o["min"], rtol=1e-12, atol=1e-15)
    assert np.allclose(d["max"], o["max"], rtol=1e-12, atol=0)
    assert d["nonfinite"] == 0
    assert d["tumour_area"] == pytest.approx(o["tumour_area"])
    assert d["gap_area"] == pytest.approx(o["gap_area"])


def test_checkpoint_resume_is_bitwise():
    """Reading the state (with Kahan terms) and writing it into a fresh
    simulation continues the run bit for bit."""
    p = inputs.plain_128(140, 90, steps=100)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", steps_per_pass=4) as a:
        a.step(50)
        snap = {f: a.read(f, fp64=False) for f in ("u", "v", "w", "comp_u", "comp_v", "comp_w")}
        a.step(50)
        full = a.state(fp64=False)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", steps_per_pass=4) as b:
        for f, arr in snap.items():
            b.write(f, arr)
        b.step(50)
        resumed = b.state(fp64=False)
    for x, y in zip(full, resumed):
        assert np.array_equal(x, y)


def test_transpose_symmetry():
    nx, ny = 90, 61
    p = inputs.plain_128(nx, ny, steps=80)
    p.lx, p.ly = 1.0, 0.8
    p.u0, p.v0, p.w0 = inputs.random_state(nx, ny, 82)
    q = inputs.plain_128(ny, nx, steps=80)
    q.lx, q.ly = 0.8, 1.0
    q.theta = np.ascontiguousarray(np.pi / 2 - p.theta.T)
    q.lambda1, q.lambda2 = np.ascontiguousarray(p.lambda1.T), np.ascontiguousarray(p.lambda2.T)
    q.u0, q.v0, q.w0 = (np.ascontiguousarray(x.T) for x in (p.u0, p.v0, p.w0))
    for precision, tol in (("fp64", 1e-12), ("fp32_kahan", 1e-6)):
        dt_p = gg.GGSim.from_problem(p, precision="fp64").dt
        _, a = run_gpu(p, p.steps, precision, dt=dt_p)
        _, b = run_gpu(q, q.steps, precision, dt=dt_p)
        for x, y in zip(a, b):
            assert rel_err(y.T, x) <= tol


def test_invalid_inputs_are_reported():
    p = inputs.plain_128(16, 16)
    bad = p.lambda1.copy()
    bad[3, 4] = -0.1
    with pytest.raises(gg.GGError) as e:
        gg.GGSim(16, 16, p.theta, bad, p.lambda2, p.u0, p.v0, p.w0, 1, 1, 1e-3, 70)
    assert e.value.status == gg.GG_ERR_NOT_SPD
    u = p.u0.copy()
    u[0, 0] = np.nan
    with pytest.raises(gg.GGError) as e:
        gg.GGSim(16, 16, p.theta, p.lambda1, p.lambda2, u, p.v0, p.w0, 1, 1, 1e-3, 70)
    assert e.value.status == gg.GG_ERR_ARG
    with pytest.raises(gg.GGError) as e:
        gg.GGSim(16, 16, p.theta, p.lambda1, p.lambda2, p.u0, p.v0, p.w0, 1, 1, 1e-3, 70, dt=1.0)
    assert e.value.status == gg.GG_ERR_CFL
    with gg.GGSim(16, 16, p.theta, p.lambda1, p.lambda2, p.u0, p.v0, p.w0, 1, 1, 1e-3, 70, dt=5e-3,
                  allow_unstable=True, precision="fp32") as sim:
        sim.step(400)
        d = sim.diagnostics()
        assert d["nonfinite"] > 0 and d["status"] == gg.GG_ERR_NONFINITE


def test_dt_rule_matches_oracle():
    for p in (inputs.plain_128(), inputs.layered_1024(nx=256), inputs.hetero_8192(nx=256)):
        s, a = oracle.setup_for(p)
        with gg.GGSim.from_problem(p, precision="fp32") as sim:
            assert sim.dt == pytest.approx(s.dt, rel=1e-14)
            assert sim.dt <= (1.0 / p.nx) ** 2 / (4 * oracle.lambda_max(*a))


def test_tensor_entries_match_oracle():
    p = inputs.hetero_8192(nx=96, ny=80)
    a = oracle.coefficients(p.theta, p.lambda1, p.lambda2)
    with gg.GGSim.from_problem(p, precision="fp64") as sim:
        for f, r in zip(("a11", "a12", "a22"), a):
            assert np.max(np.abs(sim.read(f) - r)) <= 1e-15
    with gg.GGSim.from_problem(p, precision="fp32") as sim:
        for f, r in zip(("a11", "a12", "a22"), a):
            assert np.max(np.abs(sim.read(f) - r)) <= 1e-15 * np.max(np.abs(r))
        # the weights the FP32 kernels read (Table 2), rounded once from FP64
        dx, dy = 1.0 / p.nx, 1.0 / p.ny
        a11, a12, a22 = a
        fx = np.zeros_like(a11)
        fx[:, :-1] = (a11[:, :-1] + a11[:, 1:]) / (2 * dx * dx)
        fy = np.zeros_like(a22)
        fy[:-1, :] = (a22[:-1, :] + a22[1:, :]) / (2 * dy * dy)
        for f, r in (("face_x", fx), ("face_y", fy), ("cross", a12 / (4 * dx * dy))):
            got = sim.read(f)
            assert np.all(np.abs(got - r) <= 6e-8 * np.abs(r) + 1e-30), f
        assert np.all(sim.read("face_x")[:, -1] == 0) and np.all(sim.read("face_y")[-1, :] == 0)


@pytest.mark.parametrize("delta", [0.5, 12.5])
def test_layered_1024_prefix_and_full_run(delta):
    """Layered tissue (1024 x 1024): the first 150 steps element by element
    against the oracle; the full 20000 steps of FP32 + Kahan against the
    plain FP64 kernel, with the bounds U in [0,1], V in [0,1]."""
    p = inputs.layered_1024(delta)
    s, ref = run_oracle(p, 150)
    _, got = run_gpu(p, 150, "fp32_kahan")
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= 1e-5
    _, g32 = run_gpu(p, p.steps, "fp32_kahan")
    _, g64 = run_gpu(p, p.steps, "fp64")
    for a, b in zip(g32, g64):
        assert rel_err(a, b) <= 1e-5
    u, v, w = g32
    assert u.min() >= 0 and u.max() <= 1 and v.min() >= 0 and v.max() <= 1 + 1e-6


def test_hetero_8192_subsample_512():
    """The 8192 x 8192 tissue at 512 x 512 (same grid-independent field),
    5000 steps (the bench's step count) against the oracle."""
    p = inputs.hetero_8192(nx=512)
    s, ref = run_oracle(p, 5000)
    _, got = run_gpu(p, 5000, "fp32_kahan", steps_per_pass=3)
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= 1e-5


def test_read_into_caller_host_arrays():
    """gg_read into a caller's host array (pageable or pinned, FP32 or FP64)
    gives the same values as a fresh read."""
    import torch
    p = inputs.plain_128(100, 70, steps=30)
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        sim.step(30)
        for f in ("u", "v", "w", "comp_v"):
            ref32, ref64 = sim.read(f, fp64=False), sim.read(f)
            a32 = np.empty((70, 100), dtype=np.float32)
            assert sim.read(f, out=a32) is a32 and np.array_equal(a32, ref32)
            pinned = torch.empty((70, 100), dtype=torch.float64).pin_memory().numpy()
            sim.read(f, out=pinned)
            assert np.array_equal(pinned, ref64)
