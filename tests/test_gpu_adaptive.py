"""The adaptive step Delta t_k (gg_params.adapt_every > 0): reduced from the
state on the device, read there by every step kernel, against the FP64
oracle's run with the same rule (ggo_run_adaptive).

Tolerances: FP32 + Kahan 1e-5 and FP64 1e-12 relative max-norm per field
(as the fixed-step parity tests); Delta t_k and the simulated time 1e-6
(FP32: the maxima of the rule are taken in the state's precision) and 1e-12
(FP64)."""
import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import build, gg, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp32_kahan": 1e-5, "fp64": 1e-12}
TOL_DT = {"fp32_kahan": 1e-6, "fp64": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    gg.lib()


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def oracle_adaptive(p, every, steps):
    a = oracle.coefficients(p.theta, p.lambda1, p.lambda2)
    s = oracle.Setup(p.nx, p.ny, p.delta, p.rho, p.D, p.c, 0.0, False, p.lx, p.ly)
    return oracle.run_adaptive(s, *a, oracle.lambda_max(*a), p.cfl, every, p.u0, p.v0, p.w0, steps)


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp64"])
@pytest.mark.parametrize("nx,ny,lx,ly,every", [(64, 48, 1.0, 1.0, 25), (53, 37, 1.0, 0.7, 10)])
def test_adaptive_run_matches_oracle(precision, nx, ny, lx, ly, every):
    """The growing tumour (U = 1 everywhere at first, so the tumour flux is
    closed and Delta t_k starts well above the fixed step, then shrinks as U
    falls): final fields, the last Delta t_k and the simulated time."""
    steps = 700
    p = inputs.growing_tumour(nx, ny, steps=steps, lx=lx, ly=ly)
    (U, V, W), t, dt = oracle_adaptive(p, every, steps)
    with gg.GGSim.from_problem(p, precision=precision, adapt_every=every) as sim:
        dt0 = sim.dt
        sim.step(steps)
        got = sim.state()
        assert sim.steps == steps
        assert abs(sim.dt - dt) <= TOL_DT[precision] * dt
        assert abs(sim.time - t) <= TOL_DT[precision] * t
        assert dt0 > 1.5 * sim.dt_max * p.cfl  # the rule allowed more than the fixed step at first
        assert sim.dt < 0.95 * dt0              # ... and less once the tumour flux opened
    for name, g, r in zip("uvw", got, (U, V, W)):
        assert rel_err(g, r) <= TOL[precision], name


PLANS = ([("warp", T) for T in (1, 2, 3, 4)] + [("warp2", T) for T in (1, 2, 3, 4)]
         + [("smem", T) for T in (1, 2, 4, 8)])


def test_adaptive_every_plan_is_bitwise_identical():
    """Passes never straddle a recomputation of Delta t_k, so every plan (any
    T, even one that does not divide the interval) takes the same steps with
    the same Delta t_k and gives the same bits; so does splitting the run
    over several gg_step calls."""
    p = inputs.growing_tumour(70, 45, steps=300)
    base = None
    for kind, T in PLANS:
        with gg.GGSim.from_problem(p, precision="fp32_kahan", adapt_every=12) as sim:
            sim.set_plan(kind, T, chunk=19)
            sim.step(p.steps)
            got = sim.state(fp64=False) + (np.array([sim.dt, sim.time]),)
        if base is None:
            base = got
        else:
            for g, b in zip(got, base):
                assert np.array_equal(g, b), (kind, T)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", adapt_every=12) as sim:
        for n in (7, 18, 100, 175):
            sim.step(n)
        got = sim.state(fp64=False) + (np.array([sim.dt, sim.time]),)
    for g, b in zip(got, base):
        assert np.array_equal(g, b)


def test_adaptive_step_refusals():
    """An explicit dt with the adaptive step, a negative interval and an
    adaptive ensemble are rejected; the adjoint, which holds dt fixed, is not
    available with the adaptive step."""
    p = inputs.growing_tumour(32, 32, steps=10)
    with pytest.raises(gg.GGError) as e:
        gg.GGSim.from_problem(p, precision="fp32_kahan", adapt_every=5, dt=1e-5)
    assert e.value.status == gg.GG_ERR_ARG
    with pytest.raises(gg.GGError):
        gg.GGSim.from_problem(p, precision="fp32_kahan", adapt_every=-1)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", adapt_every=5) as sim:
        with pytest.raises(gg.GGError) as e:
            sim.adjoint(10)
        assert e.value.status == gg.GG_ERR_STATE
