"""Parity of the CUDA discrete adjoint (gg_adjoint through the C ABI) with the
FP64 oracle's adjoint, checkpoint invariance, finite differences of the GPU
FP64 forward at small and full size, and the torch.autograd wrapper.

Tolerance: relative max-norm <= 1e-5 per gradient field (FP32 + Kahan adjoint
against the FP64 oracle), <= 1e-5 relative for the four rate gradients."""
import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import build, gg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    gg.lib()
    return torch


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def small_problem(nx, ny, seed=5, steps=120):
    p = inputs.plain_128(nx, ny, steps=steps, seed=seed)
    p.D = 2e-3
    p.u0, p.v0, p.w0 = inputs.random_state(nx, ny, seed + 1)
    return p


def oracle_adjoint(p, steps, Vstar, dLdU, dLdW):
    s, a = oracle.setup_for(p)
    U, V, W = oracle.run(s, *a, p.u0, p.v0, p.w0, steps)
    gV = oracle.misfit_grad(V, Vstar, s.dx, s.dy)
    lam0, ga, gs = oracle.adjoint(s, *a, p.u0, p.v0, p.w0, steps, dLdU, gV, dLdW)
    gth, gl1, gl2 = oracle.coefficients_vjp(p.theta, p.lambda1, p.lambda2, *ga)
    return dict(theta=gth, lambda1=gl1, lambda2=gl2, u0=lam0[0], v0=lam0[1], w0=lam0[2], scalars=gs, V=V, s=s)


def gpu_adjoint(torch, p, steps, dLdU, dLdV, dLdW, precision="fp32_kahan", checkpoint_every=0):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().view(-1)
    with gg.GGSim.from_problem(p, precision=precision) as sim:
        r = sim.adjoint(steps, t(dLdU), t(dLdV), t(dLdW), checkpoint_every=checkpoint_every)
        r = {k: (v.cpu().numpy().astype(np.float64) if k != "scalars" else v) for k, v in r.items()}
        r["steps"] = sim.steps
    return r


@pytest.mark.parametrize("nx,ny,steps", [(40, 33, 120), (64, 64, 200), (256, 256, 100), (5, 1, 50), (1, 6, 50)])
def test_adjoint_matches_oracle(torch, nx, ny, steps):
    p = small_problem(nx, ny, steps=steps)
    Vstar = inputs.random_state(nx, ny, 99)[1]
    dLdU = 1e-3 * inputs.white_noise(nx, ny, 7, -1, 1)
    dLdW = 1e-3 * inputs.white_noise(nx, ny, 8, -1, 1)
    ref = oracle_adjoint(p, steps, Vstar, dLdU, dLdW)
    gV = oracle.misfit_grad(ref["V"], Vstar, ref["s"].dx, ref["s"].dy)
    got = gpu_adjoint(torch, p, steps, dLdU, gV, dLdW)
    assert got["steps"] == steps
    for k in ("theta", "lambda1", "lambda2", "u0", "v0", "w0"):
        assert rel_err(got[k], ref[k]) <= 1e-5, k
    for q in range(4):
        assert abs(got["scalars"][q] - ref["scalars"][q]) <= 1e-5 * max(abs(ref["scalars"][q]), 1e-12), q


def test_adjoint_matches_oracle_on_rectangular_cells(torch):
    """dx != dy (lx = 1, ly = 0.7 on 48 x 40 cells): every x / y factor of the
    transpose and of the tensor gradients is exercised separately."""
    nx, ny, steps = 48, 40, 150
    p = small_problem(nx, ny, steps=steps)
    p.lx, p.ly = 1.0, 0.7
    Vstar = inputs.random_state(nx, ny, 98)[1]
    dLdU = 1e-3 * inputs.white_noise(nx, ny, 17, -1, 1)
    dLdW = 1e-3 * inputs.white_noise(nx, ny, 18, -1, 1)
    ref = oracle_adjoint(p, steps, Vstar, dLdU, dLdW)
    assert ref["s"].dx != ref["s"].dy
    gV = oracle.misfit_grad(ref["V"], Vstar, ref["s"].dx, ref["s"].dy)
    got = gpu_adjoint(torch, p, steps, dLdU, gV, dLdW)
    for k in ("theta", "lambda1", "lambda2", "u0", "v0", "w0"):
        assert rel_err(got[k], ref[k]) <= 1e-5, k
    for q in range(4):
        assert abs(got["scalars"][q] - ref["scalars"][q]) <= 1e-5 * max(abs(ref["scalars"][q]), 1e-12), q


def test_adjoint_without_kahan_and_without_reactions(torch):
    nx, ny, steps = 48, 40, 100
    p = small_problem(nx, ny, steps=steps)
    Vstar = inputs.random_state(nx, ny, 98)[1]
    z = np.zeros((ny, nx))
    s, a = oracle.setup_for(p, no_reaction=True)
    U, V, W = oracle.run(s, *a, p.u0, p.v0, p.w0, steps)
    gV = oracle.misfit_grad(V, Vstar, s.dx, s.dy)
    lam0, ga, gs = oracle.adjoint(s, *a, p.u0, p.v0, p.w0, steps, z, gV, z)
    gth = oracle.coefficients_vjp(p.theta, p.lambda1, p.lambda2, *ga)[0]
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda().view(-1)
    for precision, tol in (("fp32_kahan", 1e-5), ("fp32", 1e-4)):
        with gg.GGSim.from_problem(p, precision=precision, no_reaction=True) as sim:
            r = sim.adjoint(steps, None, t(gV), None)
        assert rel_err(r["theta"].cpu().numpy(), gth) <= tol
        assert rel_err(r["v0"].cpu().numpy(), lam0[1]) <= tol
        assert abs(r["scalars"][2] - gs[2]) <= tol * abs(gs[2])
        assert r["scalars"][0] == 0 and r["scalars"][1] == 0 and r["scalars"][3] == 0


def test_checkpoint_spacing_does_not_change_the_result(torch):
    """The stored states (every other step) are bitwise those of the forward
    pass for every checkpoint spacing K; the two-step reverse pass rebuilds
    the state between two stored ones without its Kahan term, which changes
    it by its last rounding at most, and which states are rebuilt depends on
    K, as does the grouping of the per-cell gradient sums.  So the gradient
    fields agree across K to 3e-6 (measured: 1.5e-6) and the rate gradients to
    2e-5: on this rough random state with unit adjoint sources the D gradient
    is a sum over the grid that cancels to a small part of its terms (measured
    spread across K: 8e-6)."""
    nx, ny, steps = 70, 50, 97
    p = small_problem(nx, ny, steps=steps)
    dU = inputs.white_noise(nx, ny, 1, -1, 1)
    dV = inputs.white_noise(nx, ny, 2, -1, 1)
    dW = inputs.white_noise(nx, ny, 3, -1, 1)
    base = gpu_adjoint(torch, p, steps, dU, dV, dW, checkpoint_every=0)
    for K in (1, 2, 7, 96, 97, 500):
        r = gpu_adjoint(torch, p, steps, dU, dV, dW, checkpoint_every=K)
        for k in ("theta", "lambda1", "lambda2", "u0", "v0", "w0"):
            assert rel_err(r[k], base[k]) <= 3e-6, (K, k)
        assert np.allclose(r["scalars"], base["scalars"], rtol=2e-5, atol=0), K


@pytest.mark.parametrize("K", [0, 7])
def test_forward_plan_does_not_change_the_adjoint(torch, K):
    """The adjoint's forward and recompute passes run the simulation's plan
    (its kernel kind, steps per pass and chunk height), writing the even
    states from the intermediate levels of each pass: with T = 4 level 2
    (passes from even steps) or levels 1 and 3 (odd), with T = 3 level 2 or
    level 1, with T = 2 level 1 from odd steps.  Every plan gives the forward's
    bits, so the stored states and the whole adjoint are bitwise the same
    for every plan; 41 steps and K = 7 give passes from odd steps."""
    nx, ny, steps = 130, 77, 41
    p = small_problem(nx, ny, steps=steps)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().view(-1)
    dU = t(inputs.white_noise(nx, ny, 11, -1, 1))
    dV = t(inputs.white_noise(nx, ny, 12, -1, 1))
    dW = t(inputs.white_noise(nx, ny, 13, -1, 1))
    base = None
    for kind, T in [("warp", 1), ("warp2", 2), ("warp2", 3), ("warp2", 4), ("warp", 3), ("warp", 4)]:
        with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
            sim.set_plan(kind, T, chunk=24)
            r = sim.adjoint(steps, dU, dV, dW, checkpoint_every=K)
            r = {k: (v.cpu().numpy() if k != "scalars" else np.asarray(v)) for k, v in r.items()}
            r["state"] = np.stack(sim.state(fp64=False))
        if base is None:
            base = r
            continue
        for k in base:
            assert np.array_equal(r[k], base[k]), (kind, T, k)


def test_workspace_reuse_and_release(torch):
    """A second call on the same simulation reuses the workspace (kept
    states included) and a call after gg_adjoint_release allocates it again;
    from the same state both give the first call's bits."""
    nx, ny, steps = 70, 50, 97
    p = small_problem(nx, ny, steps=steps)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().view(-1)
    dV = t(inputs.white_noise(nx, ny, 2, -1, 1))
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        names = ("u", "v", "w", "comp_u", "comp_v", "comp_w")
        x0 = [sim.read(f, fp64=False) for f in names]

        def run():
            for f, x in zip(names, x0):
                sim.write(f, x)
            r = sim.adjoint(steps, None, dV, None)
            return {k: (v.cpu().numpy() if k != "scalars" else v) for k, v in r.items()}

        first = run()
        again = run()
        sim.release_adjoint()
        sim.release_adjoint()  # a no-op without a workspace
        after = run()
        for r in (again, after):
            for k in first:
                assert np.array_equal(r[k], first[k]), k


def _fp64_loss(p, dt, steps, Vstar, **over):
    q = inputs.Problem(**{**p.__dict__, **over})
    with gg.GGSim.from_problem(q, precision="fp64", dt=dt) as sim:
        sim.step(steps)
        V = sim.read("v")
    return 0.5 / (p.nx * p.ny) * float(np.sum((V - Vstar) ** 2))


def test_adjoint_matches_finite_differences_of_gpu_fp64_forward(torch):
    nx = ny = 64
    steps = 200
    p = small_problem(nx, ny, steps=steps, seed=21)
    Vstar = inputs.random_state(nx, ny, 22)[1]
    with gg.GGSim.from_problem(p, precision="fp64") as sim:
        dt = sim.dt
        sim.step(steps)
        V = sim.read("v")
    gV = (V - Vstar) / (nx * ny)
    z = np.zeros((ny, nx))
    with gg.GGSim.from_problem(p, precision="fp32_kahan", dt=dt) as sim:
        t = torch.from_numpy(gV.astype(np.float32)).cuda().view(-1)
        r = sim.adjoint(steps, None, t, None)
    rng = np.random.default_rng(3)
    for name in ("theta", "lambda1", "lambda2"):
        g = r[name].cpu().numpy()
        scale = np.max(np.abs(g))
        for k in rng.choice(nx * ny, size=6, replace=False):
            eps = 1e-3
            xp, xm = getattr(p, name).copy(), getattr(p, name).copy()
            xp.flat[k] += eps
            xm.flat[k] -= eps
            fd = (_fp64_loss(p, dt, steps, Vstar, **{name: xp}) - _fp64_loss(p, dt, steps, Vstar, **{name: xm})) / (2 * eps)
            assert abs(fd - g.flat[k]) <= 2e-4 * scale, (name, k, fd, g.flat[k])
    for q, name in enumerate(("delta", "rho", "D", "c")):
        h = 1e-4 * max(1.0, abs(getattr(p, name)))
        fd = (_fp64_loss(p, dt, steps, Vstar, **{name: getattr(p, name) + h})
              - _fp64_loss(p, dt, steps, Vstar, **{name: getattr(p, name) - h})) / (2 * h)
        assert abs(fd - r["scalars"][q]) <= 1e-4 * abs(fd) + 1e-12, name


def _fp64_loss_vw(p, dt, steps, Vstar, **over):
    q = inputs.Problem(**{**p.__dict__, **over})
    with gg.GGSim.from_problem(q, precision="fp64", dt=dt) as sim:
        sim.step(steps)
        V, W = sim.read("v"), sim.read("w")
    return (0.5 * float(np.sum((V - Vstar) ** 2)) + float(np.sum(W))) / p.cells


def _twin_misfit_seed(p, tgt, dt, steps):
    """V* of the twin run (tensor from seed + 1) and dL/dV^N of the v-misfit,
    both from FP64 forward runs with the fixed dt (so the seed given to the
    adjoint is the one the finite differences of the FP64 loss see)."""
    with gg.GGSim.from_problem(tgt, precision="fp64", dt=dt) as sim:
        sim.step(steps)
        Vstar = sim.read("v")
    with gg.GGSim.from_problem(p, precision="fp64", dt=dt) as sim:
        sim.step(steps)
        V = sim.read("v")
    return Vstar, (V - Vstar) / p.cells


def test_adjoint_2048_rate_gradients_against_finite_differences(torch):
    """Full-size adjoint workload (2048 x 2048, 10^4 steps, sqrt(N)
    checkpointing).  Over its short physical time (t = 10^4 dt, about 5e-4)
    the v-misfit alone has gradients near 1e-20, so the checked loss adds the
    acid mass: L = dx dy [ sum (V - V*)^2 / 2 + sum W ].  Its seeds dL/dX^N are
    taken from the FP64 forward (the misfit V - V* is small enough that the
    FP32 forward's rounding would change it), and the FP32 adjoint's rate
    gradients are compared with central differences of the GPU FP64 forward
    (dt held fixed).

    The loss is strongly curved in D over this short time (the central
    difference with h = 1e-3 D is off by 1.5e-3, with h = 3e-2 D it has the
    wrong sign), so D is differenced with h = 1e-4 D, where the difference
    has converged to about 1e-5; the other rates with h = 1e-3 of their value.
    Measured: c 8e-9, rho 5e-7, D 7e-6; delta within the rounding floor of the
    central difference.  Every gradient is held to 3e-5 plus that floor."""
    p = inputs.adjoint_2048()
    tgt = inputs.adjoint_2048(target=True)
    with gg.GGSim.from_problem(p, precision="fp64") as sim:
        dt = sim.dt
    Vstar, gV = _twin_misfit_seed(p, tgt, dt, p.steps)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", dt=dt) as sim:
        tv = torch.from_numpy(gV.astype(np.float32)).cuda().view(-1)
        tw = torch.full((p.cells,), 1.0 / p.cells, dtype=torch.float32, device="cuda")
        r = sim.adjoint(p.steps, None, tv, tw, outputs=("theta",))
        assert sim.steps == p.steps
    assert np.all(np.isfinite(r["theta"].cpu().numpy()))
    L0 = _fp64_loss_vw(p, dt, p.steps, Vstar)
    bad = []
    for q, name in ((3, "c"), (2, "D"), (1, "rho"), (0, "delta")):
        h = (1e-4 if name == "D" else 1e-3) * getattr(p, name)
        fd = (_fp64_loss_vw(p, dt, p.steps, Vstar, **{name: getattr(p, name) + h})
              - _fp64_loss_vw(p, dt, p.steps, Vstar, **{name: getattr(p, name) - h})) / (2 * h)
        noise = 1e-16 * abs(L0) / h   # rounding floor of the central difference
        if name == "c":
            assert abs(fd) > 1e3 * noise   # the acid rate carries the signal
        print(f"{name}: fd {fd:.12e} adjoint {r['scalars'][q]:.12e} rel {abs(fd - r['scalars'][q]) / abs(fd):.3e}")
        if abs(fd - r["scalars"][q]) > 3e-5 * abs(fd) + 10 * noise:
            bad.append((name, fd, r["scalars"][q], noise))
    assert not bad, bad


@pytest.mark.parametrize("loss", ["v_misfit", "v_misfit_plus_w_mass"])
def test_adjoint_10k_steps_matches_oracle(torch, loss):
    """The adjoint workload's rates, tensor field, twin target and step count
    (10^4 steps, sqrt(N) checkpointing) on a 128 x 128 grid, where the
    oracle's store-all FP64 adjoint fits in host memory (3.9 GB of states).
    Every output -- dL/d(theta, lambda1, lambda2), dL/d(U, V, W) at step 0
    and the four rate gradients -- is compared element by element with the
    oracle, both sides given the same seeds (the oracle's dL/dX^N).

    v_misfit is the configured loss L = dx dy sum (V^N - V*)^2 / 2 (measured:
    every output within 1.4e-7).  v_misfit_plus_w_mass adds dx dy sum W^N, a
    uniform source for lambda_W: the tensor gradients then come from
    differences of nearly equal lambda_W values, which keep the FP32 rounding
    of the increments c lambda_W dt (about 1e-3 lambda_W per step) (measured:
    2.5e-6 for theta, 1.7e-6 for c).  Every output is held to 1e-5."""
    nx, steps = 128, 10000
    p = inputs.adjoint_2048(nx=nx, steps=steps)
    tg = inputs.adjoint_2048(nx=nx, steps=steps, target=True)
    s, a = oracle.setup_for(p)
    st, at = oracle.setup_for(tg, dt=s.dt)
    Vstar = oracle.run(st, *at, tg.u0, tg.v0, tg.w0, steps)[1]
    V = oracle.run(s, *a, p.u0, p.v0, p.w0, steps)[1]
    gV = oracle.misfit_grad(V, Vstar, s.dx, s.dy)
    gW = np.full_like(V, s.dx * s.dy) if loss == "v_misfit_plus_w_mass" else np.zeros_like(V)
    z = np.zeros_like(V)
    lam0, ga, gs = oracle.adjoint(s, *a, p.u0, p.v0, p.w0, steps, z, gV, gW)
    gth, gl1, gl2 = oracle.coefficients_vjp(p.theta, p.lambda1, p.lambda2, *ga)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda().view(-1)
    with gg.GGSim.from_problem(p, precision="fp32_kahan", dt=s.dt) as sim:
        r = sim.adjoint(steps, None, t(gV), t(gW) if loss != "v_misfit" else None)
        assert sim.steps == steps
    tensor_tol = 1e-5
    for k, ref, tol in (("theta", gth, tensor_tol), ("lambda1", gl1, tensor_tol), ("lambda2", gl2, tensor_tol),
                        ("u0", lam0[0], 1e-5), ("v0", lam0[1], 1e-5), ("w0", lam0[2], 1e-5)):
        err = rel_err(r[k].cpu().numpy().astype(np.float64), ref)
        print(f"{loss} {k}: {err:.3e}")
        assert err <= tol, (k, err)
    for q in range(4):
        err = abs(r["scalars"][q] - gs[q]) / abs(gs[q])
        print(f"{loss} scalar {q}: {err:.3e}")
        assert err <= 1e-5, (q, r["scalars"][q], gs[q])


def test_autograd_function(torch):
    from paper_2006_01748_gb300.autograd import GGStepFn
    nx, ny, steps = 48, 36, 80
    p = small_problem(nx, ny, steps=steps)
    Vstar = torch.from_numpy(inputs.random_state(nx, ny, 97)[1]).cuda().float()
    th = torch.tensor(p.theta, requires_grad=True)
    l1 = torch.tensor(p.lambda1, requires_grad=True)
    l2 = torch.tensor(p.lambda2, requires_grad=True)
    sc = torch.tensor([p.delta, p.rho, p.D, p.c], dtype=torch.float64, requires_grad=True)
    u0, v0, w0 = (torch.tensor(x, requires_grad=True) for x in (p.u0, p.v0, p.w0))
    U, V, W = GGStepFn.apply(th, l1, l2, sc, u0, v0, w0, steps)
    wgt = torch.from_numpy(1e-3 * inputs.white_noise(nx, ny, 96, -1, 1)).cuda()
    loss = 0.5 / (nx * ny) * ((V.double() - Vstar.double()) ** 2).sum() + (wgt * W.double()).sum()
    loss.backward()
    s, a = oracle.setup_for(p)
    Uo, Vo, Wo = oracle.run(s, *a, p.u0, p.v0, p.w0, steps)
    gV = oracle.misfit_grad(Vo, Vstar.double().cpu().numpy(), s.dx, s.dy)
    lam0, ga, gs = oracle.adjoint(s, *a, p.u0, p.v0, p.w0, steps, np.zeros_like(Uo), gV,
                                  1e-3 * inputs.white_noise(nx, ny, 96, -1, 1))
    gth = oracle.coefficients_vjp(p.theta, p.lambda1, p.lambda2, *ga)[0]
    assert rel_err(th.grad.numpy(), gth) <= 1e-5
    assert rel_err(w0.grad.numpy(), lam0[2]) <= 1e-5
    assert np.allclose(sc.grad.numpy(), gs, rtol=1e-5, atol=1e-12)
