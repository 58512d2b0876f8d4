"""Ensembles (gg_batch_*): one persistent cooperative graph-captured launch
advances many uneven grids.  Every tile runs the same per-cell arithmetic as
the single-grid step, so each instance must match its own gg_sim run bit for
bit, and sampled instances must match the FP64 oracle within 1e-5."""
import numpy as np
import pytest

import oracle
from test_gpu_fullsize import window_oracle
from paper_2006_01748_gb300 import build, gg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()
    gg.lib()


def rel_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def scaled_ensemble(n, scale, steps):
    specs = inputs.ensemble_specs(n)
    return [inputs.ensemble_instance(k, specs[k], steps=steps, scale=scale) for k in range(n)]


@pytest.mark.parametrize("mode", ["persistent", "passes", "passes2"])
@pytest.mark.parametrize("spp", [1, 2, 3, 4])
def test_batch_matches_single_simulations_bitwise(spp, mode):
    probs = scaled_ensemble(12, 8, 37)
    with gg.GGBatch(probs, steps_per_pass=spp) as b:
        b.set_plan(mode, spp, chunk=40)
        assert b.steps_per_pass == spp
        b.step(20)
        b.step(17)
        info = b.launch_info()
        assert info["mode"] == mode and info["T"] == spp
        for k, p in enumerate(probs):
            with gg.GGSim.from_problem(p, precision="fp32_kahan") as s:
                assert b.dt(k) == s.dt
                s.step(37)
                for f in ("u", "v", "w", "comp_u", "comp_w"):
                    assert np.array_equal(b.read(k, f, fp64=False), s.read(f, fp64=False)), (k, f)


def test_batch_matches_oracle_on_sampled_instances():
    probs = scaled_ensemble(16, 8, 300)
    with gg.GGBatch(probs) as b:
        b.autotune(trial_steps=4)
        b.step(300)
        for k in (0, 5, 11, 15):
            p = probs[k]
            s, a = oracle.setup_for(p)
            ref = oracle.run(s, *a, p.u0, p.v0, p.w0, 300)
            for f, r in zip("uvw", ref):
                assert rel_err(b.read(k, f), r) <= 1e-5, (k, f)
            d = b.diagnostics(k)
            o = oracle.diagnostics(*ref, s.dx, s.dy)
            assert np.allclose(d["mass"], o["mass"], rtol=1e-5)


def test_autotune_restores_the_state():
    probs = scaled_ensemble(6, 4, 10)
    with gg.GGBatch(probs) as b:
        before = [b.read(k, "v") for k in range(6)]
        chosen = b.autotune(trial_steps=4)
        assert chosen["T"] in (1, 2, 3, 4) and chosen["bx"] == 32 - 2 * chosen["T"] and chosen["by"] > 0
        assert chosen["mode"] in ("persistent", "passes", "passes2")
        for k in range(6):
            assert np.array_equal(b.read(k, "v"), before[k])


def test_long_step_in_passes_mode_is_launched_directly():
    """More than 4096 passes in one step are not captured into one graph;
    they run as direct launches and give the same bits."""
    probs = scaled_ensemble(3, 16, 10)
    with gg.GGBatch(probs, steps_per_pass=1) as a, gg.GGBatch(probs, steps_per_pass=1) as c:
        a.set_plan("passes", 1, chunk=32)
        a.step(4100)
        assert a.launch_info()["graph"] is False
        c.set_plan("persistent", 1, chunk=32)
        c.step(4100)
        for k in range(3):
            assert np.array_equal(a.read(k, "v", fp64=False), c.read(k, "v", fp64=False))


def test_barrier_wait_gives_up_and_reports_timeout():
    """A barrier that expects one CTA more than the launch has can never
    open: every wait must give up after its (short) limit, the call must
    report GG_ERR_TIMEOUT, and the batch must run normally afterwards."""
    probs = scaled_ensemble(4, 8, 10)
    with gg.GGBatch(probs, steps_per_pass=1) as b:
        b.set_barrier_timeout(0.05, extra_arrivals=1)
        b.step(3)                                   # passes separated by barriers
        assert b.read_status(0) == gg.GG_ERR_TIMEOUT
        b.set_barrier_timeout(2.0, extra_arrivals=0)
        b.step(3)
        assert b.read_status(0) == gg.GG_OK


def test_full_ensemble_256_instances():
    """The 256-instance ensemble (grids from {128,...,1024}^2, delta ~
    U[0.5,20], D ~ logU[1e-5,1e-3]), 5000 steps in one graph-captured
    persistent launch, against single-grid runs of sampled instances."""
    specs = inputs.ensemble_specs(256)
    probs = [inputs.ensemble_instance(k, specs[k]) for k in range(256)]
    with gg.GGBatch(probs) as b:
        b.autotune(trial_steps=8)
        # sampled cells of sampled instances against the oracle on windows
        # of half-width n + 2 (the light cone of n steps, as in
        # test_gpu_fullsize.py), in the tuned launch configuration
        n = 48
        b.step(n)
        rng = np.random.default_rng(4)
        for k in (0, 100, 200, 255):
            p = probs[k]
            got = [b.read(k, f) for f in "uvw"]
            scale = [max(float(np.max(np.abs(g))), 1e-300) for g in got]
            pts = [(0, 0), (p.nx - 1, p.ny - 1), (p.nx // 2, p.ny // 2), (p.nx // 2 + int(0.1 * p.nx), p.ny // 2)]
            pts += [(int(rng.integers(0, p.nx)), int(rng.integers(0, p.ny))) for _ in range(2)]
            for i, j in pts:
                ref = window_oracle(p, b.dt(k), i, j, n)
                for g, r, sc in zip(got, ref, scale):
                    assert abs(g[j, i] - r) <= 1e-5 * sc, (k, i, j)
        b.step(5000 - n)
        info = b.launch_info()
        assert info["graph"], "the 5000-step launch should run as a replayed CUDA graph"
        assert info["tiles"] >= info["ctas"] > 0
        cells = sorted(range(256), key=lambda k: probs[k].cells)
        for k in (cells[0], cells[1], cells[128], cells[-1]):
            with gg.GGSim.from_problem(probs[k], precision="fp32_kahan") as s:
                s.step(5000)
                for f in ("u", "v", "w"):
                    assert np.array_equal(b.read(k, f, fp64=False), s.read(f, fp64=False)), (k, f)
        for k in range(0, 256, 17):
            d = b.diagnostics(k)
            assert d["nonfinite"] == 0 and d["min"][0] >= 0 and d["max"][0] <= 1
