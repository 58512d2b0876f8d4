"""Front diagnostics on the GPU (gg_front_rays, gg_front_speed) against the
FP64 oracle on the same state, and the two invasion regimes of Section 2 on
a 2D layered tissue."""
import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import gg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_01748_gb300 import build
    build()
    return t


def check_same(got, ref):
    for key in ("front", "edge", "gap"):
        assert np.array_equal(got[key], ref[key]), (key, got[key], ref[key])
    for key in ("mass_v", "mass_u"):
        assert np.allclose(got[key], ref[key], rtol=1e-12, atol=1e-300), key


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan", "fp32"])
@pytest.mark.parametrize("nx,ny,steps", [(128, 128, 300), (100, 77, 500), (37, 1, 200)])
def test_front_rays_match_oracle(torch, precision, nx, ny, steps):
    p = inputs.plain_128(nx=nx, ny=ny)
    if (nx, ny) == (100, 77):
        p.ly = 0.7  # rectangular cells: the north / south rays use dy
    with gg.GGSim.from_problem(p, precision=precision) as sim:
        sim.step(steps)
        U, V = sim.read("u"), sim.read("v")  # the GPU's own values, exactly, as doubles
        centres = [(nx // 2, ny // 2), (nx // 2 - 7 if nx > 14 else 0, ny // 3), (0, 0), (nx - 1, ny - 1)]
        for i0, j0 in centres:
            for thr in ((0.5, 0.5, 0.01), (0.2, 0.9, 0.3)):
                got = sim.front_rays(i0, j0, *thr)
                ref = oracle.front_rays(U, V, p.lx / nx, p.ly / ny, i0, j0, *thr)
                check_same(got, ref)


def test_front_speed_is_the_difference_of_two_measurements(torch):
    p = inputs.plain_128()
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        sim.step(200)
        i0, j0 = p.nx // 2, p.ny // 2
        first = sim.front_rays(i0, j0)
        before, after, speed = sim.front_speed(i0, j0, 400)
        assert sim.steps == 600
        check_same(before, first)
        U, V = sim.read("u"), sim.read("v")
        check_same(after, oracle.front_rays(U, V, 1.0 / p.nx, 1.0 / p.ny, i0, j0))
        ref = oracle.front_speed(before, after, 400 * sim.dt)
        assert np.allclose(speed, ref, rtol=1e-14, atol=0)
        assert np.all(np.isfinite(speed))


def test_invalid_front_arguments(torch):
    p = inputs.plain_128(nx=32)
    with gg.GGSim.from_problem(p, precision="fp32") as sim:
        for args in ((32, 0), (0, -1), (-1, 5)):
            rc, _ = gg.gg_front_rays(sim.handle, *args, 0.5, 0.5, 0.01)
            assert rc == gg.GG_ERR_ARG
        rc, _ = gg.gg_front_rays(sim.handle, 3, 3, 0.5, 0.5, 0.0)
        assert rc == gg.GG_ERR_ARG
        rc, _ = gg.gg_front_rays(sim.handle, 3, 3, float("nan"), 0.5, 0.01)
        assert rc == gg.GG_ERR_ARG
        rc, *_ = gg.gg_front_speed(sim.handle, 3, 3, 0, 0.5, 0.5, 0.01)
        assert rc == gg.GG_ERR_ARG
        assert sim.steps == 0


@pytest.mark.parametrize("delta,separated", [(12.5, True), (0.5, False)])
def test_invasion_regimes_on_a_layered_tissue(torch, delta, separated):
    """Section 2 on the layered 2D tissue at 256^2 up to t = 6 (about 1.9e6
    steps, beyond the oracle's reach at this size): for d > 1 the acid
    clears the healthy tissue ahead of the tumour, so along the rays a
    hypocellular zone separates the tumour front from the healthy edge;
    for d < 1 healthy cells stay at the front (coexistence)."""
    p = inputs.layered_1024(delta, nx=256)
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        n = int(6.0 / sim.dt)
        sim.step(n)
        f = sim.front_rays(p.nx // 2, p.ny // 2)
        d = sim.diagnostics()
    sep = f["edge"] - f["front"]
    assert np.all(f["front"] > 0.05)  # the tumour has grown from r = 0.05
    assert d["nonfinite"] == 0
    if separated:
        assert np.sum(sep >= 0.03) >= 3, sep
    else:
        assert np.all(sep == 0), sep
