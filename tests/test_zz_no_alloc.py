"""gg_diagnostics_noalloc, the diagnostics entry point for callers that
cannot allocate device memory (a framework-owned memory pool that forbids
untracked allocations, or a loop that cannot afford cudaMalloc's device-wide
synchronisation).

It is called through the C ABI on fields the test already holds on the
device and must agree with gg_diagnostics on the same states, on two calls in
a row: a large grid first, then a smaller one, so the second call runs on a
scratch array that still holds the first call's records; and on fields with
a row pitch wider than the grid whose padding columns hold garbage.  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

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


def _noalloc(torch, fields, nx, ny, dx, dy, eps, pitch=None):
    out = gg.gg_diag()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    is64 = fields[0].dtype == torch.float64
    rc = gg.lib().gg_diagnostics_noalloc(*[ctypes.c_void_p(f.data_ptr()) for f in fields], 1 if is64 else 0,
                                         nx, ny, nx if pitch is None else pitch, dx, dy, eps, stream,
                                         ctypes.byref(out))
    return rc, gg.diag_dict(out)


def _check_against_sim(torch, sim, eps):
    ref = sim.diagnostics(eps=eps)
    dtype = torch.float64 if sim.precision == gg.GG_FP64_PLAIN else torch.float32
    fields = [sim.read(f, out=torch.empty(sim.ny * sim.nx, dtype=dtype, device="cuda")) for f in "uvw"]
    rc, got = _noalloc(torch, fields, sim.nx, sim.ny, 1.0 / sim.nx, 1.0 / sim.ny, eps)
    assert rc == gg.GG_OK
    for key in ("mass", "min", "max"):
        assert np.allclose(got[key], ref[key], rtol=1e-12, atol=1e-15), key
    for key in ("nonfinite", "tumour_area", "gap_area"):
        assert got[key] == pytest.approx(ref[key], rel=1e-12), key


def test_noalloc_diagnostics_match_two_calls_in_a_row(torch):
    big = inputs.plain_128(300, 700, steps=120)
    small = inputs.plain_128(64, 48, steps=80)
    small.u0, small.v0, small.w0 = inputs.random_state(64, 48, 3)
    with gg.GGSim.from_problem(big, precision="fp32_kahan") as a, \
            gg.GGSim.from_problem(small, precision="fp64") as b:
        a.step(big.steps)
        b.step(small.steps)
        _check_against_sim(torch, a, 0.02)   # first call: 608 partial records
        _check_against_sim(torch, b, 0.3)    # second call: 48 records, fp64 fields


def test_noalloc_rejects_sizes_beyond_the_limit(torch):
    out = gg.gg_diag()
    x = torch.zeros(4, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    lib = gg.lib()
    assert lib.gg_diagnostics_noalloc(p, p, p, 0, 1 << 16, 1 << 16, 1 << 16, 1.0, 1.0, 0.01, None,
                                      ctypes.byref(out)) == gg.GG_ERR_ARG
    assert lib.gg_diagnostics_noalloc(p, p, p, 0, 4, 1, 3, 1.0, 1.0, 0.01, None, ctypes.byref(out)) == gg.GG_ERR_ARG
    assert lib.gg_diagnostics_noalloc(None, p, p, 0, 2, 2, 2, 1.0, 1.0, 0.01, None, ctypes.byref(out)) == gg.GG_ERR_ARG


def test_noalloc_pitched_rows_ignore_the_padding(torch):
    """Row j starts at element j * pitch; the pitch - nx padding columns hold
    values (NaN, huge, negative) that would change every diagnostic if they
    were read."""
    p = inputs.plain_128(50, 37, steps=60)
    with gg.GGSim.from_problem(p, precision="fp32_kahan") as sim:
        sim.step(p.steps)
        ref = sim.diagnostics(eps=0.05)
        pitch = 64
        junk = torch.tensor([float("nan"), 1e30, -7.0, 0.0], device="cuda")
        fields = []
        for f in "uvw":
            dense = sim.read(f, out=torch.empty(sim.ny * sim.nx, dtype=torch.float32, device="cuda"))
            padded = junk.repeat(sim.ny * pitch // 4).view(sim.ny, pitch).clone()
            padded[:, :sim.nx] = dense.view(sim.ny, sim.nx)
            fields.append(padded.view(-1))
        for _ in range(2):
            rc, got = _noalloc(torch, fields, sim.nx, sim.ny, 1.0 / sim.nx, 1.0 / sim.ny, 0.05, pitch=pitch)
            assert rc == gg.GG_OK
            for key in ("mass", "min", "max"):
                assert np.allclose(got[key], ref[key], rtol=1e-12, atol=1e-15), key
            for key in ("nonfinite", "tumour_area", "gap_area"):
                assert got[key] == pytest.approx(ref[key], rel=1e-12), key
