"""The oracle pins catch plausible mistakes: each mutation below is planted
in a copy of oracle/gg_oracle.c, compiled, and must make at least one pin of
tests/test_oracle_pins.py fail.  Runs on the CPU only."""
import os
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "gg_oracle.c")

MUTATIONS = {
    "drop a12 cross term of the x-face flux":
        ("+ AT(a12, i + 1, j) * (AT(W, i + 1, jn) - AT(W, i + 1, js))", ""),
    "wrong sign of the west flux": ("return (ge - gw) + (gn - gs);", "return (ge + gw) + (gn - gs);"),
    "dx instead of dy in the y-face flux": ("(0.5 / (dy * dy))", "(0.5 / (dx * dx))"),
    "wrong mirror ghost in y": ("js = clampi(j - 1, 0, ny - 1);", "js = clampi(j - 1, 1, ny - 1);"),
    "wrong mobility sign (Table 1)": ("e = (1.0 - 0.5 * (up + AT(U, i + 1, j)))", "e = (1.0 - 0.5 * (up - AT(U, i + 1, j)))"),
    "aggression acts on V instead of W": ("fu = u * (1.0 - u) - p->delta * u * w;", "fu = u * (1.0 - u) - p->delta * u * v;"),
    "swapped tensor entries": ("a11[k] = A[0][0];", "a11[k] = A[1][1];"),
    "adjoint: dropped delta U W term in lamW": ("nW[P] += bu * (-p->delta * u);", ""),
    "adjoint: wrong sign of a mirrored cross term": ("AT(nW, L, js) -= g * kc * AT(a12, L, fj);",
                                                     "AT(nW, L, js) += g * kc * AT(a12, L, fj);"),
    "step rule without the logistic rate": ("(c + rho + 1.0 + delta)", "(c + rho + delta)"),
    "gap area with or instead of and": ("if (U[k] < eps && V[k] < eps) gap += 1.0;", "if (U[k] < eps || V[k] < eps) gap += 1.0;"),
    "Table 1 without the south face": ("return (e + w) + (n + s);", "return (e + w) + n;"),
    "front ray: first instead of farthest tumour cell": ("if (v > v_front) kT = k;", "if (v > v_front && kT < 0) kT = k;"),
    "front ray: healthy edge searched from the centre": ("for (int k = kT + 1; k < L; ++k)\n            if (AT(U,",
                                                         "for (int k = 0; k < L; ++k)\n            if (AT(U,"),
    "front ray: west ray walks east": ("else if (d == 1) { L = i0 + 1; di = -1; h = dx; }",
                                       "else if (d == 1) { L = i0 + 1; di = 1; h = dx; }"),
    "front speed without the elapsed time": ("/ (elapsed * (1.0 - 0.0));", "/ (1.0 - 0.0);"),
    "adaptive step: dx for the north face": ("if (j + 1 < ny) S += (1.0 - 0.5 * (u + AT(U, i, j + 1))) / hy2;",
                                             "if (j + 1 < ny) S += (1.0 - 0.5 * (u + AT(U, i, j + 1))) / hx2;"),
    "adaptive step: logistic term with the wrong sign": ("- (p->no_reaction ? 0.0 : p->rho * (1.0 - v));",
                                                         "+ (p->no_reaction ? 0.0 : p->rho * (1.0 - v));"),
    "adaptive step: U bound without the acid": ("u + p->delta * w - 1.0;", "u - 1.0;"),
    "adaptive step: mobility of the own cell only": ("if (i - 1 >= 0) S += (1.0 - 0.5 * (u + AT(U, i - 1, j))) / hx2;",
                                                     "if (i - 1 >= 0) S += (1.0 - u) / hx2;"),
}

PIN_TESTS = [getattr(pins, n) for n in dir(pins) if n.startswith("test_")]


def _run_pins():
    """Names of the pins that fail (parametrised pins run with their first
    parameter set)."""
    failed = []
    for fn in PIN_TESTS:
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        try:
            if params:
                argnames, values = params[0].args[0], params[0].args[1]
                names = [a.strip() for a in argnames.split(",")]
                for v in values:
                    v = v if isinstance(v, tuple) and len(names) > 1 else (v,)
                    fn(**dict(zip(names, v)))
            else:
                fn()
        except AssertionError:
            failed.append(fn.__name__)
        except Exception as e:  # a crash of the mutant counts as caught too
            failed.append(f"{fn.__name__} ({type(e).__name__})")
    return failed


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d
    oracle.use_library(None)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, workdir):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    mutant = os.path.join(workdir, f"m{abs(hash(name))}.c")
    lib = mutant[:-2] + ".so"
    with open(mutant, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", lib, mutant, "-lm"],
                   check=True)
    oracle.use_library(lib)
    try:
        failed = _run_pins()
    finally:
        oracle.use_library(None)
    assert failed, f"no pin caught: {name}"


def test_unmutated_oracle_passes_every_pin():
    oracle.use_library(None)
    assert _run_pins() == []
