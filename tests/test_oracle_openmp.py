"""The multi-core build of the oracle (the OpenMP CPU baseline of bench.py)
computes the same bits as the one-core build.  Kept apart from the pins: the
planted-mistake tests run every pin against a mutant library."""
import numpy as np
import pytest

import oracle
from paper_2006_01748_gb300 import inputs


def test_openmp_build_computes_the_same_bits():
    """The multi-core CPU baseline runs the same source with the step's row
    loop spread over the host cores; every cell's arithmetic is unchanged."""
    lib = oracle.build_openmp()
    if lib is None:
        pytest.skip("the compiler has no OpenMP")
    p = inputs.plain_128(96, 70, steps=5)
    s, a = oracle.setup_for(p)
    ref = oracle.run(s, *a, p.u0, p.v0, p.w0, 5)
    oracle.use_library(lib)
    try:
        got = oracle.run(s, *a, p.u0, p.v0, p.w0, 5)
    finally:
        oracle.use_library(None)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
