"""The oracle built with OpenMP (the kick's sites and the sweeps' lines
shared out over host threads; the benchmark's all-core CPU baseline) gives
the serial build's results bit for bit: each site and line is computed by
the same code, and every sum stays serial."""
import os

import numpy as np

import oracle
from paper_1601_04641_gb300 import inputs


def test_openmp_build_equals_serial_build():
    shape, d, omega, g = (23, 19, 17), (0.3, 0.27, 0.25), (1.0, 1.3, 1.7), 15.0
    psi0 = inputs.random_field(shape, seed=31)
    oracle.renormalize(psi0, d)
    runs = {}
    for name, path in (("serial", oracle.build()), ("openmp", oracle.build_openmp())):
        with oracle.use_library(path):
            a = psi0.copy()
            oracle.step(a, d, 0.01, omega, g, False, 4)
            oracle.step(a, d, 0.004, omega, g, True, 3)
            oracle.step_strang(a, d, 0.004, omega, g, 2)
            runs[name] = (a, oracle.observables(a, d, omega, g))
    assert np.array_equal(runs["serial"][0], runs["openmp"][0])
    assert runs["serial"][1] == runs["openmp"][1]
    assert os.path.exists(oracle.build_openmp())
