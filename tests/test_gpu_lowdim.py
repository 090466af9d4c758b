"""1D and 2D condensates on the GPU (grids whose y or z axis has one node,
reading R20) against the FP64 oracle on the same seeded inputs: single
steps and runs in imaginary and real time, the Gaussian start, the
observables, the stop rule, symmetric splitting and the z-less norm of
imaginary time.  Tolerances as for 3D: FP64 1e-12 relative, FP32 steps
2e-6 of max|psi|."""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu

D = (0.3, 0.27, 0.24)
OMEGA = (1.0, 1.4, 2.0)
OBS = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z")
SHAPES = [(70, 1, 1), (41, 35, 1), (37, 1, 44), (36, 1, 40)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, dt, g, prec="f64", field="complex"):
    from paper_1601_04641_gb300.solver import GP
    return GP(shape, D, dt, OMEGA, g, prec, field)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_steps_match_oracle(shape, prec):
    dt, g = 0.004, 15.0
    psi0 = inputs.random_field(shape, seed=23)
    oracle.renormalize(psi0, D)
    if prec == "f32":
        psi0 = psi0.astype(np.complex64).astype(np.complex128)
    gp = make(shape, dt, g, prec)
    gp.set_psi(psi0.astype(gp.np_dtype))
    gp.step_imag(3)
    gp.step_real(4)
    got = gp.get_psi().astype(np.complex128)
    o = gp.observables()
    gp.close()
    ref = psi0.copy()
    oracle.step(ref, D, dt, OMEGA, g, False, 3)
    oracle.step(ref, D, dt, OMEGA, g, True, 4)
    r = oracle.observables(ref, D, OMEGA, g)
    tol = 1e-12 if prec == "f64" else 2e-6
    assert float(np.max(np.abs(got - ref))) <= tol * float(np.max(np.abs(ref)))
    for k in OBS:
        assert abs(o[k] - r[k]) <= (1e-12 if prec == "f64" else 1e-5) * max(abs(r[k]), 1e-300), (k, o[k], r[k])


@pytest.mark.parametrize("shape", SHAPES)
def test_gaussian_start_and_observables(shape):
    gp = make(shape, 0.01, 5.0)
    gp.init_gaussian()
    got = gp.get_psi()
    o = gp.observables()
    gp.close()
    ref = oracle.gaussian(shape, D, OMEGA)
    assert float(np.max(np.abs(got - ref))) <= 1e-12 * float(np.max(np.abs(ref)))
    r = oracle.observables(ref, D, OMEGA, 5.0)
    for k in OBS:
        if r[k] == 0.0:
            assert o[k] == 0.0, k  # the rms of an absent axis
        else:
            assert abs(o[k] - r[k]) <= 1e-12 * abs(r[k]), (k, o[k], r[k])


@pytest.mark.parametrize("shape", [(48, 40, 1), (44, 1, 36)])
def test_run_imag_until_matches_oracle(shape):
    """The stop rule on a 2D condensate (FP64 real field; with nz = 1 the z
    stage is the norm reduction alone) takes the oracle's steps."""
    dt, g = 0.2 * 0.24 ** 2, 30.0
    ref = oracle.gaussian(shape, D, OMEGA)
    steps_ref, mu_ref = oracle.run_imag_until(ref, D, dt, OMEGA, g, 1e-9, 10, 8000)
    gp = make(shape, dt, g, "f64", "real")
    gp.init_gaussian()
    steps = gp.run_imag_until(1e-9, 10, 8000)
    o = gp.observables()
    gp.close()
    assert steps == steps_ref
    assert abs(o["mu"] - mu_ref) <= 1e-12 * mu_ref
    assert abs(o["norm"] - 1.0) <= 1e-12


@pytest.mark.parametrize("field", ["real", "complex"])
def test_fp32_imaginary_time_2d(field):
    """FP32 fields of a z-less 2D grid: graph-replayed imaginary-time steps
    (sweeps, then the norm reduction as the z stage) follow the oracle."""
    shape, dt, g = (64, 56, 1), 0.1 * 0.24 ** 2, 20.0
    gp = make(shape, dt, g, "f32", field)
    gp.init_gaussian()
    gp.step_imag(40)
    got = gp.get_psi().astype(np.complex128)
    o = gp.observables()
    gp.close()
    ref = oracle.gaussian(shape, D, OMEGA)
    oracle.step(ref, D, dt, OMEGA, g, False, 40)
    assert float(np.max(np.abs(got - ref))) <= 1e-5 * float(np.max(np.abs(ref)))
    r = oracle.observables(ref, D, OMEGA, g)
    assert abs(o["mu"] - r["mu"]) <= 1e-5 * r["mu"]
    assert abs(o["norm"] - 1.0) <= 1e-6


def test_symmetric_splitting_2d():
    shape, dt, g = (40, 1, 36), 0.003, 25.0
    psi0 = inputs.random_field(shape, seed=29)
    oracle.renormalize(psi0, D)
    gp = make(shape, dt, g)
    gp.set_splitting(2)
    gp.set_psi(psi0)
    gp.step_real(12)
    got = gp.get_psi()
    gp.close()
    ref = psi0.copy()
    oracle.step_strang(ref, D, dt, OMEGA, g, 12)
    assert float(np.max(np.abs(got - ref))) <= 1e-12 * float(np.max(np.abs(ref)))


def test_grids_that_are_refused():
    from paper_1601_04641_gb300.solver import GP
    for shape in ((1, 8, 8), (2, 8, 8), (8, 2, 8), (8, 8, 2)):
        with pytest.raises(N.GPError) as e:
            GP(shape, D, 0.01, OMEGA, 1.0)
        assert e.value.status == N.GP_ERR_ARG, shape
