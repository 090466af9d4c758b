"""Axially symmetric condensates on the GPU (gp_axial_*) against the axial
FP64 oracle (reading R21) on the same seeded inputs (GPU only): the Gaussian
start, the observables, imaginary-time steps on real and complex fields, real
time, the stop rule, junk in the ghost and boundary nodes; FP64 to 1e-12 and
FP32 to its rounding bound."""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build

pytestmark = pytest.mark.gpu

OBS = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z")
GAMMA, LAM = 1.2, 1.9


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, drho, dz, dt, g, prec="f64", field="complex"):
    from paper_1601_04641_gb300.solver import AxialGP
    return AxialGP(shape[0], shape[1], drho, dz, dt, GAMMA, LAM, g, prec, field)


def field_of(shape, seed, complex_=True):
    rng = np.random.default_rng(seed)
    nx, nz = shape
    r = (np.arange(nx) - 0.5)[:, None] / nx
    z = np.linspace(-1, 1, nz)[None, :]
    amp = np.exp(-3 * r * r - 2 * z * z) * (1 + 0.2 * rng.standard_normal(shape))
    psi = amp * (np.exp(1j * rng.uniform(-np.pi, np.pi, shape)) if complex_ else 1.0)
    psi = np.array(psi, dtype=np.complex128)
    psi[0, :] = psi[-1, :] = 0
    psi[:, 0] = psi[:, -1] = 0
    return psi


def test_axial_gaussian_and_observables_match_oracle():
    shape, drho, dz = (37, 61), 0.2, 0.15
    gp = make(shape, drho, dz, 0.005, 30.0)
    gp.init_gaussian()
    got = gp.get_psi()
    o = gp.observables()
    gp.close()
    ref = oracle.axial_gaussian(*shape, drho, dz, GAMMA, LAM)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    r = oracle.axial_observables(ref, drho, dz, GAMMA, LAM, 30.0)
    for k in OBS:
        assert abs(o[k] - r[k]) <= 1e-12 * abs(r[k]), (k, o[k], r[k])


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
@pytest.mark.parametrize("shape", [(33, 48), (20, 101)])
def test_axial_observables_of_a_random_field(prec, tol, shape):
    drho, dz, g = 0.25, 0.2, 12.0
    psi = field_of(shape, 3)
    gp = make(shape, drho, dz, 0.01, g, prec)
    gp.set_psi(psi.astype(np.complex64 if prec == "f32" else np.complex128))
    o = gp.observables()
    gp.close()
    src = psi.astype(np.complex64).astype(np.complex128) if prec == "f32" else psi
    r = oracle.axial_observables(src, drho, dz, GAMMA, LAM, g)
    for k in OBS:
        assert abs(o[k] - r[k]) <= tol * abs(r[k]), (k, o[k], r[k])


@pytest.mark.parametrize("field", ["real", "complex"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_axial_imaginary_time_steps_match_oracle(field, prec):
    shape, drho, dz, dt, g, steps = (31, 52), 0.22, 0.18, 0.004, 20.0, 12
    psi = field_of(shape, 7, complex_=(field == "complex"))
    if field == "real":
        psi = np.abs(psi).astype(np.complex128)
    gp = make(shape, drho, dz, dt, g, prec, field)
    dtype = {("f64", "real"): np.float64, ("f64", "complex"): np.complex128,
             ("f32", "real"): np.float32, ("f32", "complex"): np.complex64}[(prec, field)]
    start = psi.real.astype(dtype) if field == "real" else psi.astype(dtype)
    gp.set_psi(start)
    gp.step_imag(steps)
    got = gp.get_psi().astype(np.complex128)
    gp.close()
    ref = np.ascontiguousarray(start.astype(np.complex128))
    oracle.axial_step(ref, drho, dz, dt, GAMMA, LAM, g, False, steps)
    tol = 1e-12 if prec == "f64" else 2e-6 * steps
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_axial_real_time_matches_oracle(prec):
    shape, drho, dz, dt, g, steps = (29, 64), 0.25, 0.2, 0.002, 15.0, 20
    psi = field_of(shape, 11)
    gp = make(shape, drho, dz, dt, g, prec)
    start = psi.astype(np.complex64 if prec == "f32" else np.complex128)
    gp.set_psi(start)
    gp.step_real(steps)
    got = gp.get_psi().astype(np.complex128)
    o = gp.observables()
    gp.close()
    ref = np.ascontiguousarray(start.astype(np.complex128))
    n0 = oracle.axial_observables(ref, drho, dz, GAMMA, LAM, g)["norm"]
    oracle.axial_step(ref, drho, dz, dt, GAMMA, LAM, g, True, steps)
    tol = 1e-12 if prec == "f64" else 2e-6 * steps
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    # the cylindrical norm is conserved
    assert abs(o["norm"] - n0) <= (1e-12 if prec == "f64" else 1e-5) * n0


def test_axial_run_imag_until_matches_oracle():
    shape, drho, dz, dt, g = (33, 56), 0.25, 0.22, 0.01, 25.0
    gp = make(shape, drho, dz, dt, g, "f64", "real")
    gp.init_gaussian()
    steps = gp.run_imag_until(1e-9, 10, 20000)
    mu = gp.observables()["mu"]
    gp.close()
    ref = oracle.axial_gaussian(*shape, drho, dz, GAMMA, LAM)
    n_ref, mu_ref = oracle.axial_run_imag_until(ref, drho, dz, dt, GAMMA, LAM, g, 1e-9)
    assert steps == n_ref
    assert abs(mu - mu_ref) <= 1e-12 * mu_ref


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_axial_ignores_junk_in_ghost_and_boundary(prec):
    shape, drho, dz, dt, g = (25, 40), 0.3, 0.25, 0.005, 10.0
    psi = field_of(shape, 5)
    junk = psi.copy()
    junk[0, :] = 3.0
    junk[-1, :] = -2.0
    junk[:, 0] = 1.5
    junk[:, -1] = -4.0
    dtype = np.complex64 if prec == "f32" else np.complex128
    gp = make(shape, drho, dz, dt, g, prec)
    gp.set_psi(junk.astype(dtype))
    gp.step_real(1)
    got = gp.get_psi().astype(np.complex128)
    gp.close()
    ref = np.ascontiguousarray(psi.astype(dtype).astype(np.complex128))
    oracle.axial_step(ref, drho, dz, dt, GAMMA, LAM, g, True, 1)
    assert np.all(got[0, :] == 0) and np.all(got[-1, :] == 0)
    assert np.all(got[:, 0] == 0) and np.all(got[:, -1] == 0)
    tol = 1e-12 if prec == "f64" else 2e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_axial_argument_checks():
    from paper_1601_04641_gb300.solver import AxialGP
    for args in ((2, 10, 0.1, 0.1, 0.01, 1, 1, 1), (10, 10, -0.1, 0.1, 0.01, 1, 1, 1),
                 (10, 10, 0.1, 0.1, 0.01, 0.0, 1, 1)):
        with pytest.raises(N.GPError) as e:
            AxialGP(*args)
        assert e.value.status == N.GP_ERR_ARG
    gp = AxialGP(10, 12, 0.2, 0.2, 0.01, 1.0, 1.0, 1.0, "f64", "real")
    with pytest.raises(N.GPError) as e:
        gp.step_real(1)
    assert e.value.status == N.GP_ERR_STATE
    gp.close()
