"""Density output: the integrated 1D densities (gp_density_profiles) and the
.npy wavefunction writer (gp_write_wavefunction).

CPU: the oracle's profiles are pinned by a brute-force triple loop, by the
norm of the C oracle's observables, and by the closed form of a separable
field; six planted mistakes (spacings of the wrong axes, a missing spacing,
sums over the wrong axes, |psi| for |psi|^2, the real part only, the cell
volume for the two spacings) each fail at least one pin.  GPU: the library's profiles against the oracle's on the same fields
(FP64 and FP32, real and complex, with a pending renormalisation and with a
pending half kick), and the written files against gp_get_psi."""
import os

import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import inputs


# ---------------------------------------------------------------- oracle pins (CPU)
# Each pin takes the profile function, so that planted mistakes can be shown
# to fail at least one of them.
def pin_brute_force(profiles):
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((4, 3, 5)) + 1j * rng.standard_normal((4, 3, 5))
    d = (0.3, 0.2, 0.7)
    rx, ry, rz = profiles(psi, d)
    bx, by, bz = np.zeros(4), np.zeros(3), np.zeros(5)
    for i in range(4):
        for j in range(3):
            for k in range(5):
                a2 = psi[i, j, k].real ** 2 + psi[i, j, k].imag ** 2
                bx[i] += a2 * d[1] * d[2]
                by[j] += a2 * d[0] * d[2]
                bz[k] += a2 * d[0] * d[1]
    return all(g.shape == w.shape and np.max(np.abs(g - w)) <= 1e-14 * np.max(np.abs(w))
               for g, w in ((rx, bx), (ry, by), (rz, bz)))


def pin_norm(profiles):
    p = inputs.imag_small()
    psi = inputs.random_field(p.shape, seed=5)
    norm = oracle.observables(psi, p.d, p.omega, p.g)["norm"]
    return all(abs(r.sum() * h - norm) <= 1e-13 * norm for r, h in zip(profiles(psi, p.d), p.d))


def pin_separable(profiles):
    # psi = a_i b_j c_k: rho_x = |a|^2 (dy sum |b|^2)(dz sum |c|^2), and so on
    rng = np.random.default_rng(11)
    a, b, c = (rng.standard_normal(n) + 1j * rng.standard_normal(n) for n in (7, 6, 9))
    d = (0.11, 0.23, 0.17)
    psi = np.einsum("i,j,k->ijk", a, b, c)
    A, B, C = (np.abs(v) ** 2 for v in (a, b, c))
    want = (A * d[1] * B.sum() * d[2] * C.sum(), B * d[0] * A.sum() * d[2] * C.sum(),
            C * d[0] * A.sum() * d[1] * B.sum())
    return all(g.shape == w.shape and np.max(np.abs(g - w)) <= 1e-13 * np.max(w)
               for g, w in zip(profiles(psi, d), want))


PINS = (pin_brute_force, pin_norm, pin_separable)


def test_profiles_equal_brute_force_loops():
    assert pin_brute_force(oracle.density_profiles)


def test_profiles_integrate_to_the_oracle_norm():
    assert pin_norm(oracle.density_profiles)


def test_profiles_of_a_separable_field():
    assert pin_separable(oracle.density_profiles)


def _rho(psi):
    psi = np.asarray(psi)
    return psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2


MUTANTS = {
    # spacings of the wrong axes
    "swapped_spacing": lambda psi, d: (_rho(psi).sum(axis=(1, 2)) * d[0] * d[2], _rho(psi).sum(axis=(0, 2)) * d[1] * d[2],
                                       _rho(psi).sum(axis=(0, 1)) * d[0] * d[1]),
    # one spacing left out
    "missing_spacing": lambda psi, d: (_rho(psi).sum(axis=(1, 2)) * d[1], _rho(psi).sum(axis=(0, 2)) * d[0] * d[2],
                                       _rho(psi).sum(axis=(0, 1)) * d[0] * d[1]),
    # summed over the profile's own axis instead of the other two
    "wrong_axes": lambda psi, d: (_rho(psi).sum(axis=(0, 1)) * d[1] * d[2], _rho(psi).sum(axis=(0, 2)) * d[0] * d[2],
                                  _rho(psi).sum(axis=(1, 2)) * d[0] * d[1]),
    # |psi| instead of |psi|^2
    "modulus_not_density": lambda psi, d: tuple(np.sqrt(_rho(psi)).sum(axis=ax) * w for ax, w in
                                                (((1, 2), d[1] * d[2]), ((0, 2), d[0] * d[2]), ((0, 1), d[0] * d[1]))),
    # real part only
    "real_part_only": lambda psi, d: tuple((np.asarray(psi).real ** 2).sum(axis=ax) * w for ax, w in
                                           (((1, 2), d[1] * d[2]), ((0, 2), d[0] * d[2]), ((0, 1), d[0] * d[1]))),
    # times the full cell volume dV instead of the two spacings
    "cell_volume": lambda psi, d: tuple(_rho(psi).sum(axis=ax) * d[0] * d[1] * d[2] for ax in ((1, 2), (0, 2), (0, 1))),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    with np.errstate(all="ignore"):
        caught = [pin.__name__ for pin in PINS if not pin(MUTANTS[name])]
    assert caught, "no pin catches " + name


# ---------------------------------------------------------------- library vs oracle (GPU)
SHAPE = (19, 14, 23)
D = (0.31, 0.27, 0.22)
OMEGA = (1.0, 1.4, 0.8)


def _gp(prec, field, dt=0.004, g=7.0):
    from paper_1601_04641_gb300 import build
    from paper_1601_04641_gb300.solver import GP
    build.build()
    return GP(SHAPE, D, dt, OMEGA, g, prec, field)


def _close(got, want, tol):
    for gv, wv in zip(got, want):
        assert np.max(np.abs(gv - wv)) <= tol * np.max(np.abs(wv))


@pytest.mark.gpu
@pytest.mark.parametrize("prec,field", [("f64", "complex"), ("f64", "real"), ("f32", "complex"), ("f32", "real")])
def test_profiles_match_oracle(prec, field):
    gp = _gp(prec, field)
    psi0 = inputs.random_field(SHAPE, seed=21, complex_=(field == "complex"))
    gp.set_psi(psi0.astype(gp.np_dtype))
    got = gp.density_profiles()
    want = oracle.density_profiles(gp.get_psi().astype(np.complex128), D)
    _close(got, want, 1e-13)
    # pending renormalisation: profiles of the scaled field, which get_psi returns
    gp.step_imag(3)
    got = gp.density_profiles()
    want = oracle.density_profiles(gp.get_psi().astype(np.complex128), D)
    _close(got, want, 1e-13 if prec == "f64" else 1e-6)
    n = gp.observables()["norm"]
    assert abs(got[0].sum() * D[0] - n) <= (1e-12 if prec == "f64" else 1e-6) * n
    gp.close()


@pytest.mark.gpu
def test_profiles_ignore_a_pending_half_kick():
    gp = _gp("f64", "complex")
    gp.set_psi(inputs.random_field(SHAPE, seed=8))
    gp.set_splitting(2)
    gp.step_real(4)  # leaves the trailing half kick pending
    got = gp.density_profiles()
    want = oracle.density_profiles(gp.get_psi(), D)  # get_psi settles it (a phase)
    _close(got, want, 1e-12)
    gp.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,field", [("f64", "complex"), ("f32", "complex"), ("f32", "real"), ("f64", "real")])
def test_write_wavefunction(tmp_path, prec, field):
    gp = _gp(prec, field)
    gp.init_gaussian()  # leaves a renormalisation factor pending
    path = os.path.join(tmp_path, "psi.npy")
    gp.write_wavefunction(path)
    psi = gp.get_psi()
    got = np.load(path)
    assert got.dtype == psi.dtype and got.shape == SHAPE
    assert np.array_equal(got, psi)
    gp.write_wavefunction(path, density=True)
    rho = np.load(path)
    real_t = np.float32 if prec == "f32" else np.float64
    want = (psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2).astype(real_t)
    assert rho.dtype == real_t and np.array_equal(rho, want)
    gp.close()


@pytest.mark.gpu
def test_write_wavefunction_errors(tmp_path):
    from paper_1601_04641_gb300 import _native as N
    gp = _gp("f32", "complex")
    gp.init_gaussian()
    bad = os.path.join(tmp_path, "no_such_dir", "psi.npy")
    with pytest.raises(N.GPError) as e:
        gp.write_wavefunction(bad)
    assert e.value.status == N.GP_ERR_IO
    assert gp.lib.gp_write_wavefunction(gp.h, b"x.npy", 5) == N.GP_ERR_ARG
    gp.close()
