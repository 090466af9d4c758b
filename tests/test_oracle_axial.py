"""Pins of the axially symmetric (rho, z) oracle (reading R21) against what the
physics and the mathematics fix, independent of the oracle's own formulas,
and planted mistakes that they catch (CPU only).

- g = 0: the imaginary-time fixed point's mu tends to the continuum
  gamma + lambda/2 (2D radial oscillator plus 1D), at second order in the
  spacing; its rms radii tend to 1/sqrt(2 gamma) and 1/sqrt(2 lambda).
- Real time: the cylindrical norm sum 2 pi rho |psi|^2 drho dz is conserved
  (the radial operator is symmetric in that inner product only if its
  weights are right).
- g > 0: the virial relation 2 K - 2 P + 3 E_int = 0 of the 3D equation
  holds on the converged ground state to second order in the spacing, with
  K, P, E_int read from the observables (P from the rms radii, E_int =
  mu - E).
- With gamma = nu the axial ground state is the 3D one: mu agrees with the
  Cartesian 3D oracle's (R1-R5, pinned in test_oracle_pins.py) on grids of
  the same spacing, within both discretisations' second-order errors.
"""
import math

import numpy as np
import pytest

import oracle


def ground(nx, nz, drho, dz, gamma, lam, g, dt, tol=1e-11):
    psi = oracle.axial_gaussian(nx, nz, drho, dz, gamma, lam)
    oracle.axial_run_imag_until(psi, drho, dz, dt, gamma, lam, g, tol)
    return psi, oracle.axial_observables(psi, drho, dz, gamma, lam, g)


def box(half, d):
    """Nodes so that the outer boundary sits at about `half` from the axis
    (radial: rho_{nx-1} = (nx - 3/2) d) and the z box spans +-half."""
    return int(round(half / d + 1.5)), 2 * int(round(half / d)) + 1


def test_axial_g0_continuum_limit():
    gamma, lam = 1.3, 2.1
    errs = []
    for d in (0.2, 0.1):
        dz = 0.75 * d  # unequal spacings: each axis's operator must use its own
        nx, nz = box(6.0, d)[0], box(6.0, dz)[1]
        psi, o = ground(nx, nz, d, dz, gamma, lam, 0.0, 0.2 * dz * dz)
        errs.append(abs(o["mu"] - (gamma + lam / 2)))
        assert abs(o["rms_x"] - 1 / math.sqrt(2 * gamma)) < 2e-2
        assert abs(o["rms_z"] - 1 / math.sqrt(2 * lam)) < 2e-2
        assert o["rms_x"] == o["rms_y"]
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, (errs, ratio)
    assert errs[1] < 5e-3


def test_axial_real_time_conserves_cylindrical_norm():
    nx, nz, drho, dz = 30, 41, 0.25, 0.3
    rng = np.random.default_rng(5)
    psi = (rng.standard_normal((nx, nz)) + 1j * rng.standard_normal((nx, nz)))
    psi[0, :] = psi[-1, :] = 0
    psi[:, 0] = psi[:, -1] = 0
    psi = np.ascontiguousarray(psi)
    n0 = oracle.axial_observables(psi, drho, dz, 1.0, 1.5, 4.0)["norm"]
    oracle.axial_step(psi, drho, dz, 0.01, 1.0, 1.5, 4.0, True, 60)
    n1 = oracle.axial_observables(psi, drho, dz, 1.0, 1.5, 4.0)["norm"]
    assert abs(n1 - n0) <= 1e-12 * n0, (n0, n1)
    # the radial sweep alone, on a field with structure near the axis
    psi2 = psi.copy()
    oracle.axial_sweep(psi2, drho, dz, 0, 0.05, True)
    n2 = oracle.axial_observables(psi2, drho, dz, 1.0, 1.5, 4.0)["norm"]
    assert abs(n2 - n1) <= 1e-12 * n1


def virial_residual(o, gamma, lam):
    # P = (gamma^2 <rho^2> + lambda^2 <z^2>) / 2 with <rho^2> = 2 rms_x^2
    pot = 0.5 * (gamma ** 2 * 2 * o["rms_x"] ** 2 + lam ** 2 * o["rms_z"] ** 2)
    eint = o["mu"] - o["energy"]
    kin = o["energy"] - pot - eint
    return (2 * kin - 2 * pot + 3 * eint) / o["energy"]


def test_axial_virial_relation():
    gamma, lam, g = 1.0, 1.6, 40.0
    res = []
    for d in (0.2, 0.1):
        nx, nz = box(5.5, d)
        _, o = ground(nx, nz, d, d, gamma, lam, g, 0.2 * d * d, 1e-10)
        res.append(abs(virial_residual(o, gamma, lam)))
    assert res[1] < 2e-3, res
    assert res[0] / res[1] > 2.5, res


def test_axial_matches_3d_cartesian():
    gamma, lam, g = 1.4, 2.0, 15.0
    d = 0.3
    half = 4.2
    # 3D: nodes x_i = (i - (N-1)/2) d, Dirichlet at the outer nodes
    n = 2 * int(round(half / d)) + 1
    psi3 = oracle.gaussian((n, n, n), (d, d, d), (gamma, gamma, lam)).astype(np.complex128)
    _, mu3 = oracle.run_imag_until(psi3, (d, d, d), 0.2 * d * d, (gamma, gamma, lam), g, 1e-10)
    nx, nz = box(half, d)
    _, o = ground(nx, nz, d, d, gamma, lam, g, 0.2 * d * d, 1e-10)
    # both are second-order approximations of the same continuum mu
    assert abs(o["mu"] - mu3) <= 1e-2 * mu3, (o["mu"], mu3)


def test_axial_refuses_bad_grids():
    with pytest.raises(RuntimeError):
        oracle.axial_gaussian(2, 10, 0.1, 0.1, 1.0, 1.0)
    with pytest.raises(RuntimeError):
        oracle.axial_gaussian(10, 10, -0.1, 0.1, 1.0, 1.0)


# ---------------------------------------------------------------- planted mistakes
MUTATIONS = {
    "radial weights of a Cartesian line": (
        "                wl = (r - 0.5 * drho) / r;\n                wr = (r + 0.5 * drho) / r;",
        "                wl = 1.0;\n                wr = 1.0;"),
    "radial weights swapped": (
        "                wl = (r - 0.5 * drho) / r;\n                wr = (r + 0.5 * drho) / r;",
        "                wl = (r + 0.5 * drho) / r;\n                wr = (r - 0.5 * drho) / r;"),
    "radial nodes on the axis": ("static double axial_rho(int i, double drho) { return (i - 0.5) * drho; }",
                                 "static double axial_rho(int i, double drho) { return (i - 1.0) * drho + 1e-3 * drho; }"),
    "measure without rho": ("return 2.0 * M_PI * axial_rho(i, drho) * drho * dz; }",
                            "return 2.0 * M_PI * drho * dz; }"),
    "radial link at the node": (
        "ekin += 0.5 * 2.0 * M_PI * (r + 0.5 * drho) * dz / drho * creal(dr * conj(dr));",
        "ekin += 0.5 * 2.0 * M_PI * r * dz / drho * creal(dr * conj(dr));"),
    "z link weight without rho": (
        "ekin += 0.5 * 2.0 * M_PI * r * drho / dz * creal(dzp * conj(dzp));",
        "ekin += 0.5 * 2.0 * M_PI * drho / dz * creal(dzp * conj(dzp));"),
    "radial trap without gamma squared": (
        "double v = 0.5 * (gamma * gamma * r * r + lambda * lambda * z * z);",
        "double v = 0.5 * (gamma * r * r + lambda * lambda * z * z);"),
    "rms_x as the full <rho^2>": ("out[3] = sqrt(0.5 * r2 / enorm);", "out[3] = sqrt(r2 / enorm);"),
    "radial CN coefficient uses dz": ("const double h = axis == 0 ? drho : dz;",
                                      "const double h = dz;"),
}

AXIAL_CHECKS = [
    test_axial_g0_continuum_limit,
    test_axial_real_time_conserves_cylindrical_norm,
    test_axial_virial_relation,
    test_axial_matches_3d_cartesian,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_axial_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(before) == 1, "mutation anchor not found: %s" % name
    lib = oracle.compile_variant(src.replace(before, after), str(tmp_path / "libmut.so"))
    caught = None
    with oracle.use_library(lib):
        for check in AXIAL_CHECKS:
            try:
                check()
            except (AssertionError, RuntimeError) as e:
                caught = e
                break
    assert caught is not None, "planted mistake not caught: %s" % name
