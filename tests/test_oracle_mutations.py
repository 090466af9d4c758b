"""Plants plausible mistakes in copies of the oracle's C source (on the CPU)
and checks that the pins in test_oracle_pins.py catch every one of them."""
import pytest

import oracle
from tests import test_oracle_pins as pins

MUTATIONS = {
    "rhs drops right neighbour": (
        "rhs[m - 1] = c * left + (1.0 - 2.0 * c) * line[m] + c * right;",
        "rhs[m - 1] = c * left + (1.0 - 2.0 * c) * line[m] + 0.0 * right;"),
    "real-time CN coefficient sign": (
        "const cplx c = (realtime ? I : 1.0) * dt",
        "const cplx c = (realtime ? -I : 1.0) * dt"),
    "CN coefficient dt/2d^2": (
        "dt / (4.0 * d[axis] * d[axis])", "dt / (2.0 * d[axis] * d[axis])"),
    "sweep uses dx on every axis": (
        "dt / (4.0 * d[axis] * d[axis])", "dt / (4.0 * d[0] * d[0])"),
    "trap axes swapped": (
        "return 0.5 * (omega[0] * omega[0] * x * x + omega[1] * omega[1] * y * y +",
        "return 0.5 * (omega[1] * omega[1] * x * x + omega[0] * omega[0] * y * y +"),
    "trap without 1/2": (
        "return 0.5 * (omega[0] * omega[0] * x * x", "return 1.0 * (omega[0] * omega[0] * x * x"),
    "real-time kick phase sign": ("psi[s] *= cexp(-I * arg);", "psi[s] *= cexp(I * arg);"),
    "kick with half g": ("double arg = dt * (trap(n, d, omega, i, j, k) + g * rho);",
                     "double arg = dt * (trap(n, d, omega, i, j, k) + 0.5 * g * rho);"),
    "grid not centred": ("return ((double)idx - 0.5 * (double)(n - 1)) * d;",
                         "return ((double)idx - 0.5 * (double)n) * d;"),
    "thomas back-substitution sign": ("x[m] = dp[m] - cp[m] * x[m + 1];",
                                      "x[m] = dp[m] + cp[m] * x[m + 1];"),
    "thomas forward sign": ("dp[m] = (rhs[m] - sub[m] * dp[m - 1]) / den;",
                            "dp[m] = (rhs[m] + sub[m] * dp[m - 1]) / den;"),
    "norm without dV": ("return cell_volume(n, d) * sum;", "return sum;"),
    "kinetic without 1/2": ("double kin = 0.5 * dv *", "double kin = dv *"),
    "mu with half interaction": ("out[1] = (kin + pot + g * inter) / norm;",
                                 "out[1] = (kin + pot + 0.5 * g * inter) / norm;"),
    "energy with full interaction": ("out[2] = (kin + pot + 0.5 * g * inter) / norm;",
                                     "out[2] = (kin + pot + g * inter) / norm;"),
    "rms axes swapped": ("out[3] = sqrt(dv * s_x2 / norm);", "out[3] = sqrt(dv * s_y2 / norm);"),
    "last z link dropped": ("if (k + 1 < n[2]) {", "if (k + 2 < n[2]) {"),
    "gaussian width": ("exp(-0.5 * omega[0] * x * x)", "exp(-omega[0] * x * x)"),
    "symmetric step with full kicks": ("int rc = oracle_kick(n, d, psi_ri, 0.5 * dt, omega, g, 1);",
                                       "int rc = oracle_kick(n, d, psi_ri, 1.0 * dt, omega, g, 1);"),
    "symmetric step without the trailing half kick": (
        "            rc = oracle_kick(n, d, psi_ri, 0.5 * dt, omega, g, 1);\n",
        "            rc = ORACLE_OK;\n"),
    "no renormalisation": ("if (rc == ORACLE_OK && !realtime)\n            rc = oracle_renormalize",
                           "if (rc == ORACLE_OK && realtime > 1)\n            rc = oracle_renormalize"),
}

CHECKS = [
    lambda: pins.test_thomas_matches_dense_lu(5),
    lambda: [pins.test_sweep_matches_dense_cn(a, rt) for a in range(3) for rt in (False, True)],
    pins.test_sweep_ignores_and_zeroes_boundary,
    pins.test_g0_fixed_point_and_observables,
    pins.test_gaussian_continuum_limit,
    pins.test_real_time_norm_is_conserved,
    pins.test_real_time_energy_drift_is_first_order,
    pins.test_imag_time_positivity_symmetry_and_energy_descent,
    pins.test_g0_mu_converges_quadratically_in_dt,
    pins.test_thomas_fermi_limit_and_virial,
    pins.test_strang_is_time_reversible,
    pins.test_strang_is_second_order,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(before) == 1, "mutation anchor not found: %s" % name
    lib = oracle.compile_variant(src.replace(before, after), str(tmp_path / "libmut.so"))
    caught = None
    with oracle.use_library(lib):
        for check in CHECKS:
            try:
                check()
            except (AssertionError, RuntimeError) as e:  # a pin failed, or the oracle refused
                caught = e
                break
    assert caught is not None, "no pin caught the planted mistake: %s" % name
