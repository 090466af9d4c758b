"""Pins for the oracle's 1D and 2D condensates (no GPU): a grid axis with a
single node is absent (reading R20: no line solve, no links, no boundary,
coordinate 0, no spacing in the cell measure).  Each check ties the
lower-dimensional oracle to something other than itself: dense CN
propagators, exact separable fixed points, the continuum Gaussian, the 1D
and 2D Thomas-Fermi limits, the D-dimensional virial relation and
unitarity."""
import math

import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import inputs
from tests.test_oracle_pins import apply_axis, cn_dense, coords, h_axis

SHAPES = {"1d": (40, 1, 1), "2d_xy": (30, 26, 1), "2d_xz": (28, 1, 24)}


def present(shape):
    return [a for a in range(3) if shape[a] > 1]


def cell(shape, d):
    return float(np.prod([d[a] for a in present(shape)]))


@pytest.mark.parametrize("name", sorted(SHAPES))
@pytest.mark.parametrize("realtime", [False, True])
def test_sweeps_are_dense_cn_on_present_axes_and_identity_on_absent(name, realtime):
    shape, d, dt = SHAPES[name], (0.31, 0.27, 0.22), 0.013
    psi = inputs.random_field(shape, seed=5, envelope=False)
    for axis in range(3):
        got = oracle.sweep(psi.copy(), d, axis, dt, realtime)
        if shape[axis] == 1:
            assert np.array_equal(got, psi)
        else:
            ref = apply_axis(cn_dense(shape[axis], d[axis], dt, realtime), psi, axis)
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_g0_fixed_point_is_the_product_over_present_axes(name):
    """Imaginary time at g = 0 converges to the outer product of the present
    axes' dominant eigenvectors of C_a diag(exp(-dt w^2 x^2/2)); mu equals the
    sum of their dense Rayleigh quotients and the absent axes' rms is 0."""
    shape, d, omega, dt = SHAPES[name], (0.5, 0.45, 0.4), (1.0, 1.4, 2.0), 0.05
    psi = oracle.gaussian(shape, d, omega)
    oracle.step(psi, d, dt, omega, 0.0, False, 800)
    vecs = []
    for a in range(3):
        if shape[a] == 1:
            vecs.append(np.ones(1))
            continue
        x = coords(shape[a], d[a])[1:-1]
        t = cn_dense(shape[a], d[a], dt, False) @ np.diag(np.exp(-dt * 0.5 * omega[a] ** 2 * x * x))
        vals, v = np.linalg.eig(t)
        top = np.real(v[:, np.argmax(np.real(vals))])
        top *= np.sign(top[len(top) // 2])
        full = np.zeros(shape[a])
        full[1:-1] = top
        vecs.append(full)
    ref = np.einsum("i,j,k->ijk", *vecs).astype(complex)
    ref /= math.sqrt(cell(shape, d) * np.sum(np.abs(ref) ** 2))
    assert np.max(np.abs(psi - ref)) <= 1e-10 * np.max(np.abs(ref))
    obs = oracle.observables(ref, d, omega, 0.0)
    mu_ref = sum(vecs[a][1:-1] @ h_axis(shape[a], d[a], omega[a]) @ vecs[a][1:-1] /
                 (vecs[a][1:-1] @ vecs[a][1:-1]) for a in present(shape))
    assert abs(obs["mu"] - mu_ref) <= 1e-12 * mu_ref
    assert abs(obs["norm"] - 1.0) <= 1e-13
    for a, key in enumerate(("rms_x", "rms_y", "rms_z")):
        if shape[a] == 1:
            assert obs[key] == 0.0


@pytest.mark.parametrize("dims", [1, 2])
def test_gaussian_continuum_limit(dims):
    """The normalised Gaussian has mu -> sum of the present w_a / 2 and
    rms_a -> 1/sqrt(2 w_a) with O(d^2) error (an absent axis's trap
    frequency, here 0, does not enter)."""
    omega = (1.0, 1.4, 0.0) if dims == 2 else (1.3, 0.0, 0.0)
    errs = []
    for n in (41, 81):
        shape = (n, n if dims == 2 else 1, 1)
        d = tuple(12.0 / (n - 1) / math.sqrt(w) if w > 0 else 1.0 for w in omega)
        psi = oracle.gaussian(shape, d, omega)
        obs = oracle.observables(psi, d, omega, 0.0)
        assert abs(obs["norm"] - 1.0) < 1e-13
        for a, key in enumerate(("rms_x", "rms_y", "rms_z")[:dims]):
            assert abs(obs[key] - 1.0 / math.sqrt(2 * omega[a])) < 1e-8
        errs.append(abs(obs["mu"] - sum(omega[:dims]) / 2))
    assert errs[0] < 2e-2
    assert 3.0 <= errs[0] / errs[1] <= 5.0


def _ground_state_lowdim(shape, omega, g, mu_tf, tol=1e-9):
    """Grid holding 1.3 Thomas-Fermi radii (and 6 oscillator lengths) per
    present axis; dt = 0.2 d^2."""
    d = []
    for n, w in zip(shape, omega):
        if n == 1:
            d.append(1.0)
            continue
        half = max(6.0 / math.sqrt(w), 1.3 * math.sqrt(2 * mu_tf) / w)
        d.append(2 * half / (n - 1))
    dt = 0.2 * min(d[a] for a in range(3) if shape[a] > 1) ** 2
    psi = oracle.gaussian(shape, d, omega)
    oracle.run_imag_until(psi, d, dt, omega, g, tol, 10, 200000)
    return tuple(d), psi


@pytest.mark.parametrize("dims", [1, 2])
def test_thomas_fermi_limit_and_virial(dims):
    """For growing g, mu approaches the D-dimensional Thomas-Fermi value from
    above (1D: (3 g gamma / 4 sqrt 2)^(2/3); 2D: sqrt(g gamma nu / pi)), and
    the virial relation 2K - 2P + D E_int = 0 holds up to discretisation
    (pins the cell measure and the interaction weight in D dimensions)."""
    if dims == 1:
        shape, omega, gs = (400, 1, 1), (1.0, 0.0, 0.0), (100.0, 1000.0)
        tf = lambda g: (3 * g * omega[0] / (4 * math.sqrt(2))) ** (2.0 / 3.0)
    else:
        shape, omega, gs = (96, 96, 1), (1.0, 1.0, 0.0), (100.0, 1000.0)
        tf = lambda g: math.sqrt(g * omega[0] * omega[1] / math.pi)
    ratios = []
    for g in gs:
        d, psi = _ground_state_lowdim(shape, omega, g, tf(g))
        obs = oracle.observables(psi, d, omega, g)
        ratios.append(obs["mu"] / tf(g))
        e_int = obs["mu"] - obs["energy"]
        pot = 0.5 * sum(omega[a] ** 2 * obs[k] ** 2 for a, k in enumerate(("rms_x", "rms_y", "rms_z")))
        kin = obs["energy"] - pot - e_int
        assert abs(2 * kin - 2 * pot + dims * e_int) <= 1e-2 * obs["energy"], (dims, g, obs)
    assert ratios[0] > ratios[1] > 1.0
    assert ratios[1] - 1.0 <= 0.05


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_real_time_norm_is_conserved(name):
    shape, d, omega, g = SHAPES[name], (0.3, 0.3, 0.3), (0.5, 1.0, 1.5), 30.0
    psi = inputs.random_field(shape, seed=13)
    oracle.renormalize(psi, d)
    oracle.step(psi, d, 0.01, omega, g, True, 500)
    assert abs(oracle.observables(psi, d, omega, g)["norm"] - 1.0) <= 1e-12


def test_grids_without_a_present_axis_or_with_two_nodes_are_refused():
    for shape in ((1, 1, 1), (2, 5, 5), (5, 2, 1)):
        with pytest.raises(RuntimeError):
            oracle.gaussian(shape, (0.3, 0.3, 0.3), (1.0, 1.0, 1.0))


# ---------------------------------------------------------------- planted mistakes
LOWDIM_MUTATIONS = {
    "absent axis spacing in the cell measure": ("        if (n[a] > 1)\n            v *= d[a];",
                                                "        if (n[a] >= 1)\n            v *= d[a];"),
    "absent axis treated as a boundary": ("    return n > 1 && (idx == 0 || idx == n - 1);",
                                          "    return (idx == 0 || idx == n - 1);"),
    "absent axis Gaussian factor": (
        "double fz = n[2] > 1 ? pow(omega[2] / M_PI, 0.25) * exp(-0.5 * omega[2] * z * z) : 1.0;",
        "double fz = pow(omega[2] / M_PI, 0.25) * exp(-0.5 * omega[2] * z * z);"),
}


@pytest.mark.parametrize("name", sorted(LOWDIM_MUTATIONS))
def test_lowdim_pins_catch_planted_mistake(name, tmp_path):
    """Copies of the oracle's source with a plausible mistake in the absent-
    axis logic fail at least one of the pins above (on the CPU)."""
    before, after = LOWDIM_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(before) == 1, "mutation anchor not found: %s" % name
    lib = oracle.compile_variant(src.replace(before, after), str(tmp_path / "libmut.so"))
    checks = [lambda: test_g0_fixed_point_is_the_product_over_present_axes("2d_xz"),
              lambda: test_g0_fixed_point_is_the_product_over_present_axes("1d"),
              lambda: test_gaussian_continuum_limit(2)]
    caught = None
    with oracle.use_library(lib):
        for check in checks:
            try:
                check()
            except (AssertionError, RuntimeError) as e:  # a pin failed, or the oracle refused
                caught = e
                break
    assert caught is not None, "no pin caught the planted mistake: %s" % name
