"""Pins for the FP64 CPU oracle (no GPU).

The paper prints no worked example, so each oracle function is tied to
something other than itself: dense linear algebra, exact separable solutions,
continuum and Thomas-Fermi limits, the virial relation, unitarity and the
order of the splitting error.  Each test names the mistake it would catch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import inputs


# ---------------------------------------------------------------- helpers
def coords(n, d):
    return (np.arange(n) - 0.5 * (n - 1)) * d


def lap_interior(n, d):
    """Second-difference matrix on the n-2 interior nodes with zero ends."""
    m = n - 2
    return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1) +
            np.diag(np.ones(m - 1), -1)) / (d * d)


def cn_dense(n, d, dt, realtime):
    """Dense CN propagator for one axis, (I - a L)^-1 (I + a L) with a = dt/4
    (imaginary time, d/dtau = (1/2) d^2/dx^2) or a = i dt/4 (real time,
    d/dt = (i/2) d^2/dx^2): the trapezoidal rule over one step dt."""
    lap = lap_interior(n, d)
    a = (0.5j if realtime else 0.5) * dt * 0.5
    eye = np.eye(n - 2)
    return np.linalg.solve(eye - a * lap, eye + a * lap)


def apply_axis(mat, psi, axis):
    """Apply a dense interior operator along one axis; boundary nodes -> 0."""
    inner = [slice(None)] * 3
    inner[axis] = slice(1, -1)
    sub = psi[tuple(inner)]
    out = np.zeros_like(psi)
    moved = np.moveaxis(sub, axis, 0)
    res = np.tensordot(mat, moved, axes=([1], [0]))
    out[tuple(inner)] = np.moveaxis(res, 0, axis)
    return out


def h_axis(n, d, w):
    """1D dense Hamiltonian -1/2 L + 1/2 w^2 x^2 on interior nodes."""
    x = coords(n, d)[1:-1]
    return -0.5 * lap_interior(n, d) + np.diag(0.5 * w * w * x * x)


# ---------------------------------------------------------------- Thomas
@pytest.mark.parametrize("n", list(range(1, 17)))
def test_thomas_matches_dense_lu(n):
    """Thomas vs numpy dense LU on random diagonally dominant complex systems
    (catches a wrong multiplier, a sign error or an off-by-one in either pass)."""
    rng = np.random.default_rng(100 + n)
    sub = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    sup = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    diag = (np.abs(sub) + np.abs(sup) + 1.0) * np.exp(1j * rng.uniform(0, 2 * np.pi, n))
    rhs = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a = np.diag(diag).astype(complex)
    if n > 1:
        a += np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
    ref = np.linalg.solve(a, rhs)
    got = oracle.thomas(sub, diag, sup, rhs)
    assert np.max(np.abs(got - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


# ---------------------------------------------------------------- one sweep
@pytest.mark.parametrize("realtime", [False, True])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_matches_dense_cn(axis, realtime):
    """One CN line solve along each axis equals the dense CN propagator applied
    along that axis (distinct sizes and spacings per axis catch a transposed
    axis, a wrong stride or the wrong spacing; the dense form catches a dropped
    RHS term or a wrong sign of c)."""
    shape, d, dt = (9, 7, 6), (0.31, 0.27, 0.22), 0.013
    psi = inputs.random_field(shape, seed=7 + axis, envelope=False)
    ref = apply_axis(cn_dense(shape[axis], d[axis], dt, realtime), psi, axis)
    got = oracle.sweep(psi.copy(), d, axis, dt, realtime)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_sweep_ignores_and_zeroes_boundary():
    """Boundary values are not read (Dirichlet zero) and are written as zero."""
    shape, d, dt = (6, 5, 7), (0.3, 0.3, 0.3), 0.02
    psi = inputs.random_field(shape, seed=3, envelope=False)
    dirty = psi.copy()
    dirty[0] = 5.0
    dirty[-1] = -3.0 + 2.0j
    a = oracle.sweep(psi.copy(), d, 0, dt, True)
    b = oracle.sweep(dirty, d, 0, dt, True)
    assert np.array_equal(a[1:-1], b[1:-1])
    assert np.all(b[0] == 0) and np.all(b[-1] == 0)


# ---------------------------------------------------------------- g = 0 separable fixed point
def separable_fixed_point(shape, d, dt, omega):
    """Dominant eigenvector per axis of T_a = C_a diag(exp(-dt w_a^2 x^2 / 2)),
    outer product, normalised with dV (exact fixed point of the g = 0 imaginary
    step, which factorises by axis)."""
    vecs = []
    for n, da, w in zip(shape, d, omega):
        x = coords(n, da)[1:-1]
        t = cn_dense(n, da, dt, False) @ np.diag(np.exp(-dt * 0.5 * w * w * x * x))
        vals, v = np.linalg.eig(t)
        top = np.real(v[:, np.argmax(np.real(vals))])
        top = top * np.sign(top[len(top) // 2])
        full = np.zeros(n)
        full[1:-1] = top
        vecs.append(full)
    psi = np.einsum("i,j,k->ijk", *vecs).astype(complex)
    psi /= math.sqrt(np.prod(d) * np.sum(np.abs(psi) ** 2))
    return psi, vecs


def test_g0_fixed_point_and_observables():
    """Imaginary time at g = 0 converges to the outer product of per-axis
    dominant eigenvectors (pins the kick's trap term, its axis assignment and
    coordinate centring), and the oracle's mu / rms on that state equal the
    per-axis dense Rayleigh quotients (pins the kinetic link sum, the
    potential sum and the rms formula, axis by axis)."""
    shape, d, omega = (14, 12, 10), (0.55, 0.5, 0.45), (1.0, 1.4, 2.0)
    dt = 0.05
    psi = oracle.gaussian(shape, d, omega)
    oracle.step(psi, d, dt, omega, 0.0, False, 600)
    ref, vecs = separable_fixed_point(shape, d, dt, omega)
    assert np.max(np.abs(psi - ref)) <= 1e-10 * np.max(np.abs(ref))

    obs = oracle.observables(ref, d, omega, 0.0)
    mu_ref = 0.0
    for n, da, w, v in zip(shape, d, omega, vecs):
        vi = v[1:-1]
        mu_ref += vi @ h_axis(n, da, w) @ vi / (vi @ vi)
    assert abs(obs["mu"] - mu_ref) <= 1e-12 * mu_ref
    assert abs(obs["energy"] - mu_ref) <= 1e-12 * mu_ref
    assert abs(obs["norm"] - 1.0) <= 1e-13
    for key, n, da, v in zip(("rms_x", "rms_y", "rms_z"), shape, d, vecs):
        x = coords(n, da)
        assert abs(obs[key] - math.sqrt(np.sum(x * x * v * v) / np.sum(v * v))) <= 1e-12


def test_g0_mu_converges_quadratically_in_dt():
    """At g = 0 the fixed-point mu tends to sum_a lambda_min(H_a) with an
    O(dt^2) error: the Lie product C K is similar to the symmetric product
    K^(1/2) C K^(1/2), so its fixed point is O(dt) from the exact eigenvector
    and the Rayleigh quotient is off by O(dt^2).  Halving dt divides the error
    by about 4 (a wrong kick weight would leave an O(1) error)."""
    shape, d, omega = (12, 11, 10), (0.6, 0.55, 0.5), (1.0, 1.4, 2.0)
    exact = sum(np.linalg.eigvalsh(h_axis(n, da, w))[0] for n, da, w in zip(shape, d, omega))
    errs = []
    for dt in (0.08, 0.04):
        ref, _ = separable_fixed_point(shape, d, dt, omega)
        psi = oracle.gaussian(shape, d, omega)
        oracle.step(psi, d, dt, omega, 0.0, False, int(round(40 / dt)))
        assert np.max(np.abs(psi - ref)) <= 1e-9
        errs.append(oracle.observables(psi, d, omega, 0.0)["mu"] - exact)
    assert errs[0] > 0 and errs[1] > 0
    assert 3.5 <= errs[0] / errs[1] <= 4.5


def test_gaussian_continuum_limit():
    """The normalised Gaussian has mu -> (gamma+nu+lambda)/2 and
    rms_a -> 1/sqrt(2 w_a) as d -> 0 with O(d^2) error (pins the initial
    state, the normalisation and the observables' continuum meaning)."""
    omega = (1.0, 1.4, 2.0)
    errs = []
    for n in (25, 49):
        shape = (n, n, n)
        d = tuple(12.0 / (n - 1) / math.sqrt(w) for w in omega)
        psi = oracle.gaussian(shape, d, omega)
        obs = oracle.observables(psi, d, omega, 0.0)
        assert abs(obs["norm"] - 1.0) < 1e-13
        for key, w in zip(("rms_x", "rms_y", "rms_z"), omega):
            assert abs(obs[key] - 1.0 / math.sqrt(2 * w)) < 1e-8
        errs.append(abs(obs["mu"] - sum(omega) / 2))
    assert errs[0] < 5e-2
    assert 3.0 <= errs[0] / errs[1] <= 5.0


# ---------------------------------------------------------------- interacting ground state
def _ground_state(g, n=32, omega=(1.0, 1.0, 1.0), dt_factor=0.2, tol=1e-8):
    p = inputs.sized_box((n, n, n), omega, g, dt_factor=dt_factor)
    psi = oracle.gaussian(p.shape, p.d, p.omega)
    oracle.run_imag_until(psi, p.d, p.dt, p.omega, p.g, tol, 10, 20000)
    return p, psi


def test_thomas_fermi_limit_and_virial():
    """For growing g the ground-state mu approaches the Thomas-Fermi value
    mu_TF = (15 g gamma nu lambda / 4 pi)^(2/5) / 2 from above, monotonically
    (pins the sign and weight of g in the kick and in mu), and the virial
    relation 2K - 2P + 3 E_int = 0 holds up to discretisation (pins the
    relative weights of kinetic, trap and interaction sums)."""
    ratios = []
    for g in (100.0, 500.0, 2000.0):
        p, psi = _ground_state(g)
        obs = oracle.observables(psi, p.d, p.omega, p.g)
        mu_tf = 0.5 * (15 * g / (4 * math.pi)) ** 0.4
        ratios.append(obs["mu"] / mu_tf)
        e_int = obs["mu"] - obs["energy"]
        pot = 0.5 * sum(w * w * obs[k] ** 2 for w, k in zip(p.omega, ("rms_x", "rms_y", "rms_z")))
        kin = obs["energy"] - pot - e_int
        virial = 2 * kin - 2 * pot + 3 * e_int
        assert abs(virial) <= 1e-2 * obs["energy"], (g, virial, obs)
    assert ratios[0] > ratios[1] > ratios[2] > 1.0
    assert ratios[2] - 1.0 <= 0.03


def test_imag_time_positivity_symmetry_and_energy_descent():
    """Imaginary time from a positive, mirror-symmetric start stays positive in
    the interior and mirror-symmetric on the centred grid, and the energy does
    not increase after the transient."""
    shape, d, omega, g = (16, 14, 12), (0.5, 0.5, 0.5), (1.0, 1.4, 2.0), 30.0
    dt = 0.1 * 0.25
    psi = oracle.gaussian(shape, d, omega)
    energies = []
    for _ in range(20):
        oracle.step(psi, d, dt, omega, g, False, 5)
        energies.append(oracle.observables(psi, d, omega, g)["energy"])
    inner = psi[1:-1, 1:-1, 1:-1]
    assert np.all(inner.real > 0) and np.all(inner.imag == 0)
    for ax in range(3):
        assert np.max(np.abs(psi - np.flip(psi, axis=ax))) <= 1e-13
    assert all(b <= a + 1e-12 for a, b in zip(energies[2:], energies[3:]))


# ---------------------------------------------------------------- real time
def test_real_time_norm_is_conserved():
    """Every real-time sub-step is unitary in the rectangle-rule norm (a phase
    kick and a Cayley transform of a Hermitian matrix): 1000 steps keep the
    norm to 1e-12 (catches a non-unitary kick or a wrong c)."""
    shape, d, omega, g = (12, 11, 10), (0.5, 0.5, 0.5), (0.5, 1.0, 1.5), 40.0
    psi = inputs.random_field(shape, seed=11)
    oracle.renormalize(psi, d)
    oracle.step(psi, d, 0.01, omega, g, True, 1000)
    assert abs(oracle.observables(psi, d, omega, g)["norm"] - 1.0) <= 1e-12


def test_real_time_energy_drift_is_first_order():
    """Lie splitting conserves the energy only to O(dt): after a quench the
    drift over a fixed time interval halves when dt halves (a kick phase or
    CN coefficient of the wrong sign makes the drift O(1) instead)."""
    shape, d, omega = (20, 18, 16), (0.4, 0.4, 0.4), (1.0, 1.4, 2.0)
    psi0 = oracle.gaussian(shape, d, omega)
    oracle.step(psi0, d, 0.02, omega, 20.0, False, 200)
    drifts = []
    for dt in (0.004, 0.002):
        psi = psi0.copy()
        e0 = oracle.observables(psi, d, omega, 40.0)["energy"]
        oracle.step(psi, d, dt, omega, 40.0, True, int(round(0.2 / dt)))
        drifts.append(abs(oracle.observables(psi, d, omega, 40.0)["energy"] - e0) / e0)
    assert drifts[0] < 2e-2
    assert 1.6 <= drifts[0] / drifts[1] <= 2.4


# ---------------------------------------------------------------- symmetric splitting
def _strang_case():
    shape, d, omega, g = (16, 14, 12), (0.35, 0.4, 0.45), (1.0, 1.3, 0.8), 20.0
    psi0 = inputs.random_field(shape, seed=3)
    oracle.renormalize(psi0, d)
    return shape, d, omega, g, psi0


def test_strang_is_time_reversible():
    """Half kick, CN sweeps, half kick is symmetric: each CN sweep with -dt is
    the inverse of the sweep with dt, the sweeps of different axes commute,
    and a real-time kick keeps |psi|, so n steps with dt then n with -dt give
    psi back to rounding.  The Lie order (kick then sweeps) does not (catches
    a missing or misplaced half kick)."""
    shape, d, omega, g, psi0 = _strang_case()
    psi = psi0.copy()
    oracle.step_strang(psi, d, 0.01, omega, g, 20)
    oracle.step_strang(psi, d, -0.01, omega, g, 20)
    assert np.max(np.abs(psi - psi0)) <= 1e-12 * np.max(np.abs(psi0))
    lie = psi0.copy()
    oracle.step(lie, d, 0.01, omega, g, True, 20)
    oracle.step(lie, d, -0.01, omega, g, True, 20)
    assert np.max(np.abs(lie - psi0)) >= 1e-4 * np.max(np.abs(psi0))


def test_strang_is_second_order():
    """Over a fixed time the symmetric splitting's error falls fourfold when
    dt halves, the Lie splitting's twofold; both against the Lie method at a
    32x finer step (pinned above), so a symmetric step with wrong kick
    weights, converging to another limit, fails too."""
    shape, d, omega, g, psi0 = _strang_case()
    T = 0.08
    ref = psi0.copy()
    oracle.step(ref, d, T / 4096, omega, g, True, 4096)
    err = {}
    for name, fn in (("strang", lambda p, dt, n: oracle.step_strang(p, d, dt, omega, g, n)),
                     ("lie", lambda p, dt, n: oracle.step(p, d, dt, omega, g, True, n))):
        e = []
        for n in (8, 16):
            p = psi0.copy()
            fn(p, T / n, n)
            e.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
        err[name] = e
    assert 3.3 <= err["strang"][0] / err["strang"][1] <= 4.7, err
    assert 1.7 <= err["lie"][0] / err["lie"][1] <= 2.6, err
    assert err["strang"][1] < 0.5 * err["lie"][1]
