"""Batched form (GPU): many uneven condensates advanced by one launch per
sweep covering all instances.  Each instance must equal the single-condensate
path configured the same way, bit for bit, and the batched convergence loop
must reach the oracle's ground states."""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def uneven(count, seed, scale=0.5, g_max=200.0):
    """A small uneven batch with the recipe of the 64-instance workload
    (grids shrunk by `scale` so the oracle stays fast)."""
    ps = inputs.batch_problems(count, seed=seed, g_max=g_max)
    out = []
    for p in ps:
        shape = tuple(max(5, int(n * scale)) for n in p.shape)
        q = inputs.sized_box(shape, p.omega, p.g)
        q.name = p.name
        out.append(q)
    return out


@pytest.mark.parametrize("prec,field", [("f32", "complex"), ("f64", "real"), ("f32", "real")])
def test_batch_instances_equal_single_runs(prec, field):
    from paper_1601_04641_gb300.solver import GP, Batch
    probs = uneven(7, seed=5)
    b = Batch(probs, prec, field)
    b.init_gaussian()
    b.step_imag(23)                       # graph blocks of 16, then 7 single launches
    w = b.window()
    n_tma = 0
    for i, p in enumerate(probs):
        gp = GP(p.shape, p.d, p.dt, p.omega, p.g, prec, field)
        # adjacent line pairs under the batch's rule (window 4, 8-byte
        # elements, even line counts, even nz for y lines): the pair forms cut
        # lines into 8-node chunks, so both must pair alike to agree bit for bit
        assert w[0] == w[1]
        gp.set_pair_lines(prec == "f32" and field == "complex" and w[0] == 4)
        # the batch takes the TMA z sweep for the instances whose rows fit
        # it, by the single handle's rule (same line arithmetic, same norm
        # summation order)
        gp.set_tma(True)
        seg, _ = b.segments(i)
        for ax in range(3):
            gp.set_axis_window(ax, w[ax])
            gp.set_segments(ax, seg[ax])
        gp.init_gaussian()
        gp.step_imag(23)
        assert np.array_equal(b.get_psi(i), gp.get_psi()), p.name
        n_tma += gp.tma_in_use()
        gp.close()
    obs = b.observables()
    assert all(o["step"] == 23 for o in obs)
    assert b.tma_count() == n_tma
    if prec == "f32":
        assert 0 < n_tma < len(probs)  # both z-sweep launches of the batch ran
    b.close()


@pytest.mark.parametrize("field", ["complex", "real"])
def test_batch_tma_z_sweep_matches_copy_form_and_oracle(field):
    """The batched z sweep with the TMA group on and off: psi agrees to FP32
    rounding (same arithmetic per line, different chunking of the windowed
    solve), and both follow the oracle's steps."""
    from paper_1601_04641_gb300.solver import Batch
    probs = uneven(6, seed=21, scale=0.6)
    out = {}
    for on in (True, False):
        b = Batch(probs, "f32", field)
        b.set_tma(on)
        assert (b.tma_count() > 0) == on
        b.init_gaussian()
        b.step_imag(12)
        out[on] = [b.get_psi(i).astype(np.float64 if field == "real" else np.complex128)
                   for i in range(len(probs))]
        b.close()
    for i, p in enumerate(probs):
        ref = oracle.gaussian(p.shape, p.d, p.omega)
        oracle.step(ref, p.d, p.dt, p.omega, p.g, False, 12)
        scale = float(np.max(np.abs(ref)))
        assert float(np.max(np.abs(out[True][i] - out[False][i]))) <= 1e-6 * scale, p.name
        assert float(np.max(np.abs(out[True][i] - ref))) <= 1e-5 * scale, p.name


def test_batch_convergence_matches_oracle_fp64():
    """FP64 batch run to |dmu| < 1e-9: every instance takes the oracle's
    number of steps and reaches its mu to 1e-12."""
    from paper_1601_04641_gb300.solver import Batch
    probs = uneven(5, seed=9, scale=0.3)
    b = Batch(probs, "f64", "real")
    b.init_gaussian()
    steps = b.run_imag_until(1e-9, 10, 4000)
    obs = b.observables()
    for i, p in enumerate(probs):
        psi = oracle.gaussian(p.shape, p.d, p.omega)
        n_ref, mu_ref = oracle.run_imag_until(psi, p.d, p.dt, p.omega, p.g, 1e-9, 10, 4000)
        assert steps[i] == n_ref, (p.name, steps[i], n_ref)
        assert abs(obs[i]["mu"] - mu_ref) <= 1e-12 * mu_ref
    b.close()


def test_batch_fp32_ground_states_match_oracle():
    """FP32 complex batch (the 64-instance workload's form) run to
    |dmu| < 1e-6: mu within 1e-5 of the FP64 oracle run with the same stop
    rule from the same start."""
    from paper_1601_04641_gb300.solver import Batch
    probs = uneven(6, seed=3, scale=0.35)
    b = Batch(probs, "f32", "complex")
    b.init_gaussian()
    steps = b.run_imag_until(1e-6, 10, 20000)
    obs = b.observables()
    for i, p in enumerate(probs):
        psi = oracle.gaussian(p.shape, p.d, p.omega)
        _, mu_ref = oracle.run_imag_until(psi, p.d, p.dt, p.omega, p.g, 1e-6, 10, 20000)
        assert steps[i] < 20000
        assert abs(obs[i]["mu"] - mu_ref) <= 1e-5 * mu_ref, (p.name, obs[i]["mu"], mu_ref)
    b.close()


def test_stop_rule_with_energy_never_stops_earlier():
    """Rule 1 (|dmu| < tol and |dE| < tol) takes at least as many steps as the
    mu-only rule and ends at least as close to a tightly converged mu, for a
    single handle and for a batch (same instances)."""
    from paper_1601_04641_gb300.solver import GP, Batch
    probs = uneven(4, seed=9)
    out = {}
    for rule in (0, 1):
        b = Batch(probs, "f64", "real")
        b.set_stop_rule(rule)
        b.init_gaussian()
        steps = b.run_imag_until(1e-7, 10, 50000)
        out[rule] = (steps, [o["mu"] for o in b.observables()])
        b.close()
    for i, p in enumerate(probs):
        gp = GP(p.shape, p.d, p.dt, p.omega, p.g, "f64", "real")
        gp.init_gaussian()
        gp.run_imag_until(1e-12, 10, 400000)
        mu_ref = gp.observables()["mu"]
        gp.set_stop_rule(1)
        gp.init_gaussian()
        gp.run_imag_until(1e-7, 10, 50000)
        mu1 = gp.observables()["mu"]
        gp.close()
        assert out[1][0][i] >= out[0][0][i]
        assert abs(out[1][1][i] - mu_ref) <= abs(out[0][1][i] - mu_ref) + 1e-12
        assert abs(out[1][1][i] - mu_ref) <= 1e-5 * mu_ref
        assert abs(mu1 - mu_ref) <= 1e-5 * mu_ref


def test_stop_rule_two_checks_matches_oracle():
    """Rule 2 (rule 1's test at two consecutive checks): the FP64 batch and a
    single handle take the oracle's number of steps, never fewer than rule 1."""
    from paper_1601_04641_gb300.solver import GP, Batch
    probs = uneven(4, seed=17, scale=0.3)
    steps = {}
    for rule in (1, 2):
        b = Batch(probs, "f64", "real")
        b.set_stop_rule(rule)
        b.init_gaussian()
        steps[rule] = b.run_imag_until(1e-8, 10, 20000)
        b.close()
    for i, p in enumerate(probs):
        psi = oracle.gaussian(p.shape, p.d, p.omega)
        n_ref, mu_ref = oracle.run_imag_until(psi, p.d, p.dt, p.omega, p.g, 1e-8, 10, 20000, rule=2)
        gp = GP(p.shape, p.d, p.dt, p.omega, p.g, "f64", "real")
        gp.set_stop_rule(2)
        gp.init_gaussian()
        n_h = gp.run_imag_until(1e-8, 10, 20000)
        mu_h = gp.observables()["mu"]
        gp.close()
        assert steps[2][i] == n_ref == n_h, (p.name, steps[2][i], n_ref, n_h)
        assert steps[2][i] >= steps[1][i]
        assert abs(mu_h - mu_ref) <= 1e-12 * mu_ref


@pytest.mark.parametrize("prec,field", [("f64", "real"), ("f32", "complex")])
def test_dt_schedule_reaches_the_target_fixed_point(prec, field):
    """Converging at 10 dt first, then at dt (gp_batch_run_imag_schedule,
    gp_run_imag_schedule) ends at the fixed point of dt -- within the stop
    rule's residual of a tightly converged plain run -- in fewer steps than
    the plain run, and leaves dt as it was."""
    from paper_1601_04641_gb300.solver import GP, Batch
    probs = uneven(5, seed=13)
    levels = [(10.0, 1e-5), (1.0, 1e-7)]
    b = Batch(probs, prec, field)
    b.set_stop_rule(1)
    b.init_gaussian()
    steps_s = b.run_imag_schedule(levels, 10, 50000)
    mu_s = [o["mu"] for o in b.observables()]
    b.init_gaussian()
    steps_p = b.run_imag_until(1e-7, 10, 50000)
    mu_p = [o["mu"] for o in b.observables()]
    b.close()
    assert sum(steps_s) < sum(steps_p), (steps_s, steps_p)
    tol = 2e-5 if prec == "f32" else 1e-5
    for i, p in enumerate(probs):
        gp = GP(p.shape, p.d, p.dt, p.omega, p.g, "f64", "real")
        gp.init_gaussian()
        gp.run_imag_until(1e-12, 10, 400000)
        mu_ref = gp.observables()["mu"]
        # the single-handle schedule, then a plain continuation at the restored dt
        gp.set_stop_rule(1)
        gp.init_gaussian()
        gp.run_imag_schedule(levels, 10, 50000)
        mu_h = gp.observables()["mu"]
        gp.run_imag_until(1e-12, 10, 400000)
        mu_after = gp.observables()["mu"]
        gp.close()
        assert abs(mu_s[i] - mu_ref) <= tol * mu_ref, (i, mu_s[i], mu_ref)
        assert abs(mu_p[i] - mu_ref) <= tol * mu_ref
        assert abs(mu_h - mu_ref) <= 1e-5 * mu_ref
        assert abs(mu_after - mu_ref) <= 1e-7 * mu_ref  # dt restored (a wrong dt moves mu by ~1e-4)


def test_batch_segment_override_keeps_results():
    """Shorter segments on the strided axes (more threads per line, W + 1
    warm-up nodes each): psi agrees with the automatic segments to FP32
    rounding and with the oracle; negative lengths are refused."""
    from paper_1601_04641_gb300 import _native as N
    from paper_1601_04641_gb300.solver import Batch
    probs = uneven(4, seed=5, scale=0.6)
    out = {}
    for seg in (0, 24, 7):
        b = Batch(probs, "f32", "complex")
        b.set_segments(seg)
        if seg:
            assert all(b.segments(i)[0][0] == min(seg, p.shape[0] - 2) for i, p in enumerate(probs))
        b.init_gaussian()
        b.step_imag(12)
        out[seg] = [b.get_psi(i).astype(np.complex128) for i in range(len(probs))]
        b.close()
    b = Batch(probs, "f32", "complex")
    with pytest.raises(N.GPError) as e:
        b.set_segments(-1)
    assert e.value.status == N.GP_ERR_ARG
    b.close()
    for i, p in enumerate(probs):
        ref = oracle.gaussian(p.shape, p.d, p.omega)
        oracle.step(ref, p.d, p.dt, p.omega, p.g, False, 12)
        scale = float(np.max(np.abs(ref)))
        for seg in (24, 7):
            assert float(np.max(np.abs(out[seg][i] - out[0][i]))) <= 1e-6 * scale, (p.name, seg)
        assert float(np.max(np.abs(out[7][i] - ref))) <= 1e-5 * scale, p.name


@pytest.mark.parametrize("field", ["complex", "real"])
def test_batch_stream_groups_are_bit_identical(field):
    """Independent instance groups on their own streams (forked and joined
    by events, captured as parallel graph branches) change no result: every
    instance's launches and norm order are the same with 1, 3 or 16 groups."""
    from paper_1601_04641_gb300 import _native as N
    from paper_1601_04641_gb300.solver import Batch
    probs = uneven(7, seed=5, scale=0.5)
    out = {}
    for streams in (1, 3, 16):
        b = Batch(probs, "f32", field)
        b.set_streams(streams)
        b.init_gaussian()
        b.step_imag(23)  # graph blocks of 16, then 7 single launches
        out[streams] = ([b.get_psi(i) for i in range(len(probs))], [o["norm"] for o in b.observables()])
        b.close()
    for streams in (3, 16):
        for i in range(len(probs)):
            assert np.array_equal(out[streams][0][i], out[1][0][i]), (streams, i)
        assert out[streams][1] == out[1][1]
    b = Batch(probs, "f32", field)
    for bad in (0, 17):
        with pytest.raises(N.GPError) as e:
            b.set_streams(bad)
        assert e.value.status == N.GP_ERR_ARG
    b.close()
