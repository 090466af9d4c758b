"""FP16 storage of a real field in imaginary time (GP_F16: half-precision psi,
FP32 arithmetic) against the FP64 oracle on the same half-precision inputs
(GPU only).

- The observables of a half field are FP32 sums of exactly widened values:
  the oracle's on the same values to 1e-6.
- One sweep (with the kick on x) rounds each result to nearest once: every
  element is within half an FP16 ulp of the oracle's sweep of the same input
  (2^-11 relative), plus the FP32 solve's own error (the z stage's pending
  renormalisation, applied by get_psi, rounds once more).
- Several steps stay within the per-sweep rounding bound, grown by the steps.
- Two and four lines per thread use the same 16-node chunks and agree bit
  for bit; the TMA and per-thread-copy forms of the x sweep agree bit for bit.
- As a coarse stage: an FP16 run to |dmu| < 1e-3, handed to an FP32 handle,
  reaches the FP32 fixed point in fewer FP32 steps than from the Gaussian.
- Calls that would need a form FP16 storage does not have are refused.
"""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu

D = (0.31, 0.27, 0.22)
OMEGA = (1.0, 1.4, 2.0)
OBS = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z")
U16 = 2.0 ** -11  # half the spacing of FP16 numbers in [1, 2), relative


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, dt=0.004, g=12.0, prec="f16", d=D):
    from paper_1601_04641_gb300.solver import GP
    return GP(shape, d, dt, OMEGA, g, prec, "real")


def half_field(shape, seed):
    return np.abs(inputs.random_field(shape, seed=seed)).astype(np.float16)


@pytest.mark.parametrize("shape", [(24, 20, 64), (37, 26, 56), (30, 1, 64), (9, 7, 72)])
def test_fp16_observables_match_oracle(shape):
    psi = half_field(shape, 3)
    gp = make(shape)
    gp.set_psi(psi)
    got = gp.observables()
    gp.close()
    ref = oracle.observables(psi.astype(np.complex128), D, OMEGA, 12.0)
    for k in OBS:
        assert abs(got[k] - ref[k]) <= 1e-6 * abs(ref[k]), (k, got[k], ref[k])


@pytest.mark.parametrize("shape", [(24, 20, 64), (37, 26, 56), (30, 1, 64)])
@pytest.mark.parametrize("stage", [0, 1, 2])
def test_fp16_sweep_rounds_once(shape, stage):
    if shape[stage] == 1:
        pytest.skip("absent axis")
    dt, g = 0.004, 12.0
    psi = half_field(shape, 11 + stage)
    gp = make(shape, dt, g)
    gp.set_psi(psi)
    gp.stage(stage, False)
    got = gp.get_psi().astype(np.float64)
    gp.close()
    ref = psi.astype(np.complex128)
    if stage == 0:
        oracle.kick(ref, D, dt, OMEGA, g, False)
    oracle.sweep(ref, D, stage, dt, False)
    roundings = 1
    if stage == 2:
        # the z stage leaves its renormalisation pending; get_psi applies it
        # to the stored half values and rounds once more
        ref = ref / np.sqrt(oracle.observables(ref, D, OMEGA, g)["norm"])
        roundings = 2
    ref = ref.real
    scale = float(np.max(np.abs(ref)))
    bound = roundings * U16 * np.abs(ref) + 2.0 ** -24 + 2e-6 * scale
    excess = np.abs(got - ref) - bound
    assert float(np.max(excess)) <= 0.0, float(np.max(np.abs(got - ref)))


def test_fp16_steps_within_rounding_bound():
    shape, dt, g, steps = (24, 20, 64), 0.004, 12.0, 6
    psi = half_field(shape, 21)
    gp = make(shape, dt, g)
    gp.set_psi(psi)
    gp.step_imag(steps)
    got = gp.get_psi().astype(np.float64)
    gp.close()
    ref = psi.astype(np.complex128)
    oracle.step(ref, D, dt, OMEGA, g, False, steps)
    ref = ref.real
    scale = float(np.max(np.abs(ref)))
    # three roundings a step, each at most 2^-11 of the largest value, carried
    # by sweeps that do not amplify (imaginary time contracts)
    assert float(np.max(np.abs(got - ref))) <= 3 * steps * U16 * scale


@pytest.mark.parametrize("window", [4, 8, 16])
def test_fp16_pairs_quads_and_tma_agree_bitwise(window):
    shape, steps = (36, 28, 64), 3
    psi = half_field(shape, 31)
    out = {}
    for lines, tma in ((4, -1), (2, -1), (4, 0), (2, 3)):
        gp = make(shape)
        gp.set_window(window)
        for ax in (0, 1):
            gp.set_lines_per_thread(ax, lines)
        gp.set_tma_lines(tma)
        assert gp.lines_per_thread(0)[:2] == (lines, lines)
        gp.set_psi(psi)
        gp.step_imag(steps)
        out[(lines, tma)] = gp.get_psi()
        gp.close()
    first = out[(4, -1)]
    for k, v in out.items():
        assert np.array_equal(v, first), k


def test_fp16_coarse_stage_then_fp32():
    """FP16 to |dmu| < 1e-3 (its fixed point is about 2^13 times farther from
    the ground state than FP32's), then FP32 from the FP16 state: fewer FP32
    steps than the FP32 run from the Gaussian, and the same fixed point."""
    shape, d = (40, 32, 64), (0.35, 0.35, 0.3)
    dt, g = 0.1 * 0.3 ** 2, 20.0
    h16 = make(shape, dt, g, "f16", d)
    h16.init_gaussian()
    h16.run_imag_until(1e-3, 10, 20000)
    psi16 = h16.get_psi()
    mu16 = h16.observables()["mu"]
    h16.close()
    runs = {}
    for start in ("gauss", "f16"):
        h = make(shape, dt, g, "f32", d)
        if start == "gauss":
            h.init_gaussian()
        else:
            h.set_psi(psi16.astype(np.float32))
        runs[start] = (h.run_imag_until(1e-7, 10, 50000), h.observables()["mu"])
        h.close()
    assert runs["f16"][0] < runs["gauss"][0], runs
    assert abs(runs["f16"][1] - runs["gauss"][1]) <= 2e-6 * runs["gauss"][1], runs
    assert abs(mu16 - runs["gauss"][1]) <= 2e-2 * runs["gauss"][1], (mu16, runs)


def test_fp16_refusals():
    from paper_1601_04641_gb300.solver import GP, Batch
    for shape, field in (((24, 20, 64), "complex"), ((24, 20, 60), "real"), ((24, 20, 48), "real")):
        with pytest.raises((N.GPError, ValueError)) as e:
            GP(shape, D, 0.004, OMEGA, 1.0, "f16", field)
        if isinstance(e.value, N.GPError):
            assert e.value.status == N.GP_ERR_ARG
    gp = make((24, 20, 64))
    for call in (lambda: gp.set_window(0), lambda: gp.set_axis_window(1, 0),
                 lambda: gp.set_lines_per_thread(0, 1), lambda: gp.set_pair_lines(False),
                 lambda: gp.set_tma(False)):
        with pytest.raises(N.GPError) as e:
            call()
        assert e.value.status == N.GP_ERR_ARG
    gp.init_gaussian()
    with pytest.raises(N.GPError) as e:
        gp.density_profiles()
    assert e.value.status == N.GP_ERR_STATE
    gp.step_imag(2)  # still usable
    gp.close()
    probs = [inputs.sized_box((24, 20, 64), (1.0, 1.2, 1.5), 5.0)]
    with pytest.raises(N.GPError) as e:
        Batch(probs, "f16", "real")
    assert e.value.status == N.GP_ERR_ARG
