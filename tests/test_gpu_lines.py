"""Strided line solves with several lines per thread, the Dirichlet end
nodes of the strided axes, and the packed complex64 observables kernel,
against the FP64 oracle on the same seeded inputs (GPU only).

- Four adjacent lines per thread (FP32 real fields, windowed solves): the
  oracle's step within the FP32 bound, and the one-line form's result to
  rounding (the four-line form cuts lines into 8-node chunks, the one-line
  form into 16-node chunks; both windowed solves are exact to roundoff).
- Junk in the end nodes of x and y lines is never read and zeros are
  written there (reading R3 of the boundary).
- The FP32 observables (for real fields the bulk-copy kernel where a plane
  is whole 16-byte units and a stage fits; the other kernels elsewhere)
  agree with the oracle and with the FP64 kernel on the same field, on grids
  that span several tiles or work items with ragged tails.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, d, dt, omega, g, prec="f64", field="complex"):
    from paper_1601_04641_gb300.solver import GP
    return GP(shape, d, dt, omega, g, prec, field)


def real_field(shape, seed):
    return np.abs(inputs.random_field(shape, seed=seed)).astype(np.float32)


# shapes: line counts of both strided axes multiples of 4 (and nz a
# multiple of 4 for the y lines), or not, so that the rule falls back to pairs
@pytest.mark.parametrize("shape,quad", [((36, 30, 44), (4, 4)), ((41, 28, 36), (4, 4)),
                                        ((37, 30, 42), (4, 2)), ((33, 29, 40), (4, 4)),
                                        ((20, 27, 34), (2, 2)), ((21, 27, 35), (1, 1))])
@pytest.mark.parametrize("window", [4, 8, 16])
def test_four_lines_per_thread_match_oracle(shape, quad, window):
    dt, g = 0.004, 12.0
    psi0 = real_field(shape, seed=60 + window)
    out = {}
    for lpt in (4, 1):
        gp = make(shape, D, dt, OMEGA, g, "f32", "real")
        gp.set_window(window)
        for ax in (0, 1):
            gp.set_lines_per_thread(ax, lpt)
        used = gp.lines_per_thread(0)
        gp.set_psi(psi0)
        gp.step_imag(3)
        out[lpt] = gp.get_psi().astype(np.float64)
        gp.close()
        if lpt == 4:
            assert used[:2] == quad and used[2] == 1, used
        else:
            assert used == (1, 1, 1)
    ref = psi0.astype(np.complex128)
    oracle.step(ref, D, dt, OMEGA, g, False, 3)
    scale = float(np.max(np.abs(ref)))
    assert float(np.max(np.abs(out[4] - ref))) <= 2e-6 * scale
    assert float(np.max(np.abs(out[4] - out[1]))) <= 1e-6 * scale


def test_lines_per_thread_arguments():
    gp = make((12, 12, 12), D, 0.004, OMEGA, 1.0, "f32", "real")
    for bad_axis, bad_lines in ((2, 4), (0, 3), (1, 8), (-1, 1)):
        with pytest.raises(N.GPError) as e:
            gp.set_lines_per_thread(bad_axis, bad_lines)
        assert e.value.status == N.GP_ERR_ARG
    gp.set_pair_lines(False)
    assert gp.lines_per_thread(0) == (1, 1, 1)
    gp.set_pair_lines(True)
    assert gp.lines_per_thread(0) == (4, 4, 1)
    gp.close()


@pytest.mark.parametrize("prec,field,realtime", [("f32", "complex", False), ("f32", "complex", True),
                                                 ("f32", "real", False), ("f64", "complex", True),
                                                 ("f64", "real", False)])
@pytest.mark.parametrize("stage", [0, 1])
def test_strided_sweeps_ignore_junk_in_the_end_nodes(prec, field, realtime, stage):
    """The x and y sweeps neither read node 0 nor node N-1 of their lines
    and write zeros there, whatever the input holds (the TMA z sweep has its
    own test)."""
    shape, dt, g = (28, 24, 20), 0.004, 9.0
    psi0 = inputs.random_field(shape, seed=81 + stage)
    if field == "real":
        psi0 = np.abs(psi0)
    if prec == "f32":
        psi0 = psi0.astype(np.float32 if field == "real" else np.complex64)
    junk = psi0.copy()
    sl = [slice(None)] * 3
    for end, val in ((0, 3.0), (-1, -2.5)):
        sl[stage] = end
        junk[tuple(sl)] = val
    gp = make(shape, D, dt, OMEGA, g, prec, field)
    gp.set_psi(junk)
    gp.stage(stage, realtime)
    got = gp.get_psi().astype(np.complex128)
    gp.close()
    ref = psi0.astype(np.complex128)
    if stage == 0:
        oracle.kick(ref, D, dt, OMEGA, g, realtime)
    oracle.sweep(ref, D, stage, dt, realtime)
    for end in (0, -1):
        sl[stage] = end
        assert np.all(got[tuple(sl)] == 0)
    tol = 1e-13 if prec == "f64" else 2e-6
    assert float(np.max(np.abs(got - ref))) <= tol * float(np.max(np.abs(ref)))


# nz even: the packed kernel; (nx, ny*nz/2) spanning several 32-plane x
# 256-pair work items with ragged tails; one grid with nz odd (the other kernel)
@pytest.mark.parametrize("shape", [(70, 33, 50), (40, 31, 64), (9, 5, 6), (37, 29, 41)])
def test_observables_complex64_match_oracle_and_fp64(shape):
    psi0 = inputs.random_field(shape, seed=4).astype(np.complex64)
    ref = oracle.observables(psi0.astype(np.complex128), D, OMEGA, 25.0)
    got = {}
    for prec in ("f32", "f64"):
        gp = make(shape, D, 0.01, OMEGA, 25.0, prec)
        gp.set_psi(psi0 if prec == "f32" else psi0.astype(np.complex128))
        got[prec] = gp.observables()
        gp.close()
    for k in OBS:
        assert abs(got["f64"][k] - ref[k]) <= 1e-12 * abs(ref[k]), (k, got["f64"][k], ref[k])
        assert abs(got["f32"][k] - ref[k]) <= 1e-6 * abs(ref[k]), (k, got["f32"][k], ref[k])


# FP32 real fields through the bulk-copy kernel (planes of whole 16-byte
# units, a stage of tile + nz + 1 sites within 12 KB): tiles of 1024 sites,
# several tiles with a ragged last one, planes smaller than a tile, runs of
# planes that start inside a column, nz at the stage limit (2046); shapes
# just past the limit or with planes that are not whole 16-byte units (the
# per-(j, k) kernel); complex64 grids (the packed and per-(j, k) kernels)
@pytest.mark.parametrize("field,shape", [
    ("complex", (70, 33, 50)), ("complex", (9, 5, 6)), ("complex", (5, 3, 510)),
    ("complex", (5, 3, 512)), ("complex", (23, 45, 47)),
    ("real", (70, 36, 50)), ("real", (33, 52, 84)), ("real", (4, 4, 2046)),
    ("real", (4, 4, 2048)), ("real", (41, 27, 37)), ("real", (6, 6, 1030))])
def test_observables_fp32_match_oracle(field, shape):
    psi0 = inputs.random_field(shape, seed=14, complex_=(field == "complex"))
    psi32 = psi0.astype(np.complex64 if field == "complex" else np.float32)
    ref = oracle.observables(psi32.astype(np.complex128), D, OMEGA, 25.0)
    gp = make(shape, D, 0.01, OMEGA, 25.0, "f32", field)
    gp.set_psi(psi32)
    got = gp.observables()
    gp.close()
    for k in OBS:
        assert abs(got[k] - ref[k]) <= 1e-6 * abs(ref[k]), (k, got[k], ref[k])


def test_observables_complex64_with_pending_scale():
    """After an imaginary-time step the renormalisation factor is pending:
    the packed kernel applies it (s^2 to the quadratic sums, s^4 to |psi|^4)."""
    shape, d, dt, g = (48, 34, 40), (0.3, 0.3, 0.3), 0.01, 30.0
    psi0 = inputs.random_field(shape, seed=9).astype(np.complex64)
    gp = make(shape, d, dt, OMEGA, g, "f32")
    gp.set_psi(psi0)
    gp.step_imag(2)
    o = gp.observables()
    psi = gp.get_psi().astype(np.complex128)
    gp.close()
    r = oracle.observables(psi, d, OMEGA, g)
    for k in OBS:
        assert abs(o[k] - r[k]) <= 1e-6 * abs(r[k]), (k, o[k], r[k])
