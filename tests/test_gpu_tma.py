"""z sweep through TMA tiles: parity with the oracle and with the per-thread
copy form on grids where the rows allow bulk tensor copies (4- or 8-byte
elements, nz * element size a multiple of 16 bytes, lines of at least one
chunk plus the window plus two nodes), including ragged line counts, the
shortest admissible lines and junk in the Dirichlet end nodes."""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu

D = (0.29, 0.26, 0.23)
OMEGA = (1.0, 1.3, 1.8)
# (nx, ny, nz): nz a multiple of 4 so that both 4- and 8-byte elements qualify;
# nx * ny not a multiple of 256 rows (a ragged last block, idle and ragged warps); nz - 2 spanning
# several chunks with a ragged tail, or exactly the shortest admissible line.
SHAPES = [(23, 17, 48), (19, 13, 100), (11, 9, 16), (7, 5, 28), (5, 3, 44)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, prec, field, dt=0.004, g=9.0):
    from paper_1601_04641_gb300.solver import GP
    return GP(shape, D, dt, OMEGA, g, prec, field)


def field_for(shape, prec, field, seed):
    psi = inputs.random_field(shape, seed=seed)
    if field == "real":
        psi = np.abs(psi)
    if prec == "f32":
        psi = psi.astype(np.float32 if field == "real" else np.complex64)
    return psi


def run(shape, prec, field, realtime, window, tma, psi0, steps=3):
    gp = make(shape, prec, field)
    gp.set_tma(tma)
    try:
        gp.set_window(window)
    except N.GPError:
        gp.close()
        return None, None
    gp.set_psi(psi0)
    (gp.step_real if realtime else gp.step_imag)(steps)
    out = gp.get_psi()
    used = gp.tma_in_use()
    gp.close()
    return out, used


CASES = [("f32", "complex", False), ("f32", "complex", True), ("f32", "real", False),
         ("f64", "real", False)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("window", [4, 8, 16])
@pytest.mark.parametrize("prec,field,realtime", CASES)
def test_tma_z_sweep_matches_oracle_and_copy_form(prec, field, realtime, window, shape):
    elem = (4 if prec == "f32" else 8) * (2 if field == "complex" else 1)
    chunk = 64 // elem
    if shape[2] - 2 < chunk + window + 2:
        pytest.skip("line shorter than a chunk plus the window: the copy form runs")
    psi0 = field_for(shape, prec, field, seed=40 + window)
    a, used = run(shape, prec, field, realtime, window, True, psi0)
    if a is None:
        pytest.skip("window %d not admissible here" % window)
    # the TMA form holds (chunk + window) pair values within 256 bytes
    assert used == ((chunk + window) * 2 * elem <= 256)
    b, _ = run(shape, prec, field, realtime, window, False, psi0)
    # same arithmetic per line in both forms
    scale = float(np.max(np.abs(b)))
    assert float(np.max(np.abs(a - b))) <= (1e-14 if prec == "f64" else 1e-6) * scale
    ref = psi0.astype(np.complex128)
    oracle.step(ref, D, 0.004, OMEGA, 9.0, realtime, 3)
    tol = 1e-12 if prec == "f64" else 2e-6
    assert float(np.max(np.abs(a.astype(np.complex128) - ref))) <= tol * float(np.max(np.abs(ref)))


@pytest.mark.parametrize("prec,field", [("f32", "complex"), ("f32", "real"), ("f64", "real")])
def test_tma_ignores_junk_in_the_end_nodes(prec, field):
    """The z sweep neither reads node 0 nor node nz-1 and writes zeros there,
    whatever the input holds (the oracle's reading of the Dirichlet ends)."""
    shape, dt = (13, 11, 40), 0.002  # dt small enough for window 8 in FP64 (the TMA form holds W <= 8 there)
    psi0 = field_for(shape, prec, field, seed=77)
    psi0[:, :, 0] = 3.0
    psi0[:, :, -1] = -2.0
    gp = make(shape, prec, field, dt=dt)
    for w in (4, 8, 16):  # the smallest window admissible in this precision
        try:
            gp.set_window(w)
            break
        except N.GPError:
            continue
    assert gp.tma_in_use()
    gp.set_psi(psi0)
    gp.stage(2, False)
    got = gp.get_psi().astype(np.complex128)
    gp.close()
    ref = psi0.astype(np.complex128)
    oracle.sweep(ref, D, 2, dt, False)
    oracle.renormalize(ref, D)
    assert np.all(got[:, :, 0] == 0) and np.all(got[:, :, -1] == 0)
    tol = 1e-12 if prec == "f64" else 2e-6
    assert float(np.max(np.abs(got - ref))) <= tol * float(np.max(np.abs(ref)))


def test_tma_norm_and_graphs():
    """Norm tracking through the TMA z sweep and graph-replayed blocks give
    the same psi and observables as kernel-by-kernel launches."""
    shape = (21, 19, 64)
    psi0 = field_for(shape, "f32", "complex", seed=3)
    out = []
    for block in (0, 8):
        gp = make(shape, "f32", "complex")
        assert gp.tma_in_use()
        gp.set_graph_block(block)
        gp.set_psi(psi0)
        gp.step_real(20)
        out.append((gp.get_psi(), gp.observables()))
        gp.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1]["norm"] == out[1][1]["norm"]
    ref = psi0.astype(np.complex128)
    oracle.step(ref, D, 0.004, OMEGA, 9.0, True, 20)
    r = oracle.observables(ref, D, OMEGA, 9.0)
    assert abs(out[0][1]["norm"] - r["norm"]) <= 1e-5 * r["norm"]
    assert abs(out[0][1]["energy"] - r["energy"]) <= 1e-5 * abs(r["energy"])
