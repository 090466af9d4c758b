"""The x and y sweeps through TMA boxes (sweep_lines_tma_kernel) against the
per-thread-copy form and the FP64 oracle (GPU only).

- Both forms do the same arithmetic in the same order on the same values,
  so psi after several steps is bit-identical: every precision and form
  (imaginary time on real and complex fields, real time), 1, 2 and 4 lines
  per thread, windows 4, 8 and 16, whole lines and lines cut into segments
  at and off chunk boundaries, odd line lengths.
- The axes that take the TMA form follow the rule: a windowed solve and a
  node stride of whole 16-byte units; the last warp of a plane (x) or of a
  row (y) may be partial (its box columns past the row read the zero fill).
- Junk in the Dirichlet end nodes is never read (the maps start at node 1)
  and zeros are written there: tests/test_gpu_lines.py runs with the TMA
  form on, its default.
"""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu

D = (0.31, 0.27, 0.22)
OMEGA = (1.0, 1.4, 2.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, dt, g, prec, field):
    from paper_1601_04641_gb300.solver import GP
    return GP(shape, D, dt, OMEGA, g, prec, field)


def start_field(shape, prec, field, seed):
    psi = inputs.random_field(shape, seed=seed, complex_=(field == "complex"))
    if field == "real":
        psi = np.abs(psi)
    if prec == "f32":
        psi = psi.astype(np.float32 if field == "real" else np.complex64)
    return psi


def run(shape, prec, field, realtime, tma_axes, window=None, seg=None, lines=None, steps=4, seed=5):
    dt, g = (0.002, 9.0) if realtime else (0.004, 12.0)
    gp = make(shape, dt, g, prec, field)
    gp.set_tma_lines(tma_axes)
    if window is not None:  # the strided axes only (z keeps its own smallest admissible window)
        for ax in (0, 1):
            gp.set_axis_window(ax, window)
    if seg is not None:
        for ax in (0, 1):
            gp.set_segments(ax, seg)
    if lines is not None:
        for ax in (0, 1):
            gp.set_lines_per_thread(ax, lines)
    axes = gp.tma_lines_in_use()
    lpt = gp.lines_per_thread(1 if realtime else 0)
    gp.set_psi(start_field(shape, prec, field, seed))
    if realtime:
        gp.step_real(steps)
    else:
        gp.step_imag(steps)
    out = gp.get_psi()
    gp.close()
    return out, axes, lpt


def expected_axes(shape, elem, window):
    nx, ny, nz = shape
    bits = 0
    for ax, stride in ((0, ny * nz), (1, nz)):
        if window > 0 and (stride * elem) % 16 == 0 and shape[ax] >= 3:
            bits |= 1 << ax
    return bits


# (shape, prec, field, realtime, window, segment override, lines per thread)
CASES = [
    ((20, 18, 64), "f32", "complex", False, None, None, None),   # pairs on x and y
    ((20, 18, 64), "f32", "complex", True, None, None, None),    # real time, pairs
    ((37, 24, 128), "f32", "real", False, None, None, None),     # quads on x and y
    ((37, 24, 128), "f32", "real", False, 16, 24, None),         # quads, segments of 24 (off chunk bounds)
    ((41, 34, 32), "f32", "complex", False, 8, None, None),      # pairs: 16 a row on y (a partial warp per row)
    ((23, 19, 50), "f32", "complex", True, 4, None, None),       # partial warps on x (475 pairs) and y (25 a row)
    ((23, 19, 52), "f32", "real", False, 8, 9, None),            # quads: 13 a row on y, 247 on x; segments of 9
    ((23, 19, 50), "f32", "real", False, 4, None, None),         # node strides of 3800 / 200 bytes: neither axis
    ((41, 33, 32), "f32", "complex", False, 8, None, 1),         # single complex64 lines on both
    ((41, 33, 32), "f32", "real", False, 4, 5, 1),               # single lines, segments of 5
    ((24, 20, 32), "f64", "complex", False, 8, None, None),      # 16-byte elements, one line per thread
    ((24, 20, 32), "f64", "complex", True, 8, 13, None),         # FP64 real time, segments of 13
    ((26, 36, 64), "f64", "real", False, 16, None, 2),           # FP64 real, pairs
    ((150, 18, 64), "f32", "complex", True, 4, None, None),      # x lines of 148 nodes: two segments
]


@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_tma_lines_bit_identical_to_copy_form(case):
    shape, prec, field, realtime, window, seg, lines = case
    on, axes, lpt = run(shape, prec, field, realtime, 3, window, seg, lines)
    off, axes_off, _ = run(shape, prec, field, realtime, 0, window, seg, lines)
    elem = {"f32": 4, "f64": 8}[prec] * (2 if field == "complex" else 1)
    w = window if window is not None else 1  # the FP32 default is windowed
    assert axes == expected_axes(shape, elem, w), (axes, lpt)
    assert axes_off == 0
    assert np.array_equal(on, off), float(np.max(np.abs(on.astype(np.complex128) - off.astype(np.complex128))))


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[5], CASES[10], CASES[11]],
                         ids=["c64", "real", "c64partial", "c128", "c128rt"])
def test_tma_lines_match_oracle(case):
    shape, prec, field, realtime, window, seg, lines = case
    steps = 4
    out, _, _ = run(shape, prec, field, realtime, 3, window, seg, lines, steps=steps)
    dt, g = (0.002, 9.0) if realtime else (0.004, 12.0)
    ref = start_field(shape, prec, field, 5).astype(np.complex128)
    oracle.step(ref, D, dt, OMEGA, g, realtime, steps)
    scale = float(np.max(np.abs(ref)))
    err = float(np.max(np.abs(out.astype(np.complex128) - ref)))
    assert err <= (1e-12 if prec == "f64" else 2e-6) * scale, err


@pytest.mark.parametrize("field", ["real", "complex"])
def test_tma_lines_axis_mask(field):
    """The default reads x through TMA boxes for real fields only; a mask
    selects the axes in both modes; masks outside -1..3 are refused."""
    from paper_1601_04641_gb300 import _native as N
    gp = make((20, 18, 64), 0.004, 12.0, "f32", field)
    default = 1 if field == "real" else 0
    assert gp.tma_lines_in_use() == default
    for m in (0, 1, 2, 3, -1):
        gp.set_tma_lines(m)
        assert gp.tma_lines_in_use() == (default if m == -1 else m)
    for bad in (-2, 4):
        with pytest.raises(N.GPError) as e:
            gp.set_tma_lines(bad)
        assert e.value.status == N.GP_ERR_ARG
    gp.close()
