"""gp_observables_noalloc against the handle-based gp_observables and the
FP64 oracle (GPU).

The no-allocation entry point is for callers that cannot call cudaMalloc --
a framework that owns all device memory through its own pool, or a loop that
must not pay cudaMalloc's implicit device synchronisation.  Its reduction
scratch is one fixed static device array shared by every call, so the test
makes two calls in a row on the same data and checks both, which also shows
that the scratch left by the first call does not leak into the second, and
that the device's free memory is the same before and after them.

The file name sorts last so that a run stopping at its first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu

KEYS = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("prec,field", [("f64", "complex"), ("f32", "complex"), ("f64", "real"),
                                        ("f32", "real")])
def test_noalloc_matches_handle_observables_on_two_calls(prec, field):
    import torch
    from paper_1601_04641_gb300.solver import GP
    shape, d, omega, g = (37, 29, 41), (0.31, 0.27, 0.22), (1.0, 1.4, 2.0), 25.0
    psi0 = inputs.random_field(shape, seed=3, complex_=(field == "complex"))
    gp = GP(shape, d, 0.01, omega, g, prec, field)
    gp.set_psi(psi0.astype(gp.np_dtype))
    ref = gp.observables()

    # the oracle on the values the field holds (rounded to its precision)
    ref_o = oracle.observables(psi0.astype(gp.np_dtype).astype(np.complex128), d, omega, g)

    ptr, pending = ctypes.c_void_p(), ctypes.c_int(0)
    assert gp.lib.gp_psi_device_ptr(gp.h, ctypes.byref(ptr), ctypes.byref(pending)) == N.GP_OK
    assert pending.value == 0
    out = torch.zeros(16, dtype=torch.float64, device=gp.device)  # the caller's output buffer
    grid = N.Grid(*shape, *d)
    codes = (N.GP_F64 if prec == "f64" else N.GP_F32, N.GP_COMPLEX if field == "complex" else N.GP_REAL)
    stream = ctypes.c_void_p(gp.stream.cuda_stream)
    # a first call may load the library's module holding the static array
    assert gp.lib.gp_observables_noalloc(ptr, grid, codes[0], codes[1], *omega, g, 1.0,
                                         ctypes.c_void_p(out.data_ptr()), stream) == N.GP_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(gp.device)[0]
    for _ in range(2):
        out.fill_(-1.0)
        st = gp.lib.gp_observables_noalloc(ptr, grid, codes[0], codes[1], *omega, g, 1.0,
                                           ctypes.c_void_p(out.data_ptr()), stream)
        assert st == N.GP_OK, gp.lib.gp_last_error(None)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[15] == 1.0
        # FP64: the same sums; FP32: the same compensated sums grouped
        # differently (the handle path sums chunks of 8 sites per segment of x)
        tol = 1e-12 if prec == "f64" else 1e-6
        for key, v in zip(KEYS, o[9:15]):
            assert abs(v - ref[key]) <= tol * abs(ref[key]), (key, v, ref[key])
            assert abs(v - ref_o[key]) <= tol * abs(ref_o[key]), (key, v, ref_o[key])
    assert torch.cuda.mem_get_info(gp.device)[0] == free_before  # nothing allocated

    # the read scale multiplies psi: the norm grows by its square, mu does not
    out.fill_(-1.0)
    st = gp.lib.gp_observables_noalloc(ptr, grid, codes[0], codes[1], *omega, 0.0, 2.0,
                                       ctypes.c_void_p(out.data_ptr()), stream)
    assert st == N.GP_OK
    torch.cuda.synchronize()
    assert abs(out[9].item() - 4.0 * ref["norm"]) <= tol * 4.0 * ref["norm"]
    gp.close()


def test_noalloc_rejects_planes_beyond_its_scratch():
    import torch
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    psi = torch.zeros(8, dtype=torch.complex128, device="cuda")
    grid = N.Grid(3, 2048, 1025, 0.1, 0.1, 0.1)  # ny * nz = 2,099,200 > 2,097,152
    lib = N.load()
    st = lib.gp_observables_noalloc(ctypes.c_void_p(psi.data_ptr()), grid, N.GP_F64, N.GP_COMPLEX,
                                    1.0, 1.0, 1.0, 1.0, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == N.GP_ERR_ARG
    assert b"no-allocation limit" in lib.gp_last_error(None)
    assert torch.all(out == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_with_the_pending_factor_after_imaginary_time(prec):
    """After imaginary-time steps the handle's buffer holds psi times a
    pending renormalisation factor: passing gp_pending_scale's factor as the
    read scale gives the handle's observables and the oracle's on the
    settled psi (the |psi|^4 term scales as the factor to the fourth)."""
    import torch
    from paper_1601_04641_gb300.solver import GP
    shape, d, omega, g = (30, 26, 24), (0.3, 0.3, 0.3), (1.0, 1.4, 2.0), 40.0
    psi0 = inputs.random_field(shape, seed=8)
    gp = GP(shape, d, 0.01, omega, g, prec, "complex")
    gp.set_psi(psi0.astype(gp.np_dtype))
    gp.step_imag(3)
    ptr, pending, scale = ctypes.c_void_p(), ctypes.c_int(0), ctypes.c_double(0.0)
    assert gp.lib.gp_psi_device_ptr(gp.h, ctypes.byref(ptr), ctypes.byref(pending)) == N.GP_OK
    assert gp.lib.gp_pending_scale(gp.h, ctypes.byref(scale)) == N.GP_OK
    assert pending.value == 1 and abs(scale.value - 1.0) > 1e-6
    out = torch.zeros(16, dtype=torch.float64, device=gp.device)
    st = gp.lib.gp_observables_noalloc(ptr, N.Grid(*shape, *d), N.GP_F64 if prec == "f64" else N.GP_F32,
                                       N.GP_COMPLEX, *omega, g, scale.value, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(gp.stream.cuda_stream))
    assert st == N.GP_OK, gp.lib.gp_last_error(None)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    ref = gp.observables()
    settled = oracle.observables(gp.get_psi().astype(np.complex128), d, omega, g)
    gp.close()
    tol = 1e-12 if prec == "f64" else 1e-6
    for key, v in zip(KEYS, o[9:15]):
        assert abs(v - ref[key]) <= tol * abs(ref[key]), (key, v, ref[key])
        assert abs(v - settled[key]) <= (tol if prec == "f64" else 1e-6) * abs(settled[key]), key
