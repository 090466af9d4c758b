"""Failure detection without a GPU fault: the bounded device wait gives up and
reports (a wait that nothing can satisfy, a short bound, nothing copied);
an expired wait's status word, raised from the host, is reported and makes
psi unusable until it is set again; allocation failures made on the host
return GP_ERR_NOMEM and leave no device memory behind; odd line lengths
(3, 5, 33, 127) against the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_bounded_wait_gives_up_and_reports():
    import torch
    lib = N.load()
    done, expired = ctypes.c_int(-1), ctypes.c_int(-1)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.gp_selftest_bounded_wait(1 << 20, ctypes.c_void_p(stream), ctypes.byref(done), ctypes.byref(expired))
    assert st == N.GP_OK, lib.gp_last_error(None)
    assert done.value == 1 and expired.value == 1
    # the context is still usable
    from paper_1601_04641_gb300.solver import GP
    gp = GP((12, 10, 16), (0.3, 0.3, 0.3), 0.01, (1, 1, 1), 1.0, "f32", "complex")
    gp.init_gaussian()
    gp.step_imag(5)
    assert abs(gp.observables()["norm"] - 1.0) < 1e-5
    gp.close()
    assert lib.gp_selftest_bounded_wait(0, None, ctypes.byref(done), ctypes.byref(expired)) == N.GP_ERR_ARG


def test_reported_timeout_loses_psi_until_it_is_set_again():
    from paper_1601_04641_gb300.solver import GP
    gp = GP((16, 14, 32), (0.3, 0.3, 0.3), 0.01, (1, 1, 1), 1.0, "f32", "complex")
    gp.init_gaussian()
    gp.step_imag(2)
    assert gp.lib.gp_debug_raise_status(gp.h, 1) == N.GP_OK
    with pytest.raises(N.GPError) as e:
        gp.sync()
    assert e.value.status == N.GP_ERR_TIMEOUT
    for call in (lambda: gp.step_imag(1), gp.observables, gp.get_psi, lambda: gp.run_imag_until(1e-6, 10, 20)):
        with pytest.raises(N.GPError) as e:
            call()
        assert e.value.status == N.GP_ERR_STATE
    gp.init_gaussian()  # psi set again: usable
    gp.step_imag(3)
    assert abs(gp.observables()["norm"] - 1.0) < 1e-5
    gp.close()


def test_reported_observables_timeout_keeps_psi():
    """An expired wait of the observables kernel (status 2) invalidates that
    call's observables only: psi stays usable and the next call succeeds."""
    from paper_1601_04641_gb300.solver import GP
    gp = GP((16, 14, 32), (0.3, 0.3, 0.3), 0.01, (1, 1, 1), 1.0, "f32", "complex")
    gp.init_gaussian()
    gp.step_imag(2)
    ref = gp.observables()
    for bad in (0, 4, 7):
        with pytest.raises(N.GPError) as e:
            N.check(gp.lib.gp_debug_raise_status(gp.h, bad), gp.h)
        assert e.value.status == N.GP_ERR_ARG
    assert gp.lib.gp_debug_raise_status(gp.h, 2) == N.GP_OK
    with pytest.raises(N.GPError) as e:
        gp.observables()
    assert e.value.status == N.GP_ERR_TIMEOUT
    again = gp.observables()
    assert again["mu"] == ref["mu"] and again["norm"] == ref["norm"]
    gp.step_imag(1)
    gp.get_psi()
    gp.close()


def _creates():
    from paper_1601_04641_gb300.solver import GP, Batch
    from paper_1601_04641_gb300.warmstart import Net
    ps = inputs.batch_problems(3, seed=3)
    ps = [inputs.sized_box((20, 16, 12), p.omega, p.g) for p in ps]
    return {
        "handle": lambda: GP((20, 18, 16), (0.3, 0.3, 0.3), 0.01, (1, 1, 1), 1.0, "f32", "complex"),
        "batch": lambda: Batch(ps, "f32", "real"),
        "net": lambda: Net(seed=1),
    }


@pytest.mark.parametrize("kind", ["handle", "batch", "net"])
def test_allocation_failures_return_nomem_and_free_everything(kind):
    import torch
    lib = N.load()
    make = _creates()[kind]
    obj = make()  # warm up: lazily loaded modules, first-use allocations
    obj.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 40):
        lib.gp_debug_fail_alloc(k)
        try:
            obj = make()
        except N.GPError as e:
            assert e.status == N.GP_ERR_NOMEM, str(e)
            failures += 1
            continue
        finally:
            lib.gp_debug_fail_alloc(0)
        obj.close()  # k exceeded the allocations of one create: it succeeded
        break
    else:
        pytest.fail("a create still failed after 39 allocations")
    assert failures >= 4
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 8 << 20


@pytest.mark.parametrize("shape", [(33, 5, 127), (127, 3, 33), (5, 127, 3)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_odd_line_lengths(shape, prec):
    from paper_1601_04641_gb300.solver import GP
    d, omega, g, dt = (0.21, 0.27, 0.19), (1.2, 0.9, 1.6), 6.0, 0.003
    psi0 = inputs.random_field(shape, seed=17)
    for realtime in (False, True):
        gp = GP(shape, d, dt, omega, g, prec, "complex")
        gp.set_psi(psi0.astype(gp.np_dtype))
        (gp.step_real if realtime else gp.step_imag)(4)
        got = gp.get_psi().astype(np.complex128)
        gp.close()
        ref = psi0.astype(np.complex64).astype(np.complex128) if prec == "f32" else psi0.copy()
        oracle.step(ref, d, dt, omega, g, realtime, 4)
        tol = 1e-12 if prec == "f64" else 4e-6
        assert float(np.max(np.abs(got - ref))) <= tol * float(np.max(np.abs(ref))), (shape, prec, realtime)
