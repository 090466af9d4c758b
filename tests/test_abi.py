"""C ABI checks that need no GPU: libgpcn.so builds for sm_103a, loads, exports
every function include/gp.h declares, and rejects bad arguments on the host
before touching CUDA."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1601_04641_gb300 import _native as N
from paper_1601_04641_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return N.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gp_create", "gp_step_imag", "gp_step_real", "gp_observables"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(gp_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for name in declared_functions():
        getattr(lib, name)


def test_binding_declares_exactly_the_header():
    assert sorted(N.SIGNATURES) == declared_functions()


def _create(lib, **kw):
    args = dict(nx=8, ny=8, nz=8, dx=0.1, dy=0.1, dz=0.1, dt=1e-3, gamma=1.0, nu=1.0, lam=1.0,
                g=1.0, prec=N.GP_F64, field=N.GP_COMPLEX)
    args.update(kw)
    h = N.Handle()
    grid = N.Grid(args["nx"], args["ny"], args["nz"], args["dx"], args["dy"], args["dz"])
    st = lib.gp_create(ctypes.byref(h), grid, args["dt"], args["gamma"], args["nu"], args["lam"],
                       args["g"], args["prec"], args["field"], None)
    return st, h


@pytest.mark.parametrize("bad", [dict(nx=2), dict(nz=0), dict(dx=0.0), dict(dy=-1.0),
                                 dict(dz=float("nan")), dict(dt=0.0), dict(dt=float("inf")),
                                 dict(gamma=-1.0), dict(nu=float("nan")), dict(g=float("inf")),
                                 dict(prec=7), dict(field=9)])
def test_bad_arguments_are_rejected_on_the_host(lib, bad):
    st, h = _create(lib, **bad)
    assert st == N.GP_ERR_ARG
    assert not h.value
    assert lib.gp_last_error(None)


def test_null_handle_and_out_pointers(lib):
    assert lib.gp_step_imag(None, 1) == N.GP_ERR_ARG
    assert lib.gp_observables(None, None) == N.GP_ERR_ARG
    grid = N.Grid(8, 8, 8, 0.1, 0.1, 0.1)
    assert lib.gp_create(None, grid, 1e-3, 1.0, 1.0, 1.0, 1.0, 0, 0, None) == N.GP_ERR_ARG
    lib.gp_destroy(None)
    assert b"sm_103a" in lib.gp_version()


def test_valid_create_without_gpu_reports_cuda_error(lib):
    """Valid arguments reach CUDA; with no device that is GP_ERR_CUDA, not a crash."""
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    st, h = _create(lib)
    if has_gpu:
        assert st == N.GP_OK
        lib.gp_destroy(h)
    else:
        assert st in (N.GP_ERR_CUDA, N.GP_ERR_NOMEM)


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.parametrize("nz, field", [(64, N.GP_COMPLEX), (60, N.GP_REAL), (48, N.GP_REAL)])
def test_fp16_storage_refusals_on_the_host(lib, nz, field):
    """FP16 storage holds real fields only, on z rows of whole 16-byte units
    (nz a multiple of 8) long enough for a chunk and the widest window."""
    st, h = _create(lib, nz=nz, prec=N.GP_F16, field=field)
    assert st == N.GP_ERR_ARG
    assert not h.value
    assert lib.gp_last_error(None)


def test_fp16_storage_valid_arguments_pass_the_host_checks(lib):
    st, h = _create(lib, nz=64, prec=N.GP_F16, field=N.GP_REAL)
    if _has_gpu():
        assert st == N.GP_OK
        lib.gp_destroy(h)
    else:
        assert st in (N.GP_ERR_CUDA, N.GP_ERR_NOMEM)


def _axial_create(lib, **kw):
    args = dict(nx=16, nz=24, drho=0.2, dz=0.2, dt=1e-3, gamma=1.0, lam=2.0, g=5.0,
                prec=N.GP_F64, field=N.GP_COMPLEX)
    args.update(kw)
    h = N.Handle()
    st = lib.gp_axial_create(ctypes.byref(h), args["nx"], args["nz"], args["drho"], args["dz"], args["dt"],
                             args["gamma"], args["lam"], args["g"], args["prec"], args["field"], None)
    return st, h


@pytest.mark.parametrize("bad", [dict(nx=2), dict(nz=2), dict(drho=0.0), dict(dz=-0.1),
                                 dict(dt=float("nan")), dict(gamma=0.0), dict(lam=float("inf")),
                                 dict(g=float("nan")), dict(prec=N.GP_F16), dict(prec=5), dict(field=3)])
def test_axial_bad_arguments_are_rejected_on_the_host(lib, bad):
    st, h = _axial_create(lib, **bad)
    assert st == N.GP_ERR_ARG
    assert not h.value
    assert lib.gp_axial_last_error(None)


def test_axial_null_handle_and_out_pointers(lib):
    grid_args = (16, 24, 0.2, 0.2, 1e-3, 1.0, 2.0, 5.0, N.GP_F64, N.GP_COMPLEX, None)
    assert lib.gp_axial_create(None, *grid_args) == N.GP_ERR_ARG
    for call in (lambda: lib.gp_axial_init_gaussian(None),
                 lambda: lib.gp_axial_set_psi(None, None, 0),
                 lambda: lib.gp_axial_get_psi(None, None, 0),
                 lambda: lib.gp_axial_step_imag(None, 1),
                 lambda: lib.gp_axial_step_real(None, 1),
                 lambda: lib.gp_axial_observables(None, None),
                 lambda: lib.gp_axial_run_imag_until(None, 1e-6, 10, 100, None)):
        assert call() == N.GP_ERR_ARG
    lib.gp_axial_destroy(None)
    assert b"NULL" in lib.gp_axial_last_error(None)


def test_axial_valid_create_without_gpu_reports_cuda_error(lib):
    st, h = _axial_create(lib)
    if _has_gpu():
        assert st == N.GP_OK
        lib.gp_axial_destroy(h)
    else:
        assert st == N.GP_ERR_CUDA
        assert not h.value


C_CLIENT = r"""
#include <stdio.h>
#include "gp.h"
int main(void) {
    gp_handle h = 0;
    gp_grid grid = {48, 40, 32, 0.1, 0.1, 0.1};
    gp_status st = gp_create(&h, grid, 1e-3, 0.5, 1.0, 1.5, 20.0, GP_F32, GP_COMPLEX, NULL);
    gp_axial a = 0;
    gp_status sa = gp_axial_create(&a, 16, 24, 0.2, 0.2, 1e-3, 1.0, 2.0, 5.0, GP_F64, GP_REAL, NULL);
    gp_status bad = gp_create(&h, grid, -1.0, 0.5, 1.0, 1.5, 20.0, GP_F32, GP_COMPLEX, NULL);
    if (st == GP_OK) gp_destroy(h);
    if (sa == GP_OK) gp_axial_destroy(a);
    printf("%d %d %d\n", (int)st, (int)sa, (int)bad);
    return 0;
}
"""


def test_header_is_plain_c_and_links(tmp_path):
    """A C99 client (pedantic, warnings as errors) includes gp.h, links
    libgpcn.so and gets statuses back (no GPU here: GP_ERR_CUDA)."""
    build.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(N.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lgpcn",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split()
    st, sa, bad = (int(x) for x in out)
    assert bad == N.GP_ERR_ARG
    if _has_gpu():
        assert st == N.GP_OK and sa == N.GP_OK
    else:
        assert st == N.GP_ERR_CUDA and sa == N.GP_ERR_CUDA


def test_last_error_without_handle_is_per_thread(lib):
    """gp_last_error(NULL) reports the calling thread's last failure: two
    threads failing with different messages at the same time each read back
    their own (ctypes releases the interpreter lock during the calls)."""
    import threading
    cases = {"dt": dict(dt=-1.0), "spacing": dict(dx=0.0)}
    wrong = []
    barrier = threading.Barrier(len(cases))

    def worker(key):
        barrier.wait()
        for _ in range(2000):
            st, _ = _create(lib, **cases[key])
            msg = lib.gp_last_error(None).decode()
            if st != N.GP_ERR_ARG or key not in msg:
                wrong.append((key, st, msg))
                return

    threads = [threading.Thread(target=worker, args=(k,)) for k in cases]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not wrong, wrong[:3]


def _batch_create(lib, n=3, bad=None, prec=N.GP_F32, field=N.GP_COMPLEX):
    """gp_batch_create on n small instances; `bad` = (instance, key, value)
    overrides one parameter of one instance."""
    grids = (N.Grid * n)(*[N.Grid(12 + i, 10, 9, 0.2, 0.2, 0.25) for i in range(n)])
    arr = {k: [v] * n for k, v in dict(dt=1e-3, gamma=1.0, nu=1.2, lam=1.5, g=5.0).items()}
    if bad:
        i, key, value = bad
        if key in arr:
            arr[key][i] = value
        else:
            setattr(grids[i], key, value)
    c = {k: (ctypes.c_double * n)(*v) for k, v in arr.items()}
    h = N.Handle()
    st = lib.gp_batch_create(ctypes.byref(h), n, grids, c["dt"], c["gamma"], c["nu"], c["lam"], c["g"],
                             prec, field, None)
    return st, h


@pytest.mark.parametrize("bad", [(0, "nx", 2), (2, "nz", 1), (1, "dy", 0.0), (2, "dz", float("nan")),
                                 (1, "dt", -1e-3), (0, "g", float("inf")), (2, "gamma", -1.0),
                                 (1, "lam", float("nan"))])
def test_batch_bad_instance_is_rejected_on_the_host(lib, bad):
    st, h = _batch_create(lib, bad=bad)
    assert st == N.GP_ERR_ARG
    assert not h.value
    assert ("instance %d" % bad[0]).encode() in lib.gp_batch_last_error(None)


def test_batch_refusals_and_valid_create_without_gpu(lib):
    for kw in (dict(prec=N.GP_F16), dict(prec=9), dict(field=4), dict(n=0)):
        st, h = _batch_create(lib, **kw)
        assert st == N.GP_ERR_ARG and not h.value, kw
    st, h = _batch_create(lib)
    if _has_gpu():
        assert st == N.GP_OK
        lib.gp_batch_destroy(h)
    else:
        assert st == N.GP_ERR_CUDA and not h.value
