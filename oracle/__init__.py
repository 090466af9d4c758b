"""FP64 CPU oracle for the split-step Crank-Nicolson Gross-Pitaevskii step.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the package smoke
check and the benchmark's CPU-baseline leg may import this module.  It wraps
``gp_oracle.c`` (plain C, FP64, textbook Thomas solves over the whole grid in
the method's order) with numpy arrays; it shares no code with the CUDA path.

Arrays are complex128 with shape ``(nx, ny, nz)`` in C order, i.e. z has
stride 1, y stride nz and x stride ny*nz (the paper's "Summary of revisions"
layout of the psi array).  ``d`` is ``(dx, dy, dz)`` and ``omega`` is
``(gamma, nu, lambda)``.

Every function here is pinned by ``tests/test_oracle_pins.py`` against things
other than itself: dense LU solves, the separable g = 0 fixed point, the
continuum and Thomas-Fermi limits, the virial relation, unitarity in real
time, and the O(dt) energy drift of first-order splitting.

The ``axial_*`` functions are the axially symmetric (rho, z) variant
(reading R21 in gp_oracle.c): arrays of shape ``(nx, nz)``, radial node i at
rho = (i - 1/2) drho with node 0 a ghost and node nx-1 the boundary.  They are
pinned by ``tests/test_oracle_axial.py``: the g = 0 continuum limit at second
order, conservation of the cylindrical norm in real time, the virial
relation, and the 3D Cartesian oracle's mu for gamma = nu.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgporacle.so")
_OMP_PATH = os.path.join(_HERE, "libgporacle_omp.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _compile(out_path: str, extra, force: bool) -> str:
    if force or not os.path.exists(out_path) or (
            os.path.getmtime(out_path) < os.path.getmtime(_SRC)):
        tmp = out_path + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared"] + list(extra) + [
            _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile ``gp_oracle.c`` into ``libgporacle.so`` next to it (gcc, no
    fused multiply-add contraction so x86 and Arm give the same bits)."""
    return _compile(_LIB_PATH, [], force)


def build_openmp(force: bool = False) -> str:
    """The same source built with -fopenmp into ``libgporacle_omp.so``: the
    kick's sites and the sweeps' lines are shared out over the host cores
    (OMP_NUM_THREADS), each computed exactly as in the serial build; every
    sum stays serial.  Use it through ``use_library``."""
    return _compile(_OMP_PATH, ["-fopenmp"], force)


_AXIAL = ("oracle_axial_gaussian", "oracle_axial_kick", "oracle_axial_sweep", "oracle_axial_step",
          "oracle_axial_observables")


def _set_axial_types(lib):
    _i, _d = ctypes.c_int, ctypes.c_double
    lib.oracle_axial_gaussian.argtypes = [_i, _i, _d, _d, _d, _d, _dp]
    lib.oracle_axial_kick.argtypes = [_i, _i, _d, _d, _dp, _d, _d, _d, _d, _i]
    lib.oracle_axial_sweep.argtypes = [_i, _i, _d, _d, _dp, _i, _d, _i]
    lib.oracle_axial_step.argtypes = [_i, _i, _d, _d, _dp, _d, _d, _d, _d, _i, _i]
    lib.oracle_axial_observables.argtypes = [_i, _i, _d, _d, _dp, _d, _d, _d, _dp]
    for name in _AXIAL:
        getattr(lib, name).restype = ctypes.c_int


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_thomas.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
            lib.oracle_gaussian.argtypes = [_ip, _dp, _dp, _dp]
            lib.oracle_kick.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp,
                                        ctypes.c_double, ctypes.c_int]
            lib.oracle_sweep.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int]
            lib.oracle_renormalize.argtypes = [_ip, _dp, _dp]
            lib.oracle_step.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int]
            lib.oracle_observables.argtypes = [_ip, _dp, _dp, _dp, ctypes.c_double, _dp]
            lib.oracle_step_strang.argtypes = [_ip, _dp, _dp, ctypes.c_double, _dp, ctypes.c_double,
                                               ctypes.c_int]
            _set_axial_types(lib)
            for f in (lib.oracle_thomas, lib.oracle_gaussian, lib.oracle_kick,
                      lib.oracle_sweep, lib.oracle_renormalize, lib.oracle_step,
                      lib.oracle_observables, lib.oracle_step_strang):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


class use_library:
    """Context manager that points this module at another build of the oracle
    (used by the mutation test, which compiles copies with planted mistakes)."""

    def __init__(self, path):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved = _lib
            lib = ctypes.CDLL(self.path)
            for name in ("oracle_thomas", "oracle_gaussian", "oracle_kick", "oracle_sweep",
                         "oracle_renormalize", "oracle_step", "oracle_observables", "oracle_step_strang") + _AXIAL:
                getattr(lib, name).argtypes = getattr(self.saved, name).argtypes
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile C source text with the oracle's flags into ``out_path``."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    src, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ints(v):
    a = (ctypes.c_int * 3)(*[int(x) for x in v])
    return ctypes.cast(a, _ip), a


def _dbls(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    return a.ctypes.data_as(_dp), a


def _field(psi: np.ndarray) -> np.ndarray:
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.ndim != 3:
        raise TypeError("oracle fields are C-contiguous complex128 arrays of shape (nx, ny, nz)")
    return psi


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def thomas(sub, diag, sup, rhs) -> np.ndarray:
    """Textbook Thomas solve of sub[m] x[m-1] + diag[m] x[m] + sup[m] x[m+1] = rhs[m]."""
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.complex128)) for a in (sub, diag, sup, rhs)]
    n = arrs[3].shape[0]
    x = np.zeros(n, dtype=np.complex128)
    ptrs = [a.ctypes.data_as(_dp) for a in arrs]
    _check(_load().oracle_thomas(n, *ptrs, x.ctypes.data_as(_dp)), "thomas")
    return x


def gaussian(shape, d, omega) -> np.ndarray:
    """Normalised product-Gaussian initial state, zero on the boundary."""
    psi = np.zeros(tuple(int(s) for s in shape), dtype=np.complex128)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    po, _c = _dbls(omega)
    _check(_load().oracle_gaussian(pn, pd, po, psi.ctypes.data_as(_dp)), "gaussian")
    return psi


def kick(psi, d, dt, omega, g, realtime) -> np.ndarray:
    """In-place potential-plus-nonlinear step (calcnu)."""
    psi = _field(psi)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    po, _c = _dbls(omega)
    _check(_load().oracle_kick(pn, pd, psi.ctypes.data_as(_dp), float(dt), po, float(g),
                               int(bool(realtime))), "kick")
    return psi


def sweep(psi, d, axis, dt, realtime) -> np.ndarray:
    """In-place CN line solve along ``axis`` (0 = x, 1 = y, 2 = z)."""
    psi = _field(psi)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    _check(_load().oracle_sweep(pn, pd, psi.ctypes.data_as(_dp), int(axis), float(dt),
                                int(bool(realtime))), "sweep")
    return psi


def renormalize(psi, d) -> np.ndarray:
    psi = _field(psi)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    _check(_load().oracle_renormalize(pn, pd, psi.ctypes.data_as(_dp)), "renormalize")
    return psi


def step(psi, d, dt, omega, g, realtime, nsteps=1) -> np.ndarray:
    """In-place ``nsteps`` split-step CN steps (kick, x, y, z [, renorm])."""
    psi = _field(psi)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    po, _c = _dbls(omega)
    _check(_load().oracle_step(pn, pd, psi.ctypes.data_as(_dp), float(dt), po, float(g),
                               int(bool(realtime)), int(nsteps)), "step")
    return psi


def step_strang(psi, d, dt, omega, g, nsteps=1) -> np.ndarray:
    """In-place ``nsteps`` real-time steps with symmetric splitting: half
    kick, x, y, z line solves, half kick (reading R17)."""
    psi = _field(psi)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    po, _c = _dbls(omega)
    _check(_load().oracle_step_strang(pn, pd, psi.ctypes.data_as(_dp), float(dt), po, float(g), int(nsteps)),
           "step_strang")
    return psi


OBS_KEYS = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z")


def observables(psi, d, omega, g) -> dict:
    """Norm, chemical potential, energy and rms radii (calcmuen, calcrms)."""
    psi = _field(psi)
    pn, _a = _ints(psi.shape)
    pd, _b = _dbls(d)
    po, _c = _dbls(omega)
    out = np.zeros(6, dtype=np.float64)
    _check(_load().oracle_observables(pn, pd, psi.ctypes.data_as(_dp), po, float(g),
                                      out.ctypes.data_as(_dp)), "observables")
    return dict(zip(OBS_KEYS, (float(v) for v in out)))


def run_imag_until(psi, d, dt, omega, g, mu_tol, check_every=10, max_steps=100000, rule=0):
    """Imaginary-time propagation with the stop rule |mu(n) - mu(n-K)| < tol,
    checked every K steps (reading R6); rule 1 also requires
    |E(n) - E(n-K)| < tol, rule 2 rule 1's test at two consecutive checks.
    Returns (steps taken, last mu)."""
    o = observables(psi, d, omega, g)
    mu_prev, e_prev = o["mu"], o["energy"]
    steps, streak = 0, 0
    while steps < max_steps:
        step(psi, d, dt, omega, g, False, check_every)
        steps += check_every
        o = observables(psi, d, omega, g)
        ok = abs(o["mu"] - mu_prev) < mu_tol and (rule == 0 or abs(o["energy"] - e_prev) < mu_tol)
        streak = streak + 1 if ok else 0
        if streak >= (2 if rule == 2 else 1):
            return steps, o["mu"]
        mu_prev, e_prev = o["mu"], o["energy"]
    return steps, mu_prev


def density_profiles(psi, d):
    """Integrated 1D densities of a field (the programs' density output):
    rho_x[i] = dy dz sum_{j,k} |psi_ijk|^2, rho_y[j] = dx dz sum_{i,k}
    |psi_ijk|^2, rho_z[k] = dx dy sum_{i,j} |psi_ijk|^2 -- |psi|^2 summed over
    the other two axes times their spacings, so that sum_i rho_x[i] dx is the
    norm.  Plain numpy sums in FP64 (the definition itself)."""
    psi = np.asarray(psi)
    rho = psi.real.astype(np.float64) ** 2 + psi.imag.astype(np.float64) ** 2
    return (rho.sum(axis=(1, 2)) * d[1] * d[2], rho.sum(axis=(0, 2)) * d[0] * d[2],
            rho.sum(axis=(0, 1)) * d[0] * d[1])


# -------------------------------------------------------- axially symmetric (R21)
def _axial_field(psi: np.ndarray) -> np.ndarray:
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous or psi.ndim != 2:
        raise TypeError("axial fields are C-contiguous complex128 arrays of shape (nx, nz)")
    return psi


def axial_gaussian(nx, nz, drho, dz, gamma, lam) -> np.ndarray:
    """The normalised g = 0 continuum ground state on the (rho, z) grid (R21)."""
    psi = np.zeros((int(nx), int(nz)), dtype=np.complex128)
    _check(_load().oracle_axial_gaussian(int(nx), int(nz), float(drho), float(dz), float(gamma), float(lam),
                                         psi.ctypes.data_as(_dp)), "axial_gaussian")
    return psi


def axial_kick(psi, drho, dz, dt, gamma, lam, g, realtime) -> np.ndarray:
    psi = _axial_field(psi)
    _check(_load().oracle_axial_kick(psi.shape[0], psi.shape[1], float(drho), float(dz), psi.ctypes.data_as(_dp),
                                     float(dt), float(gamma), float(lam), float(g), int(bool(realtime))),
           "axial_kick")
    return psi


def axial_sweep(psi, drho, dz, axis, dt, realtime) -> np.ndarray:
    """CN line solves along rho (axis 0) or z (axis 1), in place."""
    psi = _axial_field(psi)
    _check(_load().oracle_axial_sweep(psi.shape[0], psi.shape[1], float(drho), float(dz), psi.ctypes.data_as(_dp),
                                      int(axis), float(dt), int(bool(realtime))), "axial_sweep")
    return psi


def axial_step(psi, drho, dz, dt, gamma, lam, g, realtime, nsteps=1) -> np.ndarray:
    """In-place split-step CN steps of the axially symmetric equation (R21)."""
    psi = _axial_field(psi)
    _check(_load().oracle_axial_step(psi.shape[0], psi.shape[1], float(drho), float(dz), psi.ctypes.data_as(_dp),
                                     float(dt), float(gamma), float(lam), float(g), int(bool(realtime)),
                                     int(nsteps)), "axial_step")
    return psi


def axial_observables(psi, drho, dz, gamma, lam, g) -> dict:
    psi = _axial_field(psi)
    out = np.zeros(6, dtype=np.float64)
    _check(_load().oracle_axial_observables(psi.shape[0], psi.shape[1], float(drho), float(dz),
                                            psi.ctypes.data_as(_dp), float(gamma), float(lam), float(g),
                                            out.ctypes.data_as(_dp)), "axial_observables")
    return dict(zip(OBS_KEYS, (float(v) for v in out)))


def axial_run_imag_until(psi, drho, dz, dt, gamma, lam, g, mu_tol, check_every=10, max_steps=200000):
    """Imaginary time with the stop rule |mu(n) - mu(n-K)| < tol (R6).
    Returns (steps taken, last mu)."""
    mu_prev = axial_observables(psi, drho, dz, gamma, lam, g)["mu"]
    steps = 0
    while steps < max_steps:
        axial_step(psi, drho, dz, dt, gamma, lam, g, False, check_every)
        steps += check_every
        mu = axial_observables(psi, drho, dz, gamma, lam, g)["mu"]
        if abs(mu - mu_prev) < mu_tol:
            return steps, mu
        mu_prev = mu
    return steps, mu_prev
