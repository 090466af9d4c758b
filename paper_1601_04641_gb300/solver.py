"""Python front end of libgpcn: one condensate on one GPU.

PyTorch provides the device memory of psi and the CUDA stream; every step of
the method runs in the library's CUDA kernels through the C ABI.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _native as N

_TORCH_DTYPES = {("f64", "complex"): "complex128", ("f32", "complex"): "complex64",
                 ("f64", "real"): "float64", ("f32", "real"): "float32", ("f16", "real"): "float16"}
_NP_DTYPES = {("f64", "complex"): np.complex128, ("f32", "complex"): np.complex64,
              ("f64", "real"): np.float64, ("f32", "real"): np.float32, ("f16", "real"): np.float16}
_PRECISIONS = {"f64": N.GP_F64, "f32": N.GP_F32, "f16": N.GP_F16}


class GP:
    """Split-step Crank-Nicolson solver of the 3D GP equation in a fully
    anisotropic harmonic trap (imaginary or real time).

    shape: (nx, ny, nz); d: (dx, dy, dz); omega: (gamma, nu, lambda).
    precision: "f64", "f32" or "f16" (element precision of psi; reductions are
    FP64; "f16" stores psi in half precision with FP32 arithmetic, real fields);
    field: "complex" or "real" (real allows imaginary time only).
    """

    def __init__(self, shape, d, dt, omega, g, precision="f64", field="complex", device=None,
                 stream=None):
        import torch
        self._torch = torch
        self.lib = N.load()
        self.shape = tuple(int(s) for s in shape)
        self.d = tuple(float(x) for x in d)
        self.precision, self.field = precision, field
        key = (precision, field)
        if key not in _TORCH_DTYPES:
            raise ValueError("precision must be f64/f32 (or f16 with a real field) and field complex/real")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.np_dtype = _NP_DTYPES[key]
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.psi = torch.zeros(self.shape, dtype=getattr(torch, _TORCH_DTYPES[key]),
                                   device=self.device)
            grid = N.Grid(*self.shape, *self.d)
            h = N.Handle()
            st = self.lib.gp_create_ext(ctypes.byref(h), grid, float(dt), float(omega[0]),
                                        float(omega[1]), float(omega[2]), float(g),
                                        _PRECISIONS[precision],
                                        N.GP_COMPLEX if field == "complex" else N.GP_REAL,
                                        ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.c_void_p(self.psi.data_ptr()),
                                        self.psi.numel() * self.psi.element_size())
            N.check(st, None)
        self.h = h

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        N.check(st, self.h)

    # ------------------------------------------------------------ state
    def init_gaussian(self):
        self._ck(self.lib.gp_init_gaussian(self.h))

    def set_psi(self, arr):
        """Copy psi in from a numpy array or a CUDA tensor of this shape."""
        torch = self._torch
        if isinstance(arr, torch.Tensor) and arr.is_cuda:
            t = arr.to(dtype=self.psi.dtype).contiguous()
            if tuple(t.shape) != self.shape:
                raise ValueError("shape mismatch")
            self._ck(self.lib.gp_set_psi(self.h, ctypes.c_void_p(t.data_ptr()), 1))
            self._keep = t
            return
        a = np.ascontiguousarray(np.asarray(arr), dtype=self.np_dtype)
        if a.shape != self.shape:
            raise ValueError("shape mismatch")
        self._ck(self.lib.gp_set_psi(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_psi(self, as_numpy=True):
        """Current psi (pending renormalisation applied)."""
        if as_numpy:
            out = np.empty(self.shape, dtype=self.np_dtype)
            self._ck(self.lib.gp_get_psi(self.h, out.ctypes.data_as(ctypes.c_void_p), 0))
            return out
        out = self._torch.empty_like(self.psi)
        self._ck(self.lib.gp_get_psi(self.h, ctypes.c_void_p(out.data_ptr()), 1))
        return out

    def set_g(self, g):
        self._ck(self.lib.gp_set_g(self.h, float(g)))

    def set_dt(self, dt):
        self._ck(self.lib.gp_set_dt(self.h, float(dt)))

    # ------------------------------------------------------------ stepping
    def step_imag(self, nsteps=1):
        self._ck(self.lib.gp_step_imag(self.h, int(nsteps)))

    def step_real(self, nsteps=1):
        self._ck(self.lib.gp_step_real(self.h, int(nsteps)))

    def stage(self, stage, realtime=False):
        self._ck(self.lib.gp_step_stage(self.h, int(stage), int(bool(realtime))))

    def run_imag_until(self, mu_tol, check_every=10, max_steps=100000):
        taken = ctypes.c_int(0)
        self._ck(self.lib.gp_run_imag_until(self.h, float(mu_tol), int(check_every),
                                            int(max_steps), ctypes.byref(taken)))
        return taken.value

    def observables(self):
        o = N.Obs()
        self._ck(self.lib.gp_observables(self.h, ctypes.byref(o)))
        return {"norm": o.norm, "mu": o.mu, "energy": o.energy, "rms_x": o.rms_x,
                "rms_y": o.rms_y, "rms_z": o.rms_z, "step": o.step, "t": o.t}

    def density_profiles(self):
        """Integrated 1D densities (rho_x, rho_y, rho_z) of the current psi,
        each summed over the other two axes times their spacings."""
        nx, ny, nz = self.shape
        rx, ry, rz = np.empty(nx), np.empty(ny), np.empty(nz)
        dp = ctypes.POINTER(ctypes.c_double)
        self._ck(self.lib.gp_density_profiles(self.h, rx.ctypes.data_as(dp), ry.ctypes.data_as(dp),
                                              rz.ctypes.data_as(dp)))
        return rx, ry, rz

    def write_wavefunction(self, path, density=False):
        """Write psi (or |psi|^2) to `path` as a .npy file of shape (nx, ny, nz)."""
        self._ck(self.lib.gp_write_wavefunction(self.h, os.fsencode(path),
                                                N.GP_OUT_DENSITY if density else N.GP_OUT_PSI))

    def set_tracking(self, every, capacity=1024):
        """Queue the observables every `every` steps on the device (no host sync)."""
        self._ck(self.lib.gp_set_tracking(self.h, int(every), int(capacity)))

    def tracking(self, max_records=1 << 16):
        """Tracked records so far, oldest first."""
        buf = (N.Obs * max_records)()
        cnt = ctypes.c_int(0)
        self._ck(self.lib.gp_get_tracking(self.h, buf, int(max_records), ctypes.byref(cnt)))
        return [{"norm": o.norm, "mu": o.mu, "energy": o.energy, "rms_x": o.rms_x, "rms_y": o.rms_y,
                 "rms_z": o.rms_z, "step": o.step, "t": o.t} for o in buf[:min(cnt.value, max_records)]]

    def sync(self):
        self._ck(self.lib.gp_sync(self.h))

    # ------------------------------------------------------------ tuning
    def window(self, mode=0):
        w = (ctypes.c_int * 3)()
        self._ck(self.lib.gp_get_window(self.h, int(mode), w))
        return tuple(w)

    def set_window(self, window):
        self._ck(self.lib.gp_set_window(self.h, int(window)))

    def set_segments(self, axis, seg_len):
        self._ck(self.lib.gp_set_segments(self.h, int(axis), int(seg_len)))

    def segments(self, mode=0):
        a = (ctypes.c_int * 3)()
        b = (ctypes.c_int * 3)()
        self._ck(self.lib.gp_get_segments(self.h, int(mode), a, b))
        return tuple(a), tuple(b)

    def autotune(self, realtime=False, reps=5, cache_path=None):
        """Time candidate launch settings per axis and keep the fastest."""
        self._ck(self.lib.gp_autotune(self.h, int(bool(realtime)), int(reps),
                                      cache_path.encode() if cache_path else None))

    def set_graph_block(self, steps):
        self._ck(self.lib.gp_set_graph_block(self.h, int(steps)))

    def set_axis_window(self, axis, window):
        self._ck(self.lib.gp_set_axis_window(self.h, int(axis), int(window)))

    def set_pair_lines(self, on):
        """Widest line groups per thread on the strided axes (on) or one line."""
        self._ck(self.lib.gp_set_pair_lines(self.h, int(bool(on))))

    def set_lines_per_thread(self, axis, lines):
        """Most adjacent lines per thread on axis 0 (x) or 1 (y): 1, 2 or 4."""
        self._ck(self.lib.gp_set_lines_per_thread(self.h, int(axis), int(lines)))

    def lines_per_thread(self, mode=0):
        a = (ctypes.c_int * 3)()
        self._ck(self.lib.gp_get_lines_per_thread(self.h, int(mode), a))
        return tuple(a)

    def set_tma(self, on):
        """z sweep through TMA tiles (default where the grid allows it)."""
        self._ck(self.lib.gp_set_tma(self.h, int(bool(on))))

    def set_tma_lines(self, axes):
        """Axes (bit 0: x, bit 1: y) whose sweeps read through TMA boxes where the grid allows it;
        -1 (default): x for real fields (imaginary time), none for complex fields."""
        self._ck(self.lib.gp_set_tma_lines(self.h, int(axes)))

    def tma_lines_in_use(self):
        """Axes (bit 0: x, bit 1: y) whose sweeps take the TMA box form."""
        v = ctypes.c_int(0)
        self._ck(self.lib.gp_get_tma_lines(self.h, ctypes.byref(v)))
        return v.value

    def set_stop_rule(self, rule):
        """0: |dmu| < tol (default); 1: |dmu| < tol and |dE| < tol; 2: rule 1 at two consecutive checks."""
        self._ck(self.lib.gp_set_stop_rule(self.h, int(rule)))

    def set_splitting(self, order):
        """Real-time splitting: 1 kick then sweeps (default), 2 symmetric."""
        self._ck(self.lib.gp_set_splitting(self.h, int(order)))

    def run_imag_schedule(self, levels, check_every=10, max_steps=100000):
        """levels: sequence of (dt scale, mu tol); see gp_run_imag_schedule."""
        n = len(levels)
        sc = (ctypes.c_double * n)(*[float(a) for a, _ in levels])
        tl = (ctypes.c_double * n)(*[float(b) for _, b in levels])
        taken = ctypes.c_int(0)
        self._ck(self.lib.gp_run_imag_schedule(self.h, n, sc, tl, int(check_every), int(max_steps),
                                               ctypes.byref(taken)))
        return taken.value

    def tma_in_use(self):
        v = ctypes.c_int(0)
        self._ck(self.lib.gp_get_tma(self.h, ctypes.byref(v)))
        return bool(v.value)

    def set_threads(self, axis, threads):
        self._ck(self.lib.gp_set_threads(self.h, int(axis), int(threads)))


class Batch:
    """Many independent condensates advanced together in imaginary time.

    problems: sequence of objects with .shape, .d, .dt, .omega, .g (e.g.
    paper_1601_04641_gb300.inputs.Problem).  All share precision and field.
    """

    def __init__(self, problems, precision="f32", field="complex", device=None):
        import torch
        self._torch = torch
        self.lib = N.load()
        self.problems = list(problems)
        n = len(self.problems)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.np_dtype = _NP_DTYPES[(precision, field)]
        grids = (N.Grid * n)(*[N.Grid(*p.shape, *p.d) for p in self.problems])
        arr = lambda vals: (ctypes.c_double * n)(*[float(v) for v in vals])
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            h = N.Handle()
            st = self.lib.gp_batch_create(ctypes.byref(h), n, grids, arr(p.dt for p in self.problems),
                                          arr(p.omega[0] for p in self.problems),
                                          arr(p.omega[1] for p in self.problems),
                                          arr(p.omega[2] for p in self.problems),
                                          arr(p.g for p in self.problems),
                                          _PRECISIONS[precision],
                                          N.GP_COMPLEX if field == "complex" else N.GP_REAL,
                                          ctypes.c_void_p(self.stream.cuda_stream))
            N.check(st, None, batch=True)
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        N.check(st, self.h, batch=True)

    def init_gaussian(self):
        self._ck(self.lib.gp_batch_init_gaussian(self.h))

    def set_psi(self, i, arr):
        a = np.ascontiguousarray(np.asarray(arr), dtype=self.np_dtype)
        if a.shape != tuple(self.problems[i].shape):
            raise ValueError("shape mismatch")
        self._ck(self.lib.gp_batch_set_psi(self.h, int(i), a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_psi(self, i):
        out = np.empty(tuple(self.problems[i].shape), dtype=self.np_dtype)
        self._ck(self.lib.gp_batch_get_psi(self.h, int(i), out.ctypes.data_as(ctypes.c_void_p), 0))
        return out

    def step_imag(self, nsteps=1):
        self._ck(self.lib.gp_batch_step_imag(self.h, int(nsteps)))

    def observables(self):
        buf = (N.Obs * self.n)()
        self._ck(self.lib.gp_batch_observables(self.h, buf))
        return [{"norm": o.norm, "mu": o.mu, "energy": o.energy, "rms_x": o.rms_x, "rms_y": o.rms_y,
                 "rms_z": o.rms_z, "step": o.step, "t": o.t} for o in buf]

    def run_imag_until(self, mu_tol, check_every=10, max_steps=100000):
        taken = (ctypes.c_int * self.n)()
        self._ck(self.lib.gp_batch_run_imag_until(self.h, float(mu_tol), int(check_every), int(max_steps),
                                                  taken))
        return list(taken)

    def window(self):
        w = (ctypes.c_int * 3)()
        self._ck(self.lib.gp_batch_get_window(self.h, w))
        return tuple(w)

    def segments(self, i):
        a = (ctypes.c_int * 3)()
        b = (ctypes.c_int * 3)()
        self._ck(self.lib.gp_batch_get_segments(self.h, int(i), a, b))
        return tuple(a), tuple(b)

    def set_stop_rule(self, rule):
        """0: |dmu| < tol (default); 1: |dmu| < tol and |dE| < tol; 2: rule 1 at two consecutive checks."""
        self._ck(self.lib.gp_batch_set_stop_rule(self.h, int(rule)))

    def set_dt_scale(self, scale):
        self._ck(self.lib.gp_batch_set_dt_scale(self.h, float(scale)))

    def run_imag_schedule(self, levels, check_every=10, max_steps=100000):
        """levels: sequence of (dt scale, mu tol); steps per instance."""
        n = len(levels)
        sc = (ctypes.c_double * n)(*[float(a) for a, _ in levels])
        tl = (ctypes.c_double * n)(*[float(b) for _, b in levels])
        taken = (ctypes.c_int * self.n)()
        self._ck(self.lib.gp_batch_run_imag_schedule(self.h, n, sc, tl, int(check_every), int(max_steps), taken))
        return list(taken)

    def set_graph_block(self, steps):
        self._ck(self.lib.gp_batch_set_graph_block(self.h, int(steps)))

    def set_streams(self, streams):
        """Stream groups of a step (1..16): independent chains of sweeps that overlap."""
        self._ck(self.lib.gp_batch_set_streams(self.h, int(streams)))

    def set_segments(self, seg_len):
        """Interior nodes per segment on the strided axes (0: automatic)."""
        self._ck(self.lib.gp_batch_set_segments(self.h, int(seg_len)))

    def set_tma(self, on):
        """z sweep through TMA tiles for the instances whose rows fit (default on)."""
        self._ck(self.lib.gp_batch_set_tma(self.h, int(bool(on))))

    def tma_count(self):
        v = ctypes.c_int(0)
        self._ck(self.lib.gp_batch_get_tma(self.h, ctypes.byref(v)))
        return v.value


def ground_state(shape, d, dt, omega, g, tol=1e-10, device=None, max_steps=200000,
                 levels=((30.0, 1e-6), (10.0, 1e-7), (3.0, 1e-8), (1.0, 1e-9))):
    """The imaginary-time ground state of one condensate at time step dt, as
    a float64 CUDA tensor of `shape`: an FP32 real field from the Gaussian
    through a dt schedule (`levels` of (dt scale, mu tolerance), stop rule 1),
    then FP64 imaginary time at dt from that state until
    |mu(n) - mu(n-10)| < tol.  Returns (psi, info); info holds the steps and
    seconds of both stages, mu and the last |mu(n) - mu(n-10)|."""
    import time
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g32 = GP(shape, d, dt, omega, g, "f32", "real", device=device)
    g32.set_stop_rule(1)
    g32.init_gaussian()
    n32 = g32.run_imag_schedule(levels, 10, max_steps)
    mu32 = g32.observables()["mu"]
    psi = g32.get_psi(as_numpy=False).to(torch.float64)
    g32.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g64 = GP(shape, d, dt, omega, g, "f64", "real", device=device)
    g64.set_psi(psi)
    mu_prev = g64.observables()["mu"]
    n64, dmu = 0, float("inf")
    while n64 < max_steps:
        g64.step_imag(10)
        n64 += 10
        mu = g64.observables()["mu"]
        dmu = abs(mu - mu_prev)
        mu_prev = mu
        if dmu < tol:
            break
    psi = g64.get_psi(as_numpy=False)
    g64.close()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return psi, {"fp32_schedule_steps": n32, "fp32_s": t1 - t0, "mu_fp32": mu32,
                 "fp64_steps": n64, "fp64_s": t2 - t1, "mu": mu_prev, "last_dmu": dmu, "tol": tol,
                 "converged": dmu < tol}


class AxialGP:
    """Axially symmetric condensate psi(rho, z) (trap gamma = nu, lambda):
    a C array of shape (nx, nz); radial node i at rho = (i - 1/2) drho (node 0
    a ghost, node nx-1 the boundary), z nodes centred.  See gp_axial_create."""

    def __init__(self, nx, nz, drho, dz, dt, gamma, lam, g, precision="f64", field="complex", device=None):
        import torch
        self._torch = torch
        self.lib = N.load()
        self.shape = (int(nx), int(nz))
        key = (precision, field)
        if key not in _NP_DTYPES or precision == "f16":
            raise ValueError("precision must be f64/f32 and field complex/real")
        self.np_dtype = _NP_DTYPES[key]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            h = N.Handle()
            st = self.lib.gp_axial_create(ctypes.byref(h), int(nx), int(nz), float(drho), float(dz), float(dt),
                                          float(gamma), float(lam), float(g), _PRECISIONS[precision],
                                          N.GP_COMPLEX if field == "complex" else N.GP_REAL,
                                          ctypes.c_void_p(self.stream.cuda_stream))
            N.check(st, None, axial=True)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_axial_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        N.check(st, self.h, axial=True)

    def init_gaussian(self):
        self._ck(self.lib.gp_axial_init_gaussian(self.h))

    def set_psi(self, arr):
        a = np.ascontiguousarray(np.asarray(arr), dtype=self.np_dtype)
        if a.shape != self.shape:
            raise ValueError("psi must have shape %s" % (self.shape,))
        self._ck(self.lib.gp_axial_set_psi(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_psi(self):
        out = np.empty(self.shape, dtype=self.np_dtype)
        self._ck(self.lib.gp_axial_get_psi(self.h, out.ctypes.data_as(ctypes.c_void_p), 0))
        return out

    def step_imag(self, n=1):
        self._ck(self.lib.gp_axial_step_imag(self.h, int(n)))

    def step_real(self, n=1):
        self._ck(self.lib.gp_axial_step_real(self.h, int(n)))

    def observables(self):
        o = N.Obs()
        self._ck(self.lib.gp_axial_observables(self.h, ctypes.byref(o)))
        return {k: getattr(o, k) for k in ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z", "step", "t")}

    def run_imag_until(self, mu_tol, check_every=10, max_steps=200000):
        taken = ctypes.c_int(0)
        self._ck(self.lib.gp_axial_run_imag_until(self.h, float(mu_tol), int(check_every), int(max_steps),
                                                  ctypes.byref(taken)))
        return taken.value
