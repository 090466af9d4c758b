"""Learned warm start for imaginary-time propagation.

A small network (see include/gp.h, "warm start") predicts the ground-state
amplitude of a condensate on its grid from (gamma, nu, lambda, g).  This
module drives the library's GPU kernels: it generates training targets with
the batched solver (the method's own ground states), trains the network with
the GPU forward/backward/Adam kernels, and runs imaginary time from the
prediction.  Policy: the prediction replaces the Gaussian start unless it is
non-finite or its energy is above the Gaussian's, in which case the Gaussian
is kept.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import _native as N


class Net:
    def __init__(self, seed=0, device=None):
        import torch
        self._torch = torch
        self.lib = N.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device)
            h = N.Handle()
            N.check(self.lib.gp_nn_create(ctypes.byref(h), ctypes.c_ulonglong(seed),
                                          ctypes.c_void_p(self.stream.cuda_stream)), None, nn=True)
        self.h = h
        self.count = self.lib.gp_nn_param_count()
        self._data = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        N.check(st, self.h, nn=True)

    @property
    def params(self):
        out = np.empty(self.count, dtype=np.float32)
        self._ck(self.lib.gp_nn_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.count))
        return out

    @params.setter
    def params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        self._ck(self.lib.gp_nn_set_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def set_data(self, problems, data, offsets, psi_max):
        """data: float32 CUDA tensor holding every instance's target amplitudes."""
        n = len(problems)
        grids = (N.Grid * n)(*[N.Grid(*p.shape, *p.d) for p in problems])
        arr = lambda vals: (ctypes.c_double * n)(*[float(v) for v in vals])
        offs = (ctypes.c_longlong * n)(*[int(o) for o in offsets])
        mx = (ctypes.c_float * n)(*[float(m) for m in psi_max])
        self._data = data  # keep the device buffer alive
        self._ck(self.lib.gp_nn_set_data(self.h, n, grids, arr(p.omega[0] for p in problems),
                                         arr(p.omega[1] for p in problems), arr(p.omega[2] for p in problems),
                                         arr(p.g for p in problems), ctypes.c_void_p(data.data_ptr()), offs, mx))

    def train(self, steps, points=32768, lr=1e-3, seed=0):
        loss = ctypes.c_float(0.0)
        self._ck(self.lib.gp_nn_train(self.h, int(steps), int(points), ctypes.c_float(lr), ctypes.c_ulonglong(seed),
                                      ctypes.byref(loss)))
        return float(loss.value)

    def loss_grad(self, instance, site):
        inst = np.ascontiguousarray(instance, dtype=np.int32)
        st = np.ascontiguousarray(site, dtype=np.int64)
        loss = ctypes.c_float(0.0)
        grad = np.empty(self.count, dtype=np.float32)
        self._ck(self.lib.gp_nn_loss_grad(self.h, inst.size, inst.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                          st.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), ctypes.byref(loss),
                                          grad.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return float(loss.value), grad

    def predict(self, gp):
        self._ck(self.lib.gp_nn_predict(self.h, gp.h))

    def predict_batch(self, batch):
        self._ck(self.lib.gp_nn_predict_batch(self.h, batch.h))


def ground_states(problems, tol, max_steps=40000, chunk=256, device=None, polish=0,
                  levels=((10.0, 1e-5), (3.0, 1e-6)), with_info=False):
    """Ground states of `problems` from the batched solver (the method's own
    ground states), in chunks of `chunk` condensates:
    - polish 0: FP32 real-field batches run to |mu(n) - mu(n-10)| < tol;
    - polish > 0: FP32 real-field batches through the dt schedule `levels`
      ((dt scale, mu tolerance)) and then at dt to |mu(n) - mu(n-10)| < tol
      (stop rule 1; the FP32 iteration settles bit for bit at its fixed
      point, so any tolerance is reached), then `polish` FP64 imaginary-time
      steps of each state at dt.
    Returns (data, offsets, psi_max, mu), and a dict of steps and times with
    with_info; data is a float32 CUDA tensor with the normalised amplitudes
    concatenated."""
    import torch
    from .solver import Batch
    sizes = [p.sites for p in problems]
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    data = torch.empty(int(sum(sizes)), dtype=torch.float32, device=device or "cuda")
    psi_max, mu = [], []
    info = {"fp32_steps_max": 0, "fp64_steps_max": 0, "fp32_s": 0.0, "fp64_s": 0.0, "tol": tol,
            "converged": 0, "of": len(problems)}
    for c0 in range(0, len(problems), chunk):
        part = problems[c0:c0 + chunk]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = Batch(part, "f32", "real", device=device)
        b.init_gaussian()
        if polish:
            b.set_stop_rule(1)
            steps = b.run_imag_schedule(list(levels) + [(1.0, tol)], 10, max_steps)
        else:
            steps = b.run_imag_until(tol, 10, max_steps)
        info["fp32_steps_max"] = max(info["fp32_steps_max"], max(steps))
        if polish:
            # FP64 from the FP32 states (the same fixed point up to FP32 rounding)
            tmp = [torch.empty(p.shape, dtype=torch.float32, device=data.device) for p in part]
            for i, t in enumerate(tmp):
                N.check(b.lib.gp_batch_get_psi(b.h, i, ctypes.c_void_p(t.data_ptr()), 1), b.h, batch=True)
            torch.cuda.synchronize()
            b.close()
            info["fp32_s"] += time.perf_counter() - t0
            t0 = time.perf_counter()
            b = Batch(part, "f64", "real", device=device)
            for i, t in enumerate(tmp):
                t64 = t.to(torch.float64)
                N.check(b.lib.gp_batch_set_psi(b.h, i, ctypes.c_void_p(t64.data_ptr()), 1), b.h, batch=True)
                torch.cuda.synchronize()
            del tmp
            b.step_imag(polish)
            info["fp64_steps_max"] = polish
        info["converged"] += sum(x < max_steps * ((len(levels) + 1) if polish else 1) for x in steps)
        mu += [o["mu"] for o in b.observables()]
        for i in range(len(part)):
            off = int(offsets[c0 + i])
            view = data[off:off + part[i].sites]
            if polish:
                t64 = torch.empty(part[i].sites, dtype=torch.float64, device=data.device)
                N.check(b.lib.gp_batch_get_psi(b.h, i, ctypes.c_void_p(t64.data_ptr()), 1), b.h, batch=True)
                view.copy_(t64)
            else:
                N.check(b.lib.gp_batch_get_psi(b.h, i, ctypes.c_void_p(view.data_ptr()), 1), b.h, batch=True)
        torch.cuda.synchronize()
        for i in range(len(part)):
            off = int(offsets[c0 + i])
            psi_max.append(float(data[off:off + part[i].sites].abs().max().item()))
        b.close()
        info["fp64_s" if polish else "fp32_s"] += time.perf_counter() - t0
    if with_info:
        return data, offsets, psi_max, mu, info
    return data, offsets, psi_max, mu


def train(net, steps, points=32768, lr=(3e-3, 3e-4), seed=0, report=None):
    """Adam with a geometric learning-rate decay from lr[0] to lr[1], in
    blocks of 100 steps; returns the loss of each block's last step."""
    losses = []
    blocks = max(1, steps // 100)
    for b in range(blocks):
        rate = lr[0] * (lr[1] / lr[0]) ** (b / max(1, blocks - 1))
        losses.append(net.train(100, points, rate, seed + b))
        if report:
            report(b, losses[-1])
    return losses


def run_from_starts(net, problems, tol, precision="f64", field="real", max_steps=40000, device=None,
                    stop_rule=1):
    """Imaginary time to |dmu| < tol (and |dE| < tol with stop_rule 1, see
    gp_set_stop_rule) from the Gaussian and from the network's prediction
    (with the energy fallback), each as one batch.  Returns a dict of
    per-instance steps, energies of the starts, converged mu and times."""
    import torch
    from .solver import GP, Batch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bg = Batch(problems, precision, field, device=device)
    bg.set_stop_rule(stop_rule)
    bg.init_gaussian()
    e_gauss = [o["energy"] for o in bg.observables()]
    steps_g = bg.run_imag_until(tol, 10, max_steps)
    mu_g = [o["mu"] for o in bg.observables()]
    torch.cuda.synchronize()
    t_gauss = time.perf_counter() - t0
    bg.close()

    t0 = time.perf_counter()
    bn = Batch(problems, precision, field, device=device)
    bn.set_stop_rule(stop_rule)
    net.predict_batch(bn)
    try:
        e_nn = [o["energy"] for o in bn.observables()]
    except N.GPError:
        e_nn = [float("nan")] * len(problems)
    fallback = [not (np.isfinite(en) and en <= eg) for en, eg in zip(e_nn, e_gauss)]
    for i, fb in enumerate(fallback):
        if fb:
            p = problems[i]
            g = GP(p.shape, p.d, p.dt, p.omega, p.g, precision, field, device=device)
            g.init_gaussian()
            bn.set_psi(i, g.get_psi())
            g.close()
    steps_n = bn.run_imag_until(tol, 10, max_steps)
    mu_n = [o["mu"] for o in bn.observables()]
    torch.cuda.synchronize()
    t_nn = time.perf_counter() - t0
    bn.close()
    return {"steps_gauss": steps_g, "steps_nn": steps_n, "e_gauss": e_gauss, "e_nn": e_nn,
            "mu_gauss": mu_g, "mu_nn": mu_n, "fallback": fallback, "time_gauss_s": t_gauss,
            "time_nn_s": t_nn}
