"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
(numpy PCG64, ``numpy.random.default_rng(seed)``) and lays out the problem
parameters of the workloads.  Both the CUDA path and the CPU oracle receive
the arrays it returns, unchanged.

The paper runs its programs on its own supplied input files, which are not
available; the workloads below stand in for them with the grid sizes, trap
anisotropies and nonlinearities of the paper's problem class (fully
anisotropic harmonic trap, imaginary- and real-time propagation).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np


@dataclass
class Problem:
    """One condensate: grid, spacings, time step, trap and nonlinearity."""
    shape: Tuple[int, int, int]
    d: Tuple[float, float, float]
    dt: float
    omega: Tuple[float, float, float]  # (gamma, nu, lambda)
    g: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def sites(self) -> int:
        return int(self.shape[0]) * int(self.shape[1]) * int(self.shape[2])


def imag_small() -> Problem:
    """64x48x40, d = 0.2, dt = 0.1 d^2, trap (1, 1.4, 2), g = 10, 300 imaginary steps."""
    return Problem((64, 48, 40), (0.2, 0.2, 0.2), 0.1 * 0.2 ** 2, (1.0, 1.4, 2.0), 10.0,
                   name="imag 64x48x40 fp64 real, 300 steps", meta={"steps": 300})


def real_medium() -> Problem:
    """240x200x160, d = 0.1, dt = 0.02 d^2, trap (0.5, 1, 1.5), quench g 20 -> 40, 1000 steps."""
    return Problem((240, 200, 160), (0.1, 0.1, 0.1), 0.02 * 0.1 ** 2, (0.5, 1.0, 1.5), 40.0,
                   name="real 240x200x160 fp64 complex, quench g 20->40, 1000 steps",
                   meta={"steps": 1000, "g_prepare": 20.0})


def real_large() -> Problem:
    """480x400x320, d = 0.05 (same box as the 240x200x160 case), dt = 0.02 d^2, 500 steps."""
    return Problem((480, 400, 320), (0.05, 0.05, 0.05), 0.02 * 0.05 ** 2, (0.5, 1.0, 1.5), 40.0,
                   name="real 480x400x320 complex64, quench g 20->40, 500 steps",
                   meta={"steps": 500, "g_prepare": 20.0})


def real_large_half() -> Problem:
    """480x400x160 slab of the 480x400x320 workload (same spacing, dt and
    trap): a capture-sized case (246 MB complex64, still above L2) for
    profiling the same kernels."""
    p = real_large()
    return Problem((480, 400, 160), p.d, p.dt, p.omega, p.g,
                   name="real 480x400x160 complex64 (half-depth profiling case)", meta=dict(p.meta))


def imag_large() -> Problem:
    """The 480x400x320 grid of the real-time workload (d = 0.05, trap
    (0.5, 1, 1.5)) in imaginary time at g = 20, dt = 0.1 d^2: the precision
    variants of the imaginary-time path (FP32 real field against FP32
    complex) on an HBM-sized grid."""
    p = real_large()
    return Problem(p.shape, p.d, 0.1 * p.d[0] ** 2, p.omega, 20.0,
                   name="imag 480x400x320, g 20, dt 0.1 d^2", meta={})


def imag_large_half() -> Problem:
    """480x400x160 slab of the imaginary-time 480x400x320 workload (same
    spacing, dt, trap and g): a capture-sized case for profiling the same
    kernels."""
    p = imag_large()
    return Problem((480, 400, 160), p.d, p.dt, p.omega, p.g,
                   name="imag 480x400x160, g 20, dt 0.1 d^2 (half-depth profiling case)", meta={})


def imag_xl() -> Problem:
    """The imaginary-time workload on a larger grid, 640x480x400 at d = 0.05
    (trap (0.5, 1, 1.5), g = 20), at dt = d^2: the step of a schedule's
    coarse level (ten times the fine dt), where the FP16 storage variant
    runs.  At 640x480x400 an FP16 field (246 MB) exceeds the 129 MB L2; at
    480x400x320 it would fit."""
    p = imag_large()
    return Problem((640, 480, 400), p.d, p.d[0] ** 2, p.omega, p.g,
                   name="imag 640x480x400, g 20, dt d^2 (coarse level)", meta={})


def sized_box(shape, omega, g, dt_factor=0.1) -> Problem:
    """Grid spacing that holds both the g = 0 Gaussian (6 oscillator lengths)
    and 1.3x the Thomas-Fermi radius in the half-box, per axis."""
    gamma, nu, lam = omega
    mu_tf = 0.5 * (15.0 * g * gamma * nu * lam / (4.0 * math.pi)) ** 0.4
    d = []
    for n, w in zip(shape, omega):
        r_tf = math.sqrt(2.0 * mu_tf) / w
        half = max(6.0 / math.sqrt(w), 1.3 * r_tf)
        d.append(2.0 * half / (n - 1))
    dt = dt_factor * min(d) ** 2
    return Problem(tuple(int(n) for n in shape), tuple(d), dt, tuple(omega), float(g))


def batch_problems(count=64, seed=0, g_max=200.0) -> List[Problem]:
    """Uneven batch: Nx in [32, 128], Ny in [32, 96], Nz in [32, 80];
    gamma, nu, lambda ~ U[0.5, 3]; log g ~ U[ln 1, ln g_max]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        shape = (int(rng.integers(32, 129)), int(rng.integers(32, 97)), int(rng.integers(32, 81)))
        omega = tuple(float(x) for x in rng.uniform(0.5, 3.0, size=3))
        g = float(math.exp(rng.uniform(0.0, math.log(g_max))))
        p = sized_box(shape, omega, g)
        p.name = "batch[%d]" % b
        out.append(p)
    return out


def random_field(shape, seed=0, complex_=True, envelope=True) -> np.ndarray:
    """A seeded random field that is zero on the boundary nodes (of the axes
    with more than one node).

    With ``envelope`` the values are a smooth bump times (1 + 0.25 noise) with a
    random phase, which resembles a perturbed condensate; without it they are
    plain standard normal noise.  Returned as complex128 (or float64).
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(s) for s in shape)
    re = rng.standard_normal((nx, ny, nz))
    im = rng.standard_normal((nx, ny, nz)) if complex_ else None
    if envelope:
        # an axis of one node (an absent axis of a 1D or 2D grid) sits at the centre
        ax = [np.linspace(-1.0, 1.0, n) if n > 1 else np.zeros(1) for n in (nx, ny, nz)]
        bump = (np.cos(0.5 * math.pi * ax[0])[:, None, None] *
                np.cos(0.5 * math.pi * ax[1])[None, :, None] *
                np.cos(0.5 * math.pi * ax[2])[None, None, :])
        amp = bump * (1.0 + 0.25 * re)
        if complex_:
            phase = rng.uniform(-math.pi, math.pi, size=(nx, ny, nz))
            f = amp * np.exp(1j * phase)
        else:
            f = amp
    else:
        f = re + 1j * im if complex_ else re
    f = np.array(f, dtype=np.complex128 if complex_ else np.float64)
    for axis, n in enumerate((nx, ny, nz)):
        if n > 1:  # an axis of one node has no boundary nodes
            sl = [slice(None)] * 3
            for end in (0, -1):
                sl[axis] = end
                f[tuple(sl)] = 0
    return f
