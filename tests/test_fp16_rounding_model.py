"""Why FP16 storage is only a coarse stage (CPU): the FP64 oracle's step with
every sweep's output rounded to IEEE half, as GP_F16 stores psi, against the
unrounded step from the same Gaussian.  At dt = 2.5e-4 a step changes psi by
less than the rounding and the imaginary-time evolution stalls (mu stays
several per cent above the FP64 value after 250 steps); at ten times that
dt the rounded run follows to a few parts in a thousand.  The same gaps
(4.7 % and 0.2 %) were measured on the GPU's FP16 path on 640x480x400."""
import numpy as np

import oracle

SHAPE, D, OMEGA, G = (41, 33, 29), (0.5, 0.5, 0.5), (0.5, 1.0, 1.5), 20.0


def mu_after(dt, steps, half):
    psi = oracle.gaussian(SHAPE, D, OMEGA).astype(np.complex128)
    if half:
        psi = np.ascontiguousarray(psi.real.astype(np.float16).astype(np.complex128))
    for _ in range(steps):
        oracle.kick(psi, D, dt, OMEGA, G, False)
        for ax in range(3):
            oracle.sweep(psi, D, ax, dt, False)
            if half:
                psi = np.ascontiguousarray(psi.real.astype(np.float16).astype(np.complex128))
        oracle.renormalize(psi, D)
    return oracle.observables(psi, D, OMEGA, G)["mu"]


def test_fp16_rounding_stalls_small_dt_only():
    small = [mu_after(2.5e-4, 250, h) for h in (False, True)]
    large = [mu_after(2.5e-3, 250, h) for h in (False, True)]
    assert (small[1] - small[0]) / small[0] > 0.02, small
    assert abs(large[1] - large[0]) / large[0] < 0.005, large
