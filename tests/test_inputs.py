"""The seeded input recipe (CPU): the workloads' sizes and parameters, the
box-sizing rule of the batched and warm-start condensates (the half-box holds
6 oscillator lengths and 1.3 Thomas-Fermi radii), the batch's parameter
ranges, determinism of every generator, and the parity fields' boundary."""
import math

import numpy as np

from paper_1601_04641_gb300 import inputs


def test_benchmark_workloads():
    p = inputs.real_large()
    assert p.shape == (480, 400, 320) and p.d == (0.05, 0.05, 0.05)
    assert abs(p.dt - 0.02 * 0.05 ** 2) < 1e-18 and p.omega == (0.5, 1.0, 1.5) and p.g == 40.0
    assert p.meta["g_prepare"] == 20.0 and p.sites == 480 * 400 * 320
    m = inputs.real_medium()
    assert m.shape == (240, 200, 160) and m.d == (0.1, 0.1, 0.1) and m.g == 40.0
    s = inputs.imag_small()
    assert s.shape == (64, 48, 40) and s.omega == (1.0, 1.4, 2.0) and s.g == 10.0
    h = inputs.real_large_half()
    assert h.shape == (480, 400, 160) and h.d == p.d and h.dt == p.dt


def test_sized_box_holds_gaussian_and_thomas_fermi_radius():
    for shape, omega, g in (((64, 48, 40), (1.0, 1.4, 2.0), 10.0), ((33, 95, 71), (0.5, 3.0, 1.7), 199.0),
                            ((128, 96, 80), (2.9, 0.6, 1.1), 1.0)):
        p = inputs.sized_box(shape, omega, g)
        mu_tf = 0.5 * (15.0 * g * omega[0] * omega[1] * omega[2] / (4.0 * math.pi)) ** 0.4
        for n, d, w in zip(shape, p.d, omega):
            half = 0.5 * (n - 1) * d
            assert half >= 6.0 / math.sqrt(w) - 1e-12            # the g = 0 Gaussian
            assert half >= 1.3 * math.sqrt(2.0 * mu_tf) / w - 1e-12  # 1.3 Thomas-Fermi radii
            assert abs(half - max(6.0 / math.sqrt(w), 1.3 * math.sqrt(2.0 * mu_tf) / w)) < 1e-12
        assert abs(p.dt - 0.1 * min(p.d) ** 2) < 1e-15


def test_batch_ranges_and_determinism():
    a = inputs.batch_problems(64, seed=0)
    b = inputs.batch_problems(64, seed=0)
    assert [(p.shape, p.omega, p.g) for p in a] == [(p.shape, p.omega, p.g) for p in b]
    for p in a:
        assert 32 <= p.shape[0] <= 128 and 32 <= p.shape[1] <= 96 and 32 <= p.shape[2] <= 80
        assert all(0.5 <= w <= 3.0 for w in p.omega)
        assert 1.0 <= p.g <= 200.0
    total = sum(p.sites for p in a)
    assert 1.0e7 < total < 3.0e7  # about 1.8e7 expected
    c = inputs.batch_problems(64, seed=1)
    assert [p.shape for p in c] != [p.shape for p in a]


def test_random_field_is_seeded_and_zero_on_the_boundary():
    f = inputs.random_field((9, 8, 7), seed=3)
    assert np.array_equal(f, inputs.random_field((9, 8, 7), seed=3))
    assert not np.array_equal(f, inputs.random_field((9, 8, 7), seed=4))
    for ax in range(3):
        for idx in (0, f.shape[ax] - 1):
            assert np.all(np.take(f, idx, axis=ax) == 0)
    assert np.all(np.abs(f[1:-1, 1:-1, 1:-1]) > 0)
