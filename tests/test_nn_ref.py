"""Pins for the numpy FP64 reference of the warm-start network (CPU): its
backward pass against central finite differences, and its features against
their definition's closed-form special values."""
import math

import numpy as np

from oracle import nn_ref


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = nn_ref.init(1)
    x = rng.uniform(-1, 1, (40, nn_ref.IN))
    x[:, 9:] = 0.0
    t = rng.uniform(0, 1, 40)
    _, grad = nn_ref.loss_and_grad(theta, x, t)
    idx = rng.choice(nn_ref.COUNT, 300, replace=False)
    idx = np.concatenate([idx, [nn_ref.COUNT - 1]])  # b3
    h = 1e-6
    for q in idx:
        if 9 * nn_ref.H <= q < nn_ref.IN * nn_ref.H:
            continue  # padded input rows: features are zero, gradient zero
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (nn_ref.loss_and_grad(tp, x, t)[0] - nn_ref.loss_and_grad(tm, x, t)[0]) / (2 * h)
        assert abs(fd - grad[q]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (q, fd, grad[q])


def test_padded_inputs_have_zero_gradient():
    rng = np.random.default_rng(2)
    theta = nn_ref.init(3)
    x = rng.uniform(-1, 1, (16, nn_ref.IN))
    x[:, 9:] = 0.0
    _, grad = nn_ref.loss_and_grad(theta, x, rng.uniform(0, 1, 16))
    w0 = grad[:nn_ref.IN * nn_ref.H].reshape(nn_ref.IN, nn_ref.H)
    assert np.all(w0[9:] == 0.0)


def test_features_special_values():
    """Centre node of an odd grid: coordinates 0, so f0..f4 take their
    offsets; f5 and f6..f8 follow g and the trap."""
    f = nn_ref.features((5, 7, 9), (0.3, 0.2, 0.1), (1.0, 1.75, 3.0), math.exp(3.1), [2 * 63 + 3 * 9 + 4])
    assert np.allclose(f[0, :5], [-1, -1, -1, -1, -1])
    assert abs(f[0, 5]) < 1e-15
    assert np.allclose(f[0, 6:9], [-0.6, 0.0, 1.0])
    assert np.all(f[0, 9:] == 0)
    # a node on the x axis at the Thomas-Fermi radius: sum (x/R)^2 = 1 -> f3 = -0.5
    w, g = (1.0, 1.0, 1.0), 100.0
    r = math.sqrt(2 * 0.5 * (15 * g / (4 * math.pi)) ** 0.4)
    n = 201
    d = r / 50.0
    f = nn_ref.features((n, 3, 3), (d, 1, 1), w, g, [(100 + 50) * 9 + 1 * 3 + 1])
    assert abs(f[0, 3] + 0.5) < 1e-12
    assert abs(f[0, 0] - (0.125 * min(r * r, 16.0) - 1.0)) < 1e-12


def test_features_are_even_in_each_coordinate():
    """Mirror nodes (i, j, k) and (n-1-i, n-1-j, n-1-k), and each single
    reflection, have identical features: the network's output is even in x,
    y and z, like the ground state of the symmetric trap on the symmetric grid."""
    shape, d = (6, 7, 8), (0.3, 0.25, 0.2)
    nx, ny, nz = shape
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    site = lambda a, b, c: (a * ny + b) * nz + c
    f = nn_ref.features(shape, d, (1.2, 0.7, 2.1), 40.0, site(i, j, k).ravel())
    for mi, mj, mk in ((nx - 1 - i, j, k), (i, ny - 1 - j, k), (i, j, nz - 1 - k), (nx - 1 - i, ny - 1 - j, nz - 1 - k)):
        assert np.array_equal(f, nn_ref.features(shape, d, (1.2, 0.7, 2.1), 40.0, site(mi, mj, mk).ravel()))
