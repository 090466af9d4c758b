"""Learned warm start on the GPU: tensor-core forward/backward kernels against
the FP64 numpy reference, training, and the gain over the Gaussian start."""
import numpy as np
import pytest

import oracle
from oracle import nn_ref
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def small_set(count, seed, shape=(14, 12, 10)):
    ps = inputs.batch_problems(count, seed=seed, g_max=300.0)
    return [inputs.sized_box(shape, p.omega, p.g) for p in ps]


def upload_targets(problems):
    """Oracle Gaussian amplitudes as float32 targets on the device."""
    import torch
    arrays = [np.abs(oracle.gaussian(p.shape, p.d, p.omega)).astype(np.float32).ravel() for p in problems]
    offsets = np.concatenate([[0], np.cumsum([a.size for a in arrays])[:-1]])
    data = torch.tensor(np.concatenate(arrays), device="cuda")
    return data, offsets, [float(a.max()) for a in arrays], arrays


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_gradients_match_fp64_reference():
    """GPU loss and gradients (BF16 tensor-core operands, FP32 accumulation)
    against the FP64 reference on the same parameters and samples: relative
    L2 of every parameter tensor within 2e-2."""
    from paper_1601_04641_gb300.warmstart import Net
    probs = small_set(3, seed=4)
    data, offsets, pmax, arrays = upload_targets(probs)
    net = Net(seed=1)
    theta = nn_ref.init(7).astype(np.float32)
    net.params = theta
    net.set_data(probs, data, offsets, pmax)
    rng = np.random.default_rng(5)
    P = 512
    inst = rng.integers(0, len(probs), P)
    site = np.array([rng.integers(0, probs[i].sites) for i in inst])
    loss, grad = net.loss_grad(inst, site)
    x = np.zeros((P, nn_ref.IN))
    t = np.zeros(P)
    for i, p in enumerate(probs):
        sel = inst == i
        x[sel] = nn_ref.features(p.shape, p.d, p.omega, p.g, site[sel])
        t[sel] = arrays[i][site[sel]] / pmax[i]
    loss_ref, grad_ref = nn_ref.loss_and_grad(theta.astype(np.float64), x, t)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    off = 0
    for name, n in nn_ref.SIZES:
        assert rel_l2(grad[off:off + n], grad_ref[off:off + n]) <= 2e-2, name
        off += n
    net.close()


def test_prediction_matches_reference_forward():
    from paper_1601_04641_gb300.solver import GP
    from paper_1601_04641_gb300.warmstart import Net
    p = small_set(1, seed=8, shape=(18, 15, 13))[0]
    net = Net(seed=2)
    theta = nn_ref.init(9).astype(np.float32)
    net.params = theta
    gp = GP(p.shape, p.d, p.dt, p.omega, p.g, "f64", "real")
    net.predict(gp)
    got = gp.get_psi()
    x = nn_ref.features(p.shape, p.d, p.omega, p.g, np.arange(p.sites))
    y, _ = nn_ref.forward(theta.astype(np.float64), x)
    ref = y.reshape(p.shape)
    ref[0], ref[-1], ref[:, 0], ref[:, -1], ref[:, :, 0], ref[:, :, -1] = 0, 0, 0, 0, 0, 0
    ref /= np.sqrt(np.prod(p.d) * np.sum(ref ** 2))
    assert rel_l2(got, ref) <= 2e-2
    assert abs(gp.observables()["norm"] - 1.0) <= 1e-12
    net.close()


def test_training_reduces_the_loss():
    from paper_1601_04641_gb300.warmstart import Net
    probs = small_set(6, seed=11)
    data, offsets, pmax, _ = upload_targets(probs)
    net = Net(seed=3)
    net.set_data(probs, data, offsets, pmax)
    first = net.train(1, 8192, 3e-3, seed=1)
    last = net.train(400, 8192, 3e-3, seed=2)
    assert np.isfinite(last) and last < 0.1 * first
    net.close()


def test_warm_start_gain_on_held_out_condensates():
    """Trained on the method's own ground states, the network's start reaches
    |dmu| < 1e-7 in fewer imaginary-time steps than the Gaussian on held-out
    parameters, and both starts reach the same mu (to 1e-5 relative: the stop
    rule leaves a residual of about tol r / (1 - r) for a contraction r per
    check, so two starts stop up to a few tol apart)."""
    from paper_1601_04641_gb300 import warmstart as W
    shape = (40, 32, 28)
    train_p = [inputs.sized_box(shape, p.omega, p.g) for p in inputs.batch_problems(96, seed=21, g_max=500.0)]
    held = [inputs.sized_box(shape, p.omega, p.g) for p in inputs.batch_problems(12, seed=22, g_max=500.0)]
    data, offsets, pmax, _ = W.ground_states(train_p, 1e-7)
    net = W.Net(seed=4)
    net.set_data(train_p, data, offsets, pmax)
    W.train(net, 3000, points=16384)
    r = W.run_from_starts(net, held, 1e-7)
    ratio = np.array(r["steps_gauss"]) / np.array(r["steps_nn"])
    print("warm-start step ratio (gauss / nn): median %.2f min %.2f max %.2f, fallbacks %d" %
          (np.median(ratio), ratio.min(), ratio.max(), sum(r["fallback"])))
    assert np.median(ratio) > 1.2, r
    for a, b in zip(r["mu_gauss"], r["mu_nn"]):
        assert abs(a - b) <= 1e-5 * abs(a)
    net.close()


def test_fallback_to_gaussian_with_corrupted_weights():
    """Weights that make the prediction worse than the Gaussian (here: a flat
    amplitude everywhere) trigger the fallback, and the run then equals the
    Gaussian start's."""
    from paper_1601_04641_gb300 import warmstart as W
    held = small_set(4, seed=31, shape=(20, 18, 16))
    net = W.Net(seed=5)
    theta = np.zeros(nn_ref.COUNT, dtype=np.float32)
    theta[-1] = 5.0  # b3: softplus(5) everywhere
    net.params = theta
    r = W.run_from_starts(net, held, 1e-7)
    assert all(r["fallback"])
    assert r["steps_nn"] == r["steps_gauss"]
    net.close()
