"""The two truncations of the line solve (CPU, numpy FP64): windowed back
substitution and segment warm-up, against a dense solve.

The Thomas recurrences contract by |cp| < 1 per node, so
  - a chunk of B outputs whose backward recurrence starts W nodes past the
    chunk with phi ~ dp is off by at most |cp|max^(W+1) max|phi| there;
  - a segment whose forward sweep starts W+1 nodes before it from dp = 0 is
    off by at most |cp|max^(W+2) max|dp| at its first node, decaying after.
The window rule takes the smallest W in {4, 8, 16} with |cp|max^(W+1) <= u/2
(u the unit roundoff of the field's precision), else the exact two-pass
solve, so the truncation stays below the rounding of one operation.  This
model checks the bounds, the rule's outcome on the workloads' coefficients,
and that a window below the rule's is visibly inexact (so the check is not
vacuous)."""
import numpy as np
import pytest

U32 = 2.0 ** -24  # u/2 for FP32


def tables(c, n):
    cp = np.zeros(n, complex)
    ip = np.zeros(n, complex)
    for t in range(n):
        piv = (1 + 2 * c) + (c * cp[t - 1] if t > 0 else 0)
        ip[t] = 1 / piv
        cp[t] = -c * ip[t]
    return cp, ip


def rhs(psi, c):
    """CN right-hand side on the interior nodes (Dirichlet ends read as 0)."""
    p = psi.copy()
    p[0] = p[-1] = 0
    return c * p[:-2] + (1 - 2 * c) * p[1:-1] + c * p[2:]


def dense(psi, c):
    n = len(psi) - 2
    A = (np.diag(np.full(n, 1 + 2 * c)) + np.diag(np.full(n - 1, -c), 1) + np.diag(np.full(n - 1, -c), -1))
    return np.linalg.solve(A, rhs(psi, c))


def segmented_windowed(psi, c, W, B, seg_len):
    """Interior solution by segments of seg_len nodes, each warmed up over
    the W+1 nodes before it from dp = 0, and chunks of B outputs whose
    backward recurrence starts W nodes past the chunk (or at the line's end,
    where it is exact) with phi = dp."""
    n = len(psi) - 2
    cp, ip = tables(c, n)
    r = rhs(psi, c)
    out = np.full(n, np.nan, complex)
    for tb in range(0, n, seg_len):
        te = min(tb + seg_len, n)
        e = min(te + W, n)  # forward values needed up to e-1
        tw = max(0, tb - (W + 1))
        dp = np.zeros(n, complex)
        prev = 0
        for t in range(tw, e):
            dp[t] = (r[t] + c * prev) * ip[t]
            prev = dp[t]
        for t0 in range(tb, te, B):
            t1 = min(t0 + B, te)
            start = min(t1 + W, n) - 1
            phi = dp[start]
            vals = {}
            for t in range(start, t0 - 1, -1):
                if t < start:
                    phi = dp[t] - cp[t] * phi
                if t < t1:
                    vals[t] = phi
            for t in range(t0, t1):
                out[t] = vals[t]
    assert not np.isnan(out).any()
    return out, cp, dp


def field(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n + 2) + 1j * rng.standard_normal(n + 2)


@pytest.mark.parametrize("c", [0.025, 0.25, 0.005j, 0.05j, 0.2 + 0.1j])
@pytest.mark.parametrize("W", [1, 2, 4, 8])
@pytest.mark.parametrize("n, seg_len", [(37, 37), (130, 64), (257, 32), (90, 13)])
def test_truncation_bounds(c, W, n, seg_len):
    psi = field(n, 3)
    exact = dense(psi, c)
    got, cp, _ = segmented_windowed(psi, c, W, 16, seg_len)
    k = np.max(np.abs(cp))
    # forward values of the exact solve bound the warm-up term
    _, _, dp_full = segmented_windowed(psi, c, 0, 16, n)
    bound = (k ** (W + 1) * np.max(np.abs(exact)) + k ** (W + 2) * np.max(np.abs(dp_full))) / (1 - k) ** 2
    err = np.max(np.abs(got - exact))
    assert err <= 2 * bound + 1e-13 * np.max(np.abs(exact)), (err, bound)


def smallest_window(kmax, half_u):
    for W in (4, 8, 16):
        if kmax ** (W + 1) <= half_u:
            return W
    return 0


@pytest.mark.parametrize("c, want", [(0.1 / 4, 4),            # imaginary time, dt = 0.1 d^2
                                     (1.0 / 4, 16),           # dt = d^2, a schedule's coarse level
                                     (0.02 / 4 * 1j, 4),      # real time, dt = 0.02 d^2 (the quench)
                                     (10.0 / 4, 0)])          # dt = 10 d^2: the exact solve
def test_window_rule_keeps_fp32_truncation_below_rounding(c, want):
    n = 200
    psi = field(n, 5)
    cp, _ = tables(c, n)
    W = smallest_window(np.max(np.abs(cp)), U32)
    assert W == want
    if W == 0:
        return
    exact = dense(psi, c)
    scale = np.max(np.abs(exact))
    got, _, _ = segmented_windowed(psi, c, W, 16, 64)
    assert np.max(np.abs(got - exact)) <= 4 * U32 * scale
    # a window below the rule's is inexact at FP32's resolution
    low, _, _ = segmented_windowed(psi, c, max(1, W // 4), 16, 64)
    assert np.max(np.abs(low - exact)) > 4 * U32 * scale
