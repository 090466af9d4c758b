"""A CPU model of the TMA z sweep's schedule (gp_sweep_tma.cuh): which box
each read takes, when boxes are issued and waited, which ring slot a box and
an output tile occupy, and when a slot may be refilled.  It follows the
kernel's control flow step by step on one line and checks, for every chunk
length B, window W and line length N the kernel accepts:
  - every read hits a box that was waited for and still sits in its slot;
  - the Dirichlet end nodes are never used (node 0 is not read, node N-1 is
    replaced by zero), every node 0..N-1 is written exactly once;
  - an output tile is written only into the slot of its own box, after the
    box's last read, and a slot is refilled only after the tile it held was
    stored (the bulk-group count the kernel waits for covers it);
  - the result equals a dense solve to within the window's truncation bound.
This checks the schedule, not the kernel: the GPU parity tests check that."""
import numpy as np
import pytest


def thomas(c, n):
    cp = np.zeros(n, complex)
    ip = np.zeros(n, complex)
    prev = 0
    for t in range(n):
        piv = (1 + 2 * c) + (c * prev if t > 0 else 0)
        ip[t] = 1 / piv
        cp[t] = -c * ip[t]
        prev = cp[t]
    return cp, ip


def dense(psi, c):
    N = len(psi)
    n = N - 2
    r = np.array([c * (psi[t] if t > 0 else 0) + (1 - 2 * c) * psi[t + 1] + c * (psi[t + 2] if t + 2 < N - 1 else 0)
                  for t in range(n)])
    A = np.diag(np.full(n, 1 + 2 * c)) + np.diag(np.full(n - 1, -c), 1) + np.diag(np.full(n - 1, -c), -1)
    out = np.zeros(N, complex)
    out[1:-1] = np.linalg.solve(A, r)
    return out


def model(psi, c, W, B, ahead=2):
    N = len(psi)
    n = N - 2
    cp, ip = thomas(c, n)
    ipm1 = ip - 1
    khi = (W + B + 1) // B
    S = khi + ahead + 1                      # tma_slots
    nbox = (N - 1) // B + 1
    slot = [None] * S
    stored = 0
    state = {"issued": min(ahead + 1, nbox), "waited": 0}
    waited_set = set()
    last_read = {}
    clock = [0]

    def issue(b):
        if b >= S:
            assert stored - 1 - (b - S) >= 0, "slot refilled before its tile was stored"
        slot[b % S] = b

    for b in range(state["issued"]):
        issue(b)

    def need(k):
        if k < state["waited"]:
            return
        while state["waited"] <= k:
            assert state["waited"] < state["issued"]
            waited_set.add(state["waited"])
            state["waited"] += 1
        lim = min(k + ahead + 1, nbox)
        for b in range(state["issued"], lim):
            issue(b)
        state["issued"] = max(state["issued"], lim)

    def rd2(k, col):
        assert col % 2 == 0 and col + 1 < B
        assert k in waited_set and slot[k % S] == k, "read of a box not resident"
        node = k * B + col
        assert node >= 1 or col == 0
        clock[0] += 1
        last_read[k] = clock[0]
        return (psi[node] if node < N else 0), (psi[node + 1] if node + 1 < N else 0)

    out = {}
    written = {}

    def tile(k, vals):
        nonlocal stored
        assert slot[k % S] == k, "tile written over another box"
        clock[0] += 1
        written[k] = clock[0]
        slot[k % S] = ("tile", k)
        for s, v in enumerate(vals):
            if k * B + s < N:
                assert k * B + s not in out
                out[k * B + s] = v
        assert stored == k
        stored += 1

    rhs = lambda pm, p0, p1: p0 + c * (pm + p1 - 2 * p0)
    fwd = lambda r, d, im1: (r + c * d) * (1 + im1)
    back = lambda d, cpt, phi: d - cpt * phi
    carry, D, pm, dprev = 0, [0] * (B + W), 0, 0
    need(0)
    _, p0 = rd2(0, 0)                        # node 0 is not used: pm stays 0
    for t in range(W):
        if t % 2 == 0:
            need((t + 2) // B)
            p1, p1n = rd2((t + 2) // B, (t + 2) % B)
        else:
            p1 = p1n
        dprev = fwd(rhs(pm, p0, p1), dprev, ipm1[t])
        D[t], pm, p0 = dprev, p0, p1
    t0 = 0
    while t0 + B + W <= n:
        j = t0 // B
        need(j + khi)
        last_full = t0 + B + W == n
        for q in range(B):
            if q % 2 == 0:
                p1, p1n = rd2(j + (W + 2 + q) // B, (W + 2 + q) % B)
                if q == B - 2 and last_full:
                    p1n = 0                  # node N-1
            else:
                p1 = p1n
            dprev = fwd(rhs(pm, p0, p1), dprev, ipm1[t0 + W + q])
            D[W + q], pm, p0 = dprev, p0, p1
        phi = D[B + W - 1]
        for q in range(B + W - 2, B - 1, -1):
            phi = back(D[q], cp[t0 + q], phi)
        vals = [None] * B
        for q in range(B - 1, -1, -1):
            phi = back(D[q], cp[t0 + q], phi)
            if q == B - 1:
                nxt = phi
            else:
                vals[q + 1] = phi
        vals[0], carry = carry, nxt
        tile(j, vals)
        D[:W] = D[B:B + W]
        t0 += B
    j, rem = t0 // B, n - t0
    assert W <= rem < B + W
    need(nbox - 1)
    for q in range(B):
        if q < rem - W:
            if q % 2 == 0:
                p1, p1n = rd2(j + (W + 2 + q) // B, (W + 2 + q) % B)
                if q == rem - W - 2:
                    p1n = 0
            else:
                p1 = p1n
            if q == rem - W - 1 and q % 2 == 0:
                p1 = 0
            dprev = fwd(rhs(pm, p0, p1), dprev, ipm1[t0 + W + q])
            D[W + q], pm, p0 = dprev, p0, p1
    phi = 0
    for q in range(B + W - 1, -1, -1):
        if q < rem:
            phi = back(D[q], cp[t0 + q], 0 if q == rem - 1 else phi)
            D[q] = phi
    for kt in range((B + W) // B + 1):
        if (j + kt) * B <= N - 1:
            vals = []
            for s in range(B):
                q = kt * B + s - 1
                vals.append(carry if q < 0 else (D[q] if q < B + W and q < rem else 0))
            tile(j + kt, vals)
    for k, when in written.items():
        assert last_read.get(k, 0) < when, "box read after its slot became a tile"
    assert sorted(out) == list(range(N))
    assert state["waited"] == nbox == state["issued"]
    return np.array([out[i] for i in range(N)])


def kernel_ahead():
    """kTmaAhead as the kernel header defines it."""
    import os
    import re
    hdr = os.path.join(os.path.dirname(__file__), "..", "paper_1601_04641_gb300", "csrc", "gp_sweep_tma.cuh")
    with open(hdr) as f:
        return int(re.search(r"constexpr int kTmaAhead = (\d+);", f.read()).group(1))


def test_kernel_ring_depth_is_modelled():
    assert kernel_ahead() in (1, 2, 3, 4)


@pytest.mark.parametrize("ahead", [1, 2, 3, 4])
@pytest.mark.parametrize("B", [8, 16, 32])  # 64-byte box rows of 8-, 4- and 2-byte elements
@pytest.mark.parametrize("W", [4, 8, 16])
def test_tma_schedule_model(B, W, ahead):
    rng = np.random.default_rng(B * 100 + W)
    step = {8: 2, 16: 4, 32: 8}[B]           # rows must start on 16-byte boundaries
    for N in range(B + W + 4 + (-(B + W + 4)) % step, B + W + 4 + 4 * B + 2, step):
        psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        psi[0], psi[-1] = 7.0, -5.0          # must not enter the solution
        for c in (0.05j, 0.3, 0.02 + 0j):
            got = model(psi, c, W, B, ahead)
            ref = dense(psi, c)
            cpmax = np.abs(thomas(c, N)[0]).max()
            assert np.max(np.abs(got - ref)) <= (4 * cpmax ** (W + 1) + 1e-12) * np.max(np.abs(ref)), (B, W, N, c)
