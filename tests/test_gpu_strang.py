"""Symmetric (Strang) real-time splitting on the GPU against the oracle's
step-by-step form (half kick, sweeps, half kick): graph-replayed blocks,
tracking records (which settle the pending half kick mid-run), reading psi
mid-run and continuing, both precisions, odd and even grids."""
import numpy as np
import pytest

import oracle
from paper_1601_04641_gb300 import build, inputs

pytestmark = pytest.mark.gpu

D = (0.31, 0.27, 0.22)
OMEGA = (1.0, 1.4, 2.0)
DT, G = 0.004, 12.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def make(shape, prec):
    from paper_1601_04641_gb300.solver import GP
    gp = GP(shape, D, DT, OMEGA, G, prec, "complex")
    gp.set_splitting(2)
    return gp


def start(shape, prec):
    psi = inputs.random_field(shape, seed=23)
    oracle.renormalize(psi, D)
    return psi.astype(np.complex64) if prec == "f32" else psi


def tol(prec):
    return 1e-12 if prec == "f64" else 3e-6


@pytest.mark.parametrize("shape", [(37, 29, 41), (36, 30, 42)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("block", [0, 16])
def test_strang_steps_match_oracle(shape, prec, block):
    psi0 = start(shape, prec)
    gp = make(shape, prec)
    gp.set_graph_block(block)
    gp.set_psi(psi0)
    gp.step_real(12)
    got = gp.get_psi().astype(np.complex128)
    gp.close()
    ref = psi0.astype(np.complex128)
    oracle.step_strang(ref, D, DT, OMEGA, G, 12)
    assert float(np.max(np.abs(got - ref))) <= tol(prec) * float(np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_strang_reads_and_tracking_mid_run(prec):
    """Reading psi after 7 steps applies the pending half kick; 5 more steps
    then end where 12 uninterrupted steps end.  Tracking records every 4 steps
    (inside graph blocks) equal the oracle's observables at those steps."""
    shape = (36, 30, 42)
    psi0 = start(shape, prec)
    gp = make(shape, prec)
    gp.set_psi(psi0)
    gp.step_real(7)
    mid = gp.get_psi().astype(np.complex128)
    gp.step_real(5)
    got = gp.get_psi().astype(np.complex128)
    gp.close()
    ref = psi0.astype(np.complex128)
    oracle.step_strang(ref, D, DT, OMEGA, G, 7)
    assert float(np.max(np.abs(mid - ref))) <= tol(prec) * float(np.max(np.abs(ref)))
    oracle.step_strang(ref, D, DT, OMEGA, G, 5)
    assert float(np.max(np.abs(got - ref))) <= tol(prec) * float(np.max(np.abs(ref)))

    gp = make(shape, prec)
    gp.set_psi(psi0)
    gp.set_tracking(4, 16)
    gp.step_real(12)
    recs = gp.tracking()
    gp.close()
    assert [r["step"] for r in recs] == [4, 8, 12]
    ref = psi0.astype(np.complex128)
    for r in recs:
        oracle.step_strang(ref, D, DT, OMEGA, G, 4)
        o = oracle.observables(ref, D, OMEGA, G)
        for key in ("norm", "energy", "mu"):
            assert abs(r[key] - o[key]) <= (1e-12 if prec == "f64" else 2e-6) * abs(o[key]), (r["step"], key)


def test_strang_keeps_norm_and_switches_back():
    """Real-time symmetric steps keep the norm (FP64, 200 steps); switching
    back to order 1 settles the pending half kick first, so the result equals
    200 symmetric steps followed by 10 Lie steps of the oracle."""
    shape = (24, 20, 18)
    psi0 = start(shape, "f64")
    gp = make(shape, "f64")
    gp.set_psi(psi0)
    gp.step_real(200)
    assert abs(gp.observables()["norm"] - 1.0) <= 1e-12
    gp.set_splitting(1)
    gp.step_real(10)
    got = gp.get_psi()
    gp.close()
    ref = psi0.copy()
    oracle.step_strang(ref, D, DT, OMEGA, G, 200)
    oracle.step(ref, D, DT, OMEGA, G, True, 10)
    assert float(np.max(np.abs(got - ref))) <= 1e-12 * float(np.max(np.abs(ref)))
