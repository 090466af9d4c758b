"""bench.py's control flow on the host (CPU, no GPU): every step that touches
the device is replaced by a fake, and a failing secondary section must be
reported in the JSON line as {"error": ...} while the headline figures and the
other sections are still printed."""
import json
import types

import pytest

import bench


def test_guarded_passes_results_and_reports_exceptions():
    assert bench.guarded(lambda: {"a": 1}) == {"a": 1}
    assert bench.guarded(lambda: (1, 2, 3)) == (1, 2, 3)

    def boom():
        raise ValueError("no convergence")

    assert bench.guarded(boom) == {"error": "ValueError: no convergence"}
    with pytest.raises(KeyboardInterrupt):
        bench.guarded(lambda: (_ for _ in ()).throw(KeyboardInterrupt()))


class FakeGP:
    def tracking(self):
        return [{"norm": 1.0, "energy": 2.0}, {"norm": 1.0, "energy": 2.0}]

    def observables(self):
        return {"mu": 3.0}

    def close(self):
        pass


def fake_workload(torch, name, steps, warmup, dev):
    if name == "bad_workload":
        raise RuntimeError("planted failure in a secondary workload")
    p = types.SimpleNamespace(name=name, shape=(8, 8, 8), sites=512, dt=1e-3, g=1.0, omega=(1.0, 1.0, 1.0))
    prec = "f64" if name == "f64_workload" else "f32"
    return {"problem": p, "gp": FakeGP(), "prec": prec, "field": "complex", "realtime": True}


class FakeClocks:
    def __init__(self, gpu_id):
        pass

    def start(self):
        pass

    def stop(self):
        pass

    def summary(self):
        return {"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": []}


def planted(*a, **k):
    raise RuntimeError("planted failure")


@pytest.mark.parametrize("tgs_fails", [True, False])
def test_failing_sections_do_not_lose_the_line(monkeypatch, capsys, tgs_fails):
    import torch

    from paper_1601_04641_gb300 import build
    monkeypatch.setattr(torch.cuda, "set_device", lambda dev: None)
    monkeypatch.setattr(build, "build", lambda: None)
    monkeypatch.setattr(bench, "time_workload", fake_workload)
    monkeypatch.setattr(bench, "ClockSampler", FakeClocks)
    monkeypatch.setattr(bench, "gpu_id_for", lambda torch, dev: 0)
    monkeypatch.setattr(bench, "timed_region", lambda torch, res, steps, dist: 1e-3 * steps)
    monkeypatch.setattr(bench, "kernel_breakdown",
                        lambda torch, res, steps: {"kick_xsweep": 2e-6, "ysweep": 1e-6, "zsweep_norm": 1e-6})
    monkeypatch.setattr(bench, "e2e_region", lambda torch, res, steps, dist: (2e-3 * steps, 64, 8))
    monkeypatch.setattr(bench, "ground_state_of", lambda torch, p, dev: (None, {"mu": 3.0, "last_dmu": 1e-11}))
    monkeypatch.setattr(bench, "precision_vs_fp64", planted)
    monkeypatch.setattr(bench, "symmetric_splitting", lambda torch, dev, steps, warmup: {"ok": steps})
    monkeypatch.setattr(bench, "time_to_ground_state",
                        planted if tgs_fails else lambda torch, dev, count, tol, peak: ({"tgs": count}, [1.5], 5e-5))
    seen = {}

    def fake_warm_start(torch, dev, n_train, n_held, steps, mustar64=None, bar64=None):
        seen["mustar"], seen["bar"] = mustar64, bar64
        return {"ok": n_train}

    monkeypatch.setattr(bench, "warm_start", fake_warm_start)
    monkeypatch.setattr(bench, "cpu_baseline", lambda p, realtime, budget: {"value": 1.0, "cores": 1})
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    args = types.SimpleNamespace(workload="real_large", steps=20, warmup=3, also="good_workload,bad_workload,f64_workload",
                                 also_steps=10, precision=1, strang=1, gs=64, ws_train=5, ws_held=2,
                                 ws_steps=1, no_cpu=False, cpu_budget=1.0)
    assert bench.run_ours(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["value"] == pytest.approx(512 * 20 / 0.02)
    assert line["roofline"]["kernel"] == "kick_xsweep"
    assert line["precision_vs_fp64"] == {"error": "RuntimeError: planted failure"}
    assert line["symmetric_splitting"] == {"ok": 20}
    assert line["warm_start"] == {"ok": 5}
    if tgs_fails:
        assert line["time_to_ground_state"] == {"error": "RuntimeError: planted failure"}
        assert seen["mustar"] is None and seen["bar"] is None  # no reference mu from the failed section
    else:
        assert line["time_to_ground_state"] == {"tgs": 64}
        assert seen["mustar"] == [1.5] and seen["bar"] == 5e-5
    assert line["also"]["bad_workload"] == {"error": "RuntimeError: planted failure in a secondary workload"}
    good = line["also"]["good_workload"]
    assert good["ms_per_step"] == pytest.approx(1.0) and good["mu"] == 3.0 and good["start"]["mu"] == 3.0
    f64 = line["also"]["f64_workload"]
    assert f64["psi"] == "complex128" and f64["fp64_roofline"]["bound"] == "alu"
    assert "fp64_roofline" not in good
    assert line["cpu_baseline"] == {"value": 1.0, "cores": 1}
