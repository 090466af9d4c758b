"""Writes the stored expected values under tests/golden/ by calling the CPU
oracle only (never the CUDA path).

    python tests/golden/make_golden.py

imag_small_oracle.json: the 64x48x40 imaginary-time workload (d = 0.2,
dt = 0.004, trap (1, 1.4, 2), g = 10, Gaussian start, renormalisation every
step): observables after 0, 1, 10, 100 and 300 steps, plus psi at 64 seeded
sample sites after 300 steps.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1601_04641_gb300 import inputs  # noqa: E402


def imag_small():
    p = inputs.imag_small()
    psi = oracle.gaussian(p.shape, p.d, p.omega)
    record = {"problem": {"shape": p.shape, "d": p.d, "dt": p.dt, "omega": p.omega, "g": p.g},
              "checkpoints": {}}
    done = 0
    for target in (0, 1, 10, 100, 300):
        oracle.step(psi, p.d, p.dt, p.omega, p.g, False, target - done)
        done = target
        record["checkpoints"][str(target)] = oracle.observables(psi, p.d, p.omega, p.g)
    rng = np.random.default_rng(1234)
    idx = [tuple(int(rng.integers(1, n - 1)) for n in p.shape) for _ in range(64)]
    record["samples_after_300"] = [{"site": list(s), "re": float(psi[s].real), "im": float(psi[s].imag)}
                                   for s in idx]
    return record


def main():
    out = os.path.join(HERE, "imag_small_oracle.json")
    with open(out, "w") as f:
        json.dump(imag_small(), f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
