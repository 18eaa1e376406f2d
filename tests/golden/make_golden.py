"""Writes tests/golden/oracle_small_iterations.json: the FP64 oracle's output
for a few small, fixed-seed iterations (rollout costs, jump counts, updated
controls, weights diagnostics).  It calls only the oracle and the seeded input
generators; the stored values are a regression record of the oracle (and of
its agreement across host platforms), not an independent pin -- the pins are
the tests in tests/test_oracle_*.py.

    python tests/golden/make_golden.py
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1807_06108_gb300 import workloads as W  # noqa: E402


def cases():
    return {
        "cartpole_K24_T9": (W.cartpole_k1000(K=24, T=9, nu=20.0), 3),
        "quadrotor_K16_T7_laplace_bf16": (
            W.quadrotor_k4096(K=16, T=7, nu=30.0, mark_law="laplace", noise_dtype="bf16"), 11),
        "quadrotor_K8_T5_control": (
            W.quadrotor_k4096(K=8, T=5, nu=40.0, jump_channel="control", c=2.0), 0),
    }


def compute(prob, it):
    rng = np.random.default_rng(1234)
    x0 = W.random_state(prob, rng, 0.2).astype(np.float64)
    U = W.random_controls(prob, rng, 0.3).astype(np.float64)
    r = oracle.iteration(prob, x0, U, it, want_counts=True)
    return {"x0": x0.tolist(), "U_in": U.tolist(), "it": it, "S": r["S"].tolist(),
            "counts": r["counts"].astype(int).tolist(), "U": r["U"].tolist(),
            "diag": r["diag"].tolist()}


def main():
    out = {"source": "tests/golden/make_golden.py (FP64 oracle, Algorithm 1 one iteration)",
           "cases": {name: compute(p, it) for name, (p, it) in cases().items()}}
    with open(os.path.join(HERE, "oracle_small_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
