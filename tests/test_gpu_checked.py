"""The MPPI_CHECK_BOUNDS debug build on tiny configurations (K <= 8,
T <= 4), every rollout tile, both plants and jump channels: in a process
that loads libmppi_jump_checked.so, no kernel's launch check fires (status
MPPI_OK at every synchronisation) and the results match the FP64 oracle
element by element, as the normal build's do."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1807_06108_gb300 import mppi, workloads as W
from tests import parity
assert mppi.LIB_PATH.endswith("libmppi_jump_checked.so"), mppi.LIB_PATH
out = []
cases = [
    W.cartpole_k1000(K=8, T=4, nu=30.0, name="cp"),
    W.cartpole_k1000(K=5, T=3, nu=30.0, noise_dtype="bf16", jump_channel="control", name="cp_ctl"),
    W.quadrotor_k4096(K=8, T=4, nu=40.0, lam=20.0, name="qr"),
    W.quadrotor_k4096(K=7, T=4, nu=40.0, lam=20.0, jump_rows=[0, 1, 2], noise_dtype="bf16", name="qr_rows"),
]
for prob in cases:
    rng = np.random.default_rng(1)
    x0, U = W.random_state(prob, rng, 0.1), W.random_controls(prob, rng, 0.2)
    for tile in [(1, 32, 4), (2, 32, 2), (3, 32, 4), (4, 32, 4), (3, 64, 16)]:
        rep = parity.run_and_compare(prob, x0, U, 2, tile=tile)
        out.append([prob["name"], list(tile), rep["update_rel_err"]])
    s = mppi.Solver(prob)
    try:
        u0 = s.step(x0)          # the graph step; raises on any non-OK status
        s.sync()
    finally:
        s.close()
print(json.dumps(out))
'''


def test_checked_build_runs_clean_and_matches_oracle(cuda):
    from paper_1807_06108_gb300 import build as B
    lib = B.build(checked=True)
    env = dict(os.environ, MPPI_JUMP_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    rows = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(rows) == 20
    assert all(err <= 1e-4 for _, _, err in rows)
