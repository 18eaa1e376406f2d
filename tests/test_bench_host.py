"""Host-side checks of bench.py (no GPU): the helpers that name the update
kernel and count a step's launches, and the reference arm, which times the
FP64 oracle on the host cores and prints one JSON line of the benchmark
contract."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1807_06108_gb300 import workloads as W  # noqa: E402


def test_update_kernel_name_follows_the_single_block_rule():
    # cart-pole K = 1000, T = 50, FP32: 200 KB of perturbations, one block
    assert bench._update_kernel_name(W.cartpole_k1000(), (3, 96, 16)) == "update_small_kernel"
    # the block-record tile always combines records with update_kernel
    assert bench._update_kernel_name(W.cartpole_k1000(), (4, 96, 16)) == "update_kernel"
    assert bench._update_kernel_name(W.quadrotor_k4096(), (3, 96, 16)) == "update_kernel"
    assert bench._update_kernel_name(W.large_quadrotor(), (3, 128, 8)) == "update_kernel"


def test_launches_per_iteration():
    # sparse state-jump records (512 rollout blocks of 128 > 152 SMs): noise,
    # marks, rollout, update
    assert bench._launches_per_iteration(W.large_quadrotor(), (3, 128, 8), 152) == 4
    # dense records: noise, rollout, update
    assert bench._launches_per_iteration(W.quadrotor_k4096(), (3, 96, 16), 152) == 3
    assert bench._launches_per_iteration(W.cartpole_k1000(), (3, 96, 16), 152) == 3
    # fused tile: rollout and update
    assert bench._launches_per_iteration(W.large_quadrotor(), (1, 128, 8), 152) == 2


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["config"]["workload"] == "quadrotor_K65536_T200_it5_bf16"
    assert d["unit"] == "trajectory-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
