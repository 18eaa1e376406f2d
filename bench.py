"""Benchmark: MPC solves of MPPI on jump diffusions through libmppi_jump.so.

A step is one MPC solve (all iterations of rollout + weights + update, then
the shift) of the quadrotor workload: K=4096 rollouts, T=100 steps of
0.01 s, 10 iterations, velocity jumps at 2/s, float32 noise.  The headline
`value` is trajectory-steps per second (K * T * iterations per solve) with the
inputs resident in device memory; `e2e` is the same metric through the
synchronous C call with host x0 in and host u0 out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload quadrotor_k4096|cartpole_k1000|large_quadrotor]

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the only other place this script runs it).
Under torchrun each rank solves its own independent problem (seed offset by
rank): weak scaling, no collective in the data path; the timed region is
bracketed by barriers and the maximum over ranks is reported.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1807_06108_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "quadrotor_k4096": W.quadrotor_k4096,
    "cartpole_k1000": W.cartpole_k1000,
    "large_quadrotor": W.large_quadrotor,
}

# Source-level lane operations per trajectory step (each 32-bit integer or
# float32 add / mul / fma / xor / compare / select counts 1; the accurate log
# 8, sqrt 4, sincospi 20; the hardware __sincosf 3 and __fdividef 2), counted
# from the kernel source: SEQ = cost + plant + Euler step of the sequential
# rollout kernel, NOISE = Philox, Box-Muller, perturbation and jump count of
# the sampling kernel.  The fused tile does both in one kernel.
SEQ_OPS_PER_STEP = {"cartpole": 64.0, "quadrotor": 154.0}
NOISE_OPS_PER_STEP = {"cartpole": 79.0, "quadrotor": 218.0}
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([v.strip() for v in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    backend = "nccl"
    dist.init_process_group(backend=backend)
    return dist, dist.get_rank(), ws


def _max_over_ranks(dist, value):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def cpu_baseline(prob, budget_s=10.0):
    """Time the FP64 oracle (as it stands) on a bounded sample: whole MPC
    solves of the same problem until `budget_s` has elapsed (at least one)."""
    import oracle
    oracle.build()
    x0, U = W.initial_state(prob), W.initial_controls(prob)
    iters = prob["iters"]
    solves = 0
    t0 = time.perf_counter()
    it = 0
    while True:
        oracle.step(prob, x0, U, it, iters)
        it += iters
        solves += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    steps = prob["K"] * prob["T"] * iters * solves
    return {"value": steps / dt, "unit": "trajectory-steps/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{solves} full MPC solve(s) of {prob['name']} ({iters} iterations each) "
                      f"in {dt:.1f} s, FP64, OpenMP over rollouts",
            "solves_per_s": solves / dt}


def run_reference(args):
    dist, rank, ws = _dist()
    if rank != 0:
        return
    prob = WORKLOADS[args.workload]()
    budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(prob, budget_s=0.0)
    vals = [cpu_baseline(prob, budget_s=budget) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    ms = 1000.0 * prob["K"] * prob["T"] * prob["iters"] / v
    line = {
        "impl": "reference", "metric": "trajectory-steps/s (MPC solves of MPPI on jump diffusions)",
        "value": v, "unit": "trajectory-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": prob["name"], "K": prob["K"], "T": prob["T"],
                   "iters": prob["iters"], "solves_per_s": v / (prob["K"] * prob["T"] * prob["iters"])},
        "cpu_baseline": {"value": v, "unit": "trajectory-steps/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_1807_06108_gb300 import mppi

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    base = WORKLOADS[args.workload]()
    prob = WORKLOADS[args.workload](seed=base["seed"] + (rank << 40), name=base["name"])
    iters = prob["iters"]
    K, T = prob["K"], prob["T"]
    steps_per_solve = K * T * iters
    stream = torch.cuda.Stream()
    solver = mppi.Solver(prob, stream=stream)
    ctx = solver.ctx
    x0 = W.initial_state(prob)
    solver.set_x0(x0)
    with torch.cuda.stream(stream):
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]

    def one_step():
        mppi.mppi_jump_step_async(ctx, solver.x0.data_ptr(), iters, solver.u0.data_ptr())

    # rollout tile chosen by the library's autotuner (U and counter restored)
    tile, tile_ms = mppi.mppi_jump_autotune(ctx, solver.x0.data_ptr(), iters, reps=5)

    # warm-up (captures the graph)
    for _ in range(args.warmup):
        one_step()
    stream.synchronize()

    # ---- timed region A: device-resident inputs, L2 flushed between steps
    _barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                one_step()
                ev[i][1].record(stream)
        torch.cuda.synchronize()
    _barrier(dist)
    t_steps = [a.elapsed_time(b) for a, b in ev]
    total_ms = _max_over_ranks(dist, sum(t_steps))
    ms_per_step = total_ms / args.steps
    value = ws * steps_per_solve * args.steps / (total_ms / 1e3)

    # ---- timed region B: same steps with phase events inside the graph
    mppi.mppi_jump_enable_timing(ctx, True)
    for _ in range(max(1, args.warmup)):
        one_step()
    stream.synchronize()
    roll_ms, upd_ms, n_it = 0.0, 0.0, 0
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        one_step()
        r, u, n = mppi.mppi_jump_phase_times(ctx)
        roll_ms += r
        upd_ms += u
        n_it += n
    mppi.mppi_jump_enable_timing(ctx, False)
    roll_avg = roll_ms / n_it
    upd_avg = upd_ms / n_it

    # ---- timed region C: end to end through the synchronous C call
    x_host = np.ascontiguousarray(x0, dtype=np.float32)
    u_host = np.zeros(solver.m, dtype=np.float32)
    for _ in range(2):
        mppi.mppi_jump_step(ctx, x_host, iters, u_host)
    _barrier(dist)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mppi.mppi_jump_step(ctx, x_host, iters, u_host)
    e2e_s = _max_over_ranks(dist, time.perf_counter() - t0)
    e2e = ws * steps_per_solve * args.steps / e2e_s

    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sms * 128 * sm_mhz * 1e6 / 1e12  # T lane-ops/s
    ops_step = SEQ_OPS_PER_STEP[prob["system"]]
    if tile[0] == 1:
        ops_step += NOISE_OPS_PER_STEP[prob["system"]]
    ops = ops_step * K * T
    achieved = ops / (roll_avg / 1e3) / 1e12
    sb = 2 if prob["noise_dtype"] == "bf16" else 4
    m = solver.m
    upd_bytes = K * T * m * sb + 8 * K + 8 * T * m
    upd_gbs = upd_bytes / (upd_avg / 1e3) / 1e9

    clocks = clk.summary()
    if rank != 0:
        solver.close()
        return
    cpu = cpu_baseline(prob, budget_s=args.cpu_budget) if not args.no_cpu else None
    line = {
        "metric": "trajectory-steps/s (MPC solves of MPPI on jump diffusions)",
        "value": value,
        "unit": "trajectory-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": prob["name"], "K": K, "T": T, "iters": iters, "dt": prob["dt"],
                   "noise": prob["noise_dtype"], "jump_rate": prob["nu"],
                   "solves_per_s": value / steps_per_solve,
                   "rollout_tile": {"variant": "fused" if tile[0] == 1 else "split",
                                    "block": tile[1], "chunk": tile[2]},
                   "l2": "flushed between timed steps (write of 2x L2 size)"},
        "e2e": {"value": e2e, "unit": "trajectory-steps/s",
                "h2d_bytes_per_step": 4 * solver.n, "d2h_bytes_per_step": 4 * m + 4,
                "solves_per_s": e2e / steps_per_solve},
        # per iteration: noise + rollout + update kernels (split tile) or
        # rollout + update (fused tile), timed region A only
        "gpu_launches": (3 if tile[0] == 2 else 2) * iters * args.steps,
        "roofline": {"bound": "alu",
                     "kernel": "rollout_split_kernel" if tile[0] == 2 else "rollout_kernel",
                     "achieved": achieved,
                     "peak": alu_peak, "unit": "T lane-ops/s", "frac": achieved / alu_peak,
                     "traffic": None, "avg_launch_ms": roll_avg,
                     "peak_basis": f"{n_sms} SMs x 128 lanes x {sm_mhz:.0f} MHz ({peak_kind} max clock)",
                     "ops_per_trajectory_step": ops_step},
        "roofline_update": {"bound": "hbm", "kernel": "update_kernel",
                            "achieved": upd_gbs, "peak": float(peaks.get("hbm_gbs", 6800.0)),
                            "unit": "GB/s", "frac": upd_gbs / float(peaks.get("hbm_gbs", 6800.0)),
                            "avg_launch_ms": upd_avg, "algorithmic_bytes": upd_bytes,
                            "note": f"{peak_kind} peak"},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    solver.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="quadrotor_k4096")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
