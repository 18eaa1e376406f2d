"""Benchmark: MPC solves of MPPI on jump diffusions through libmppi_jump.so.

A step is one MPC solve (all iterations of rollout + weights + update, then
the shift) of the quadrotor workload: K=4096 rollouts, T=100 steps of
0.01 s, 10 iterations, velocity jumps at 2/s, float32 noise.  The headline
`value` is trajectory-steps per second (K * T * iterations per solve) with the
inputs resident in device memory; `e2e` is the same metric through the
synchronous C call with host x0 in and host u0 out.  The line also carries
the batched form (256 uneven instances in one persistent launch, against one
instance per launch) and the served form (a Poisson request stream over 64
sessions: solves/s, p50/p99 latency).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload quadrotor_k4096|cartpole_k1000|large_quadrotor]
                  [--no-cpu] [--no-extras]

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the only other place this script runs it).
Under torchrun each rank solves its own independent problem (rank-specific
Philox key): weak scaling, no collective in the data path; the timed region
is bracketed by barriers and the maximum over ranks is reported.
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

from paper_1807_06108_gb300 import dist as D  # noqa: E402
from paper_1807_06108_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "quadrotor_k4096": W.quadrotor_k4096,
    "cartpole_k1000": W.cartpole_k1000,
    "large_quadrotor": W.large_quadrotor,
    "quadrotor_alg1": W.quadrotor_alg1,
}
METRIC = "trajectory-steps/s (MPC solves of MPPI on jump diffusions)"

# Source-level lane operations per trajectory step (each 32-bit integer or
# float32 add / mul / fma / xor / compare / select counts 1; the accurate log
# 8, sqrt 4, sincospi 20; the hardware __sincosf 3 and __fdividef 2), counted
# from the kernel source: SEQ = cost + plant + Euler step of the sequential
# rollout kernel, NOISE = Philox, Box-Muller, perturbation and jump count of
# the sampling kernel.  The fused tile does both in one kernel.
SEQ_OPS_PER_STEP = {"cartpole": 64.0, "quadrotor": 154.0}
NOISE_OPS_PER_STEP = {"cartpole": 79.0, "quadrotor": 218.0}
L2_BYTES = 129 * 1024 * 1024


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as
# it stands (profiles/quadrotor_K4096_T100_it10_kernels.md,
# profiles/quadrotor_K65536_T200_it5_bf16_kernels.md); None where no capture
# of the current kernel exists.
NCU_TRAFFIC = {
    ("quadrotor_K4096_T100_it10", "rollout_staged_kernel"): 13131264 + 0,
    ("quadrotor_K4096_T100_it10", "update_kernel"): 6630144 + 0,
    ("quadrotor_K65536_T200_it5_bf16", "rollout_staged_kernel"): 314606080 + 3444224,
    ("quadrotor_K65536_T200_it5_bf16", "update_kernel"): 105188864 + 2972928,
}

VARIANT_NAMES = {1: "fused", 2: "split", 3: "staged"}
ROLLOUT_KERNELS = {1: "rollout_kernel", 2: "rollout_split_kernel", 3: "rollout_staged_kernel"}


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
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._proc = None
        self._t = None
        self._first = threading.Event()

    def _run(self):
        for line in self._proc.stdout:
            vals = [v.strip() for v in line.strip().split(",")]
            if len(vals) >= 2:
                self.samples.append(vals)
                self._first.set()

    def __enter__(self):
        # one nvidia-smi process sampling every 100 ms; the region starts
        # once its first sample has arrived
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return self
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        self._first.wait(timeout=10)
        self.samples.clear()  # the idle sample before the region
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self._proc.kill()
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [x for x in (num(s[0]) for s in self.samples) if x is not None]
        mx = [x for x in (num(s[1]) for s in self.samples) if x is not None]
        reasons = sorted({self.NAMES[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    dist.init_process_group(backend="nccl")
    return dist, dist.get_rank(), ws


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def cpu_baseline(prob, budget_s=10.0):
    """Time the FP64 oracle (as it stands) on a bounded sample: whole MPC
    solves of the same problem until `budget_s` has elapsed (at least one).
    Also returns the first solve's (u0, U) for the accuracy check."""
    import oracle
    oracle.build()
    x0, U = W.initial_state(prob), W.initial_controls(prob)
    iters = prob["iters"]
    solves = 0
    first = None
    t0 = time.perf_counter()
    it = 0
    while True:
        res = oracle.step(prob, x0, U, it, iters)
        if first is None:
            first = res
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
            "solves_per_s": solves / dt}, first


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    Each step is one MPC solve of a bounded sample of the workload -- its
    first Ks rollouts (the same Philox streams as the full problem), Ks sized
    so that the whole run takes about a minute."""
    dist, rank, ws = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    prob = WORKLOADS[args.workload]()
    K, T, iters = prob["K"], prob["T"], prob["iters"]
    x0, U = W.initial_state(prob), W.initial_controls(prob)
    # calibrate: one solve on min(K, 256) rollouts
    kc = min(K, 256)
    t0 = time.perf_counter()
    oracle.step(dict(prob, K=kc), x0, U, 0, iters)
    rate = kc * T * iters / max(time.perf_counter() - t0, 1e-6)
    per_step = 60.0 / max(1, args.steps + args.warmup)
    Ks = int(min(K, max(32, rate * per_step / (T * iters))))
    sample = dict(prob, K=Ks)
    it = 0
    for _ in range(args.warmup):
        oracle.step(sample, x0, U, it, iters)
        it += iters
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step(sample, x0, U, it, iters)
        times.append(time.perf_counter() - t0)
        it += iters
    total = sum(times)
    v = Ks * T * iters * args.steps / total
    desc = (f"{args.steps} MPC solves of the first {Ks} of {K} rollouts of {prob['name']} "
            f"({iters} iterations each) in {total:.1f} s, FP64, OpenMP over rollouts")
    line = {
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "trajectory-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * K * T * iters / v,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": prob["name"], "K": K, "T": T, "iters": iters,
                   "solves_per_s": v / (K * T * iters), "sample_rollouts": Ks},
        "cpu_baseline": {"value": v, "unit": "trajectory-steps/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "trajectory-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _update_error(prob, first):
    """Max |dU_gpu - dU_oracle| / max |dU_oracle| of one MPC solve from the
    initial state (the oracle's side comes from the CPU-baseline run)."""
    from paper_1807_06108_gb300 import mppi
    s = mppi.Solver(prob)
    try:
        u0 = s.step(W.initial_state(prob))
        U = s.controls().astype(np.float64)
    finally:
        s.close()
    u0_ref, U_ref = first
    U0 = W.initial_controls(prob).astype(np.float64)
    den = max(np.max(np.abs(U_ref[:-1] - U0[1:])), np.max(np.abs(u0_ref - U0[0])), 1e-30)
    return float(max(np.max(np.abs(U[:-1] - U_ref[:-1])), np.max(np.abs(u0 - u0_ref))) / den)


def bench_batched(reps=5):
    """256 uneven instances: one persistent launch per batched step, against
    the same instances solved one per launch."""
    import torch
    from paper_1807_06108_gb300 import mppi
    probs = W.batched_instances()
    b = mppi.Batch(probs)
    try:
        b.set_states([W.initial_state(p) for p in probs])
        block, _ = b.autotune(reps=2)
        info = b.info()
        b.step_async()
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        for _ in range(reps):
            b.step_async()
        e1.record(b.stream)
        b.sync()
        ms = e0.elapsed_time(e1) / reps
    finally:
        b.close()
    s = torch.cuda.Stream()
    solvers = [mppi.Solver(p, stream=s) for p in probs]
    try:
        for sv, p in zip(solvers, probs):
            sv.set_x0(W.initial_state(p))

        def plain_round():
            for sv, p in zip(solvers, probs):
                mppi.mppi_jump_step_async(sv.ctx, sv.x0.data_ptr(), p["iters"], sv.u0.data_ptr())

        plain_round()
        s.synchronize()
        e0.record(s)
        plain_round()
        e1.record(s)
        s.synchronize()
        plain_ms = e0.elapsed_time(e1)
    finally:
        for sv in solvers:
            sv.close()
    n = len(probs)
    return {"workload": "256 instances, half cart-pole half quadrotor, K in {512..8192}, "
                        "T in [30,150], jump rate U[0.5,3]/s, bf16 noise",
            "ms_per_batched_step": ms, "solves_per_s": n / ms * 1e3,
            "trajectory_steps_per_s": info["steps_per_solve"] / ms * 1e3,
            "one_instance_per_launch_ms": plain_ms,
            "one_instance_per_launch_solves_per_s": n / plain_ms * 1e3,
            "speedup": plain_ms / ms, "block": block, "work_items": info["items"],
            "grid": info["grid"]}


def bench_served(duration_s=3.0, rate_hz=2000.0):
    """Poisson requests over 64 sessions (one MPC step each, warm-started from
    the session's device state), admitted under a 20 GB budget."""
    from paper_1807_06108_gb300 import mppi
    probs = W.served_sessions()
    srv = mppi.Server(probs, budget_bytes=20 << 30, max_inflight=32)
    try:
        rng = np.random.default_rng(0)
        states = [W.initial_state(p).astype(np.float32) for p in probs]
        for i in range(len(probs)):  # first request per session: graph capture
            srv.submit(i, states[i])
        srv.drain()
        srv.reset_stats()
        t_arr, sess = W.arrival_trace(rate_hz, duration_s, len(probs), seed=0)
        t0 = time.perf_counter()
        for t, s in zip(t_arr, sess):
            while time.perf_counter() - t0 < t:
                pass
            states[s] = states[s] + W.state_drift(probs[s], rng)
            srv.submit(int(s), states[s])
        srv.drain(600)
        st = srv.stats()
    finally:
        srv.close()
    return {"workload": f"64 sessions (cart-pole 1 / quadrotor 10 iterations, K in {{1024..16384}}, "
                        f"T in {{50..200}}), Poisson arrivals {rate_hz:.0f}/s for {duration_s:.0f} s, "
                        "20 GB budget",
            "requests": st["completed"], "solves_per_s": st["completed"] / max(st["span_s"], 1e-9),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "evictions": st["evictions"], "resident_gb": st["resident_bytes"] / 1e9}


def run_ours(args):
    import torch
    from paper_1807_06108_gb300 import mppi

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    base = WORKLOADS[args.workload]()
    prob = WORKLOADS[args.workload](seed=D.rank_seed(base["seed"], rank), name=base["name"])
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

    # the library's default rollout tile, or the one its autotuner picks (U
    # and counter restored); a fixed default keeps runs under a profiler on
    # the same kernels as the plain run
    if args.autotune:
        tile, _ = mppi.mppi_jump_autotune(ctx, solver.x0.data_ptr(), iters, reps=5)
    else:
        if args.tile:
            mppi.mppi_jump_set_tuning(ctx, *[int(v) for v in args.tile.split(",")])
        tile = mppi.mppi_jump_get_tuning(ctx)
    for _ in range(args.warmup):  # warm-up (captures the graph)
        one_step()
    stream.synchronize()

    # clocks sampled across the three timed regions below (all under load)
    clk = ClockSampler(local).__enter__()

    # ---- timed region A: device-resident inputs, L2 flushed between steps
    _barrier(dist)
    torch.cuda.synchronize()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    _barrier(dist)
    total_ms = D.max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev), "cuda")
    ms_per_step = total_ms / args.steps
    value = ws * steps_per_solve * args.steps / (total_ms / 1e3)

    # ---- timed region B: the same steps with phase events inside the graph
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
    e2e_s = D.max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    clk.__exit__(None, None, None)
    e2e = ws * steps_per_solve * args.steps / e2e_s

    # ---- region D: the update kernel on its own (same launch configuration):
    # inside the step it shares the GPU with the next iteration's noise pass,
    # which blurs its bandwidth figure.  Each launch follows a fresh
    # rollout_cost (which arms the running minimum) and an L2 flush.
    n_iso = min(args.steps, 50)
    iso_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n_iso)]
    for i in range(n_iso + 3):
        solver.rollout_cost(x0, want_costs=False)
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            if i >= 3:
                iso_ev[i - 3][0].record(stream)
            mppi.mppi_jump_update(ctx)
            if i >= 3:
                iso_ev[i - 3][1].record(stream)
    stream.synchronize()
    upd_iso_ms = sum(a.elapsed_time(b) for a, b in iso_ev) / n_iso
    solver.close()

    peaks, peak_kind = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sms * 128 * sm_mhz * 1e6 / 1e12  # T lane-ops/s
    ops_step = SEQ_OPS_PER_STEP[prob["system"]]
    if tile[0] == 1:
        ops_step += NOISE_OPS_PER_STEP[prob["system"]]
    achieved = ops_step * K * T / (roll_avg / 1e3) / 1e12
    sb = 2 if prob["noise_dtype"] == "bf16" else 4
    m = 1 if prob["system"] == "cartpole" else 4
    upd_bytes = K * T * m * sb + 8 * K + 8 * T * m
    upd_gbs = upd_bytes / (upd_iso_ms / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    clocks = clk.summary()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        cpu, first = cpu_baseline(prob, budget_s=args.cpu_budget)
        cpu["update_rel_err_vs_oracle"] = _update_error(prob, first)
    extras = {}
    if not args.no_extras:
        extras["batched"] = bench_batched()
        extras["served"] = bench_served(duration_s=args.served_seconds)
    line = {
        "metric": METRIC,
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
                   "rollout_tile": {"variant": VARIANT_NAMES[tile[0]],
                                    "block": tile[1], "chunk": tile[2]},
                   "l2": "flushed between timed steps (write of 2x L2 size)"},
        "e2e": {"value": e2e, "unit": "trajectory-steps/s",
                "h2d_bytes_per_step": 4 * len(x0), "d2h_bytes_per_step": 4 * m + 4,
                "solves_per_s": e2e / steps_per_solve},
        # per iteration: noise + rollout + update kernels (split tile) or
        # rollout + update (fused tile), timed region A only
        "gpu_launches": (2 if tile[0] == 1 else 3) * iters * args.steps,
        "roofline": {"bound": "alu",
                     "kernel": ROLLOUT_KERNELS[tile[0]],
                     "achieved": achieved, "peak": alu_peak, "unit": "T lane-ops/s",
                     "frac": achieved / alu_peak,
                     "traffic": NCU_TRAFFIC.get((prob["name"], ROLLOUT_KERNELS[tile[0]])),
                     "avg_launch_ms": roll_avg,
                     "peak_basis": f"{n_sms} SMs x 128 lanes x {sm_mhz:.0f} MHz "
                                   f"({peak_kind} max clock)",
                     "ops_per_trajectory_step": ops_step},
        "roofline_update": {"bound": "hbm", "kernel": "update_kernel", "achieved": upd_gbs,
                            "peak": hbm, "unit": "GB/s", "frac": upd_gbs / hbm,
                            "avg_launch_ms": upd_iso_ms, "algorithmic_bytes": upd_bytes,
                            "in_step_avg_launch_ms": upd_avg,
                            "traffic": NCU_TRAFFIC.get((prob["name"], "update_kernel")),
                            "note": f"{peak_kind} peak; timed alone after an L2 flush "
                                    "(in the step it overlaps the next noise pass)"},
        "clocks": clocks,
        "cpu_baseline": cpu,
        **extras,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="quadrotor_k4096")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="time the rollout tile the library's autotuner picks")
    ap.add_argument("--tile", default="",
                    help="rollout tile 'variant,block,chunk' (1 fused, 2 split, 3 staged)")
    ap.add_argument("--served-seconds", type=float, default=3.0,
                    help="length of the served leg's Poisson arrival trace (the workload "
                         "description's full trace is 60 s)")
    ap.add_argument("--only", choices=["batched", "served"],
                    help="run only the batched or served measurement (for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        res = bench_batched() if args.only == "batched" else bench_served(duration_s=args.served_seconds)
        print(json.dumps({args.only: res}), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
