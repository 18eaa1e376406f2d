"""Benchmark: MPC solves of MPPI on jump diffusions through libmppi_jump.so.

A step is one MPC solve (all iterations of noise + rollout + weights +
update, then the shift) of the large quadrotor workload: K = 65536
rollouts, T = 200 steps of 0.005 s, 5 iterations, Laplace velocity jumps at
5/s, bfloat16 noise storage with float32 dynamics -- the largest single-GPU
workload.  The headline `value` is trajectory-steps per second (K * T *
iterations per solve) with the inputs resident in device memory; `e2e` is the
same metric through the synchronous C call with host x0 in and host u0 out.
The line also carries, each with its own rooflines and oracle baseline, the
quadrotor (K = 4096, T = 100, 10 iterations) and cart-pole (K = 1000,
T = 50) workloads; the batched form (256 uneven instances in one persistent
launch, against one instance per launch); and the served form (a Poisson
request stream over 64 sessions: solves/s and p50/p99 latency over 60 s, a
sweep of arrival rates to saturation, and the plain one-request-per-launch
path on the same mix).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large_quadrotor|quadrotor_k4096|cartpole_k1000|quadrotor_alg1]
                  [--no-cpu] [--no-extras] [--served-seconds S]

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the only other place this script runs it).
Under torchrun each rank solves its own independent problem (rank-specific
Philox key): weak scaling, no collective in the data path; the timed region
is bracketed by barriers and the maximum over ranks is reported.
"""

from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1807_06108_gb300 import dist as D  # noqa: E402
from paper_1807_06108_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "large_quadrotor": W.large_quadrotor,
    "quadrotor_k4096": W.quadrotor_k4096,
    "cartpole_k1000": W.cartpole_k1000,
    "quadrotor_alg1": W.quadrotor_alg1,
}
# workloads reported beside the headline one, (steps, CPU-baseline seconds)
SUB_WORKLOADS = {"quadrotor_k4096": (200, 5.0), "cartpole_k1000": (400, 3.0)}
METRIC = "trajectory-steps/s (MPC solves of MPPI on jump diffusions)"

# Source-level lane operations per trajectory step (each 32-bit integer or
# float32 add / mul / fma / xor / compare / select counts 1, a 32x32->64
# multiply 2; logf 8, rsqrtf 4, the octant sin/cos of 2 pi u 24; the hardware
# __sincosf 3 and __fdividef 2), counted from the kernel source: SEQ = cost +
# plant + Euler step of the sequential rollout kernel, NOISE = Philox,
# Box-Muller, perturbation and jump count of the sampling kernel.  The fused
# tile does both in one kernel.
SEQ_OPS_PER_STEP = {"cartpole": 64.0, "quadrotor": 154.0}
NOISE_OPS_PER_STEP = {"cartpole": 80.0, "quadrotor": 230.0}
L2_BYTES = 129 * 1024 * 1024

VARIANT_NAMES = {1: "fused", 2: "split", 3: "staged", 4: "staged_block_records"}
ROLLOUT_KERNELS = {1: "rollout_kernel", 2: "rollout_split_kernel", 3: "rollout_staged_kernel",
                   4: "rollout_staged_kernel"}

# DRAM traffic per launch from ncu captures, with the hash of the kernel
# sources they were taken on; a figure is reported only while the sources
# are unchanged.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
KERNEL_SOURCES = ("paper_1807_06108_gb300/csrc/kernels.cuh", "paper_1807_06108_gb300/csrc/device.cuh")


def kernel_source_hash():
    h = hashlib.sha1()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(workload, kernel):
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_sources_sha") != kernel_source_hash():
        return None
    e = t.get("entries", {}).get(f"{workload}/{kernel}")
    return None if e is None else int(e["dram_read_bytes"] + e["dram_write_bytes"])


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------
# Clocks during the timed regions
# --------------------------------------------------------------------------

REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, maximum SM clock,
    power, clock-event reasons) of the GPU that torch calls `device`."""

    def __init__(self, device):
        import torch
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.nv = nv
        self.h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(device)
        ok = False
        uuid = str(getattr(props, "uuid", "") or "")
        if uuid:
            key = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
            ok = nv.nvmlDeviceGetHandleByUUID(key.encode(), ctypes.byref(self.h)) == 0
        if not ok and hasattr(props, "pci_bus_id"):
            bus = "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
            ok = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h)) == 0
        if not ok:
            raise OSError("no NVML handle for the CUDA device")
        self.reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM
        self.max_mhz = float(mx.value)

    def sample(self):
        clk, pw, rs = ctypes.c_uint(0), ctypes.c_uint(0), ctypes.c_ulonglong(0)
        self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk))
        self.nv.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(pw))
        self.reasons_fn(self.h, ctypes.byref(rs))
        return float(clk.value), self.max_mhz, pw.value / 1000.0, int(rs.value)


class ClockSampler:
    """SM clock, power and clock-event reasons sampled every 5 ms while the
    timed regions run: read-only NVML queries, or (where NVML cannot be
    loaded) an nvidia-smi process that writes its samples to a file."""

    def __init__(self, device, period_s=0.005):
        self.device = device
        self.period = period_s
        self.samples = []  # (sm_mhz, max_mhz, watts, reason bits)
        self.active = False
        self._stop = threading.Event()
        self._t = None
        self._proc = None
        self._file = None
        self.how = "nvml"

    def _loop(self, nv):
        while not self._stop.is_set():
            if self.active:
                try:
                    self.samples.append(nv.sample())
                except OSError:
                    pass
            time.sleep(self.period)

    def start(self):
        try:
            nv = _Nvml(self.device)
            self._t = threading.Thread(target=self._loop, args=(nv,), daemon=True)
            self._t.start()
        except (OSError, AttributeError):
            self.how = "nvidia-smi"
            fd, self._file = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            try:
                self._proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.device}",
                     "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                     "--format=csv,noheader,nounits", "-lms", "100", "-f", self._file],
                    stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            except OSError:
                self._proc = None
        return self

    def region(self, on):
        """Marks the start (on) or end of a timed region."""
        self.active = bool(on)

    def stop(self):
        self._stop.set()
        if self._t is not None:
            self._t.join(timeout=5)
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self._proc.kill()
            try:
                with open(self._file) as f:
                    for line in f:
                        v = [x.strip() for x in line.split(",")]
                        try:
                            self.samples.append((float(v[0]), float(v[1]), float(v[2]), int(v[3], 16)))
                        except (ValueError, IndexError):
                            pass
                os.unlink(self._file)
            except OSError:
                pass

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "how": self.how}
        sm = [s[0] for s in self.samples]
        bits = 0
        for s in self.samples:
            bits |= s[3]
        reasons = sorted(name for b, name in REASON_BITS.items() if bits & b)
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "power_w_max": max(s[2] for s in self.samples), "reasons": reasons,
                "samples": len(self.samples), "how": self.how}


# --------------------------------------------------------------------------
# Multi-process plumbing
# --------------------------------------------------------------------------

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


# --------------------------------------------------------------------------
# The oracle on the host cores
# --------------------------------------------------------------------------

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
        "config": _config(prob, v / (K * T * iters)) | {"sample_rollouts": Ks},
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


def _config(prob, solves_per_s):
    return {"workload": prob["name"], "K": prob["K"], "T": prob["T"], "iters": prob["iters"],
            "dt": prob["dt"], "noise": prob["noise_dtype"], "jump_rate": prob["nu"],
            "mark_law": prob["mark_law"], "solves_per_s": solves_per_s}


# --------------------------------------------------------------------------
# One single-problem workload
# --------------------------------------------------------------------------

def _update_kernel_name(prob, tile):
    """The library runs the whole update in one block (update_small_kernel)
    when the perturbations of an iteration fit in 256 KB, Kpad <= 8192 and
    T*m <= 2048 (not with the block-record tile); update_kernel otherwise."""
    m = 1 if prob["system"] == "cartpole" else 4
    kpad = (prob["K"] + 31) // 32 * 32
    sb = 2 if prob["noise_dtype"] == "bf16" else 4
    small = (tile[0] != 4 and kpad <= 8192 and prob["T"] * m <= 2048
             and prob["T"] * kpad * m * sb <= 256 * 1024)
    return "update_small_kernel" if small else "update_kernel"


def _launches_per_iteration(prob, tile, n_sms):
    """Kernels of one iteration: the fused tile's rollout and update; else the
    noise pass, the rollout and the update, plus the marks pass for sparse
    state-jump records (rollout blocks of 128 beyond the SM count)."""
    if tile[0] == 1:
        return 2
    sparse = (prob["jump_channel"] == "state" and prob["nu"] > 0
              and (prob["K"] + 127) // 128 > n_sms)
    return 4 if sparse else 3


def measure_workload(prob, args, steps, warmup, clk, dist, ws, local):
    """Times `steps` MPC solves of `prob` (after `warmup`), returns the
    record: value, ms_per_step, e2e, rooflines and launches."""
    import torch
    from paper_1807_06108_gb300 import mppi

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
          for _ in range(steps)]

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
    for _ in range(warmup):  # warm-up (captures the graph)
        one_step()
    stream.synchronize()

    # ---- timed region A: device-resident inputs, L2 flushed between steps
    _barrier(dist)
    torch.cuda.synchronize()
    clk.region(True)
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk.region(False)
    _barrier(dist)
    total_ms = D.max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in ev), "cuda")
    ms_per_step = total_ms / steps
    value = ws * steps_per_solve * steps / (total_ms / 1e3)

    # ---- timed region B: the same steps with phase events inside the graph
    mppi.mppi_jump_enable_timing(ctx, True)
    for _ in range(max(1, warmup)):
        one_step()
    stream.synchronize()
    roll_ms, upd_ms, n_it = 0.0, 0.0, 0
    clk.region(True)
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        one_step()
        r, u, n = mppi.mppi_jump_phase_times(ctx)
        roll_ms += r
        upd_ms += u
        n_it += n
    clk.region(False)
    mppi.mppi_jump_enable_timing(ctx, False)
    roll_avg = roll_ms / n_it
    upd_avg = upd_ms / n_it

    # ---- timed region C: end to end through the synchronous C call
    x_host = np.ascontiguousarray(x0, dtype=np.float32)
    u_host = np.zeros(solver.m, dtype=np.float32)
    for _ in range(2):
        mppi.mppi_jump_step(ctx, x_host, iters, u_host)
    _barrier(dist)
    clk.region(True)
    t0 = time.perf_counter()
    for _ in range(steps):
        mppi.mppi_jump_step(ctx, x_host, iters, u_host)
    e2e_s = D.max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    clk.region(False)
    e2e = ws * steps_per_solve * steps / e2e_s

    # ---- region D: the update kernel on its own (same launch configuration):
    # inside the step it shares the GPU with the next iteration's noise pass,
    # which blurs its bandwidth figure.  Each launch follows a fresh
    # rollout_cost (which arms the running minimum) and an L2 flush: a write
    # of twice the L2 size, then a read of it, so that the flush's dirty lines
    # are written back before the timed launch rather than during it (a cold,
    # clean L2, as under ncu's cache control).
    n_iso = min(steps, 50)
    iso_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n_iso)]
    for i in range(n_iso + 3):
        solver.rollout_cost(x0, want_costs=False)
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
            flush.sum()
            if i >= 3:
                iso_ev[i - 3][0].record(stream)
            mppi.mppi_jump_update(ctx)
            if i >= 3:
                iso_ev[i - 3][1].record(stream)
    stream.synchronize()
    upd_iso_ms = sum(a.elapsed_time(b) for a, b in iso_ev) / n_iso
    solver.close()
    del flush

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
    if tile[0] == 4:
        # the update combines the rollout blocks' records (their perturbation
        # pass runs inside the rollout kernel)
        n_rec = (K + 31) // 32 * 32 // tile[1]
        upd_bytes = n_rec * (2 + T * m) * 4 + 8 * T * m
    else:
        upd_bytes = K * T * m * sb + 8 * K + 8 * T * m
    upd_gbs = upd_bytes / (upd_iso_ms / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    rk = ROLLOUT_KERNELS[tile[0]]
    uk = _update_kernel_name(prob, tile)
    return {
        "value": value, "ms_per_step": ms_per_step,
        "config": _config(prob, value / steps_per_solve) | {
            "rollout_tile": {"variant": VARIANT_NAMES[tile[0]], "block": tile[1], "chunk": tile[2]},
            "l2": "flushed between timed steps (write of 2x L2 size)"},
        "e2e": {"value": e2e, "unit": "trajectory-steps/s",
                "h2d_bytes_per_step": 4 * len(x0), "d2h_bytes_per_step": 4 * m + 4,
                "solves_per_s": e2e / steps_per_solve},
        # per iteration: noise (+ marks for state-channel jumps) + rollout +
        # update (split and staged tiles) or rollout + update (fused tile),
        # timed region A only
        "gpu_launches": _launches_per_iteration(prob, tile, n_sms) * iters * steps,
        "roofline": {"bound": "alu", "kernel": rk,
                     "achieved": achieved, "peak": alu_peak, "unit": "T lane-ops/s",
                     "frac": achieved / alu_peak,
                     "traffic": _traffic(prob["name"], rk),
                     "avg_launch_ms": roll_avg,
                     "peak_basis": f"{n_sms} SMs x 128 lanes x {sm_mhz:.0f} MHz "
                                   f"({peak_kind} max clock)",
                     "ops_per_trajectory_step": ops_step},
        "roofline_update": {"bound": "hbm", "kernel": uk, "achieved": upd_gbs,
                            "peak": hbm, "unit": "GB/s", "frac": upd_gbs / hbm,
                            "avg_launch_ms": upd_iso_ms, "algorithmic_bytes": upd_bytes,
                            "in_step_avg_launch_ms": upd_avg,
                            "traffic": _traffic(prob["name"], uk),
                            "note": f"{peak_kind} copy bandwidth; timed alone after an L2 flush and clean "
                                    "(in the step it overlaps the next noise pass)"},
    }


# --------------------------------------------------------------------------
# Batched and served forms
# --------------------------------------------------------------------------

def bench_batched(reps=5):
    """256 uneven instances: one persistent launch per batched step, against
    the same instances solved one per launch."""
    import torch
    from paper_1807_06108_gb300 import mppi
    probs = W.batched_instances()
    b = mppi.Batch(probs)
    try:
        b.set_states([W.initial_state(p) for p in probs])
        (block, chunk), _ = b.autotune(reps=2)
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
            "speedup": plain_ms / ms, "block": block, "chunk": chunk, "work_items": info["items"],
            "grid": info["grid"]}


def _served_run(probs, rate_hz, duration_s, seed):
    """One Poisson trace through a fresh server; returns its statistics."""
    from paper_1807_06108_gb300 import mppi
    srv = mppi.Server(probs, budget_bytes=20 << 30, max_inflight=32)
    try:
        rng = np.random.default_rng(seed)
        states = [W.initial_state(p).astype(np.float32) for p in probs]
        for i in range(len(probs)):  # first request per session: graph capture
            srv.submit(i, states[i])
        srv.drain()
        srv.reset_stats()
        t_arr, sess = W.arrival_trace(rate_hz, duration_s, len(probs), seed=seed)
        t0 = time.perf_counter()
        for t, s in zip(t_arr, sess):
            while time.perf_counter() - t0 < t:
                pass
            states[s] = states[s] + W.state_drift(probs[s], rng)
            srv.submit(int(s), states[s])
        srv.drain(900)
        st = srv.stats()
    finally:
        srv.close()
    return {"offered_per_s": rate_hz, "seconds": duration_s, "requests": st["completed"],
            "solves_per_s": st["completed"] / max(st["span_s"], 1e-9),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
            "evictions": st["evictions"], "resident_gb": st["resident_bytes"] / 1e9}


def _served_plain(probs, n_requests=2000, seed=0):
    """The plain path on the same mix: one request after another, each one
    MPC step of its session's own context launched on one stream."""
    import torch
    from paper_1807_06108_gb300 import mppi
    s = torch.cuda.Stream()
    solvers = [mppi.Solver(p, stream=s) for p in probs]
    try:
        for sv, p in zip(solvers, probs):
            sv.set_x0(W.initial_state(p))
            mppi.mppi_jump_step_async(sv.ctx, sv.x0.data_ptr(), p["iters"], sv.u0.data_ptr())
        s.synchronize()
        _, sess = W.arrival_trace(2000.0, n_requests / 2000.0 * 1.5, len(probs), seed=seed)
        sess = sess[:n_requests]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for i in sess:
            sv = solvers[int(i)]
            mppi.mppi_jump_step_async(sv.ctx, sv.x0.data_ptr(), probs[int(i)]["iters"], sv.u0.data_ptr())
        e1.record(s)
        s.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        for sv in solvers:
            sv.close()
    return {"requests": len(sess), "solves_per_s": len(sess) / ms * 1e3,
            "ms_per_request": ms / len(sess)}


def bench_served(duration_s=60.0, rate_hz=2000.0, sweep=(5000.0, 10000.0, 20000.0),
                 sweep_seconds=5.0):
    """Poisson requests over 64 sessions (one MPC step each, warm-started from
    the session's device state), admitted under a 20 GB budget: the
    workload's trace at `rate_hz`, a sweep of higher rates, and the plain
    one-request-per-launch path on the same mix."""
    probs = W.served_sessions()
    main = _served_run(probs, rate_hz, duration_s, seed=0)
    pts = [_served_run(probs, r, sweep_seconds, seed=1 + i) for i, r in enumerate(sweep)]
    plain = _served_plain(probs)
    best = max([main] + pts, key=lambda r: r["solves_per_s"])
    return {"workload": f"64 sessions (cart-pole 1 / quadrotor 10 iterations, K in {{1024..16384}}, "
                        f"T in {{50..200}}), Poisson arrivals {rate_hz:.0f}/s for {duration_s:.0f} s, "
                        "20 GB budget",
            **{k: main[k] for k in ("requests", "solves_per_s", "p50_ms", "p99_ms", "max_ms",
                                    "evictions", "resident_gb")},
            "sweep": pts, "plain": plain,
            "saturation_solves_per_s": best["solves_per_s"],
            "vs_plain": best["solves_per_s"] / plain["solves_per_s"]}


# --------------------------------------------------------------------------
# Our arm
# --------------------------------------------------------------------------

def run_ours(args):
    import torch

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    clk = ClockSampler(local).start()
    try:
        base = WORKLOADS[args.workload]()
        prob = WORKLOADS[args.workload](seed=D.rank_seed(base["seed"], rank), name=base["name"])
        head = measure_workload(prob, args, args.steps, args.warmup, clk, dist, ws, local)
        subs = {}
        if not args.no_extras:
            for name, (steps, budget) in SUB_WORKLOADS.items():
                if name == args.workload:
                    continue
                sb = WORKLOADS[name]()
                sp = WORKLOADS[name](seed=D.rank_seed(sb["seed"], rank), name=sb["name"])
                subs[name] = (sp, budget, measure_workload(sp, args, steps, max(3, args.warmup),
                                                           clk, dist, ws, local))
    finally:
        clk.stop()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        cpu, first = cpu_baseline(prob, budget_s=args.cpu_budget)
        cpu["update_rel_err_vs_oracle"] = _update_error(prob, first)
    configs = {}
    for name, (sp, budget, rec) in subs.items():
        if not args.no_cpu:
            c, f = cpu_baseline(sp, budget_s=budget)
            c["update_rel_err_vs_oracle"] = _update_error(sp, f)
            rec["cpu_baseline"] = c
            rec["update_rel_err_vs_oracle"] = c["update_rel_err_vs_oracle"]
        configs[sp["name"]] = rec
    extras = {}
    if not args.no_extras:
        extras["configs"] = configs
        extras["batched"] = bench_batched()
        extras["served"] = bench_served(duration_s=args.served_seconds)
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "trajectory-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": head["config"],
        "e2e": head["e2e"],
        "gpu_launches": head["gpu_launches"],
        "roofline": head["roofline"],
        "roofline_update": head["roofline_update"],
        "update_rel_err_vs_oracle": cpu["update_rel_err_vs_oracle"] if cpu else None,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        **extras,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large_quadrotor")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="time the rollout tile the library's autotuner picks")
    ap.add_argument("--tile", default="",
                    help="rollout tile 'variant,block,chunk' (1 fused, 2 split, 3 staged, "
                         "4 staged with block records)")
    ap.add_argument("--served-seconds", type=float, default=60.0,
                    help="length of the served leg's Poisson arrival trace at 2000 requests/s")
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
