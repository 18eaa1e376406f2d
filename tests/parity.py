"""Helpers shared by the GPU parity tests: run one iteration through the C ABI
and through the oracle on the same seeded inputs and compare element by
element with the tolerances below.

Tolerances (float32 device arithmetic against the float64 oracle):
  * jump counts: bit-exact (integer decisions on identical 32-bit words);
  * bfloat16 perturbations: bit-exact, except where the oracle flags the
    float64 value as lying within 2^-20 of a rounding midpoint, where either
    neighbour is accepted;
  * float32 perturbations and marks: |d| <= 2e-6 (|ref| + scale), a few ulps
    of the log / sqrt / sincos chain;
  * per-rollout cost S~: |S_gpu - S_ref| <= 1e-4 max(1, |S_ref|), skipping
    rollouts whose obstacle-indicator decision lies within 1e-3 of the
    boundary or whose bfloat16 rounding went the other way;
  * update: max |dU_gpu - dU_ref| / max |dU_ref| <= 1e-4.
"""

import numpy as np

import oracle
from paper_1807_06108_gb300 import workloads as W

S_RTOL = 1e-4
U_RTOL = 1e-4
NOISE_RTOL = 2e-6


def gpu_iteration(prob, x0, U, it, debug=True, tile=None):
    from paper_1807_06108_gb300 import mppi
    s = mppi.Solver(prob)
    try:
        if tile:
            mppi.mppi_jump_set_tuning(s.ctx, *tile)
        s.set_controls(U)
        s.set_iteration(it)
        if debug:
            s.enable_debug()
        costs = s.rollout_cost(x0)
        s.update()
        s.sync()
        out = {
            "S": costs.cpu().numpy().astype(np.float64),
            "U": s.controls().astype(np.float64),
            "w": s.weights().astype(np.float64),
            "fe": s.free_energy().astype(np.float64),
            "it": s.iteration(),
        }
        out["delta"] = s.noise().astype(np.float64)
        if prob["noise_dtype"] == "bf16":
            out["delta_bits"] = s.noise_bits()
        if debug:
            out["counts"] = s.dbg_counts.cpu().numpy()
            out["J"] = s.dbg_J.cpu().numpy().astype(np.float64)
    finally:
        s.close()
    return out


def oracle_iteration(prob, x0, U, it, k_count=None):
    """Oracle rollouts (all K, or the first k_count) plus, for all K, the
    weights and update."""
    K = prob["K"]
    kc = K if k_count is None else k_count
    r = oracle.rollouts(prob, x0, U, it, 0, kc, counts=True, delta=True, jumps=True,
                        ambig=True, margin=True)
    if kc == K:
        w, diag = oracle.softmin(r["S"], prob["lam"])
        r["w"], r["diag"] = w, diag
        r["U"] = oracle.update(w, r["delta"], U, prob["alpha"])
    return r


def bf16_bits(x):
    return (np.asarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def compare_noise(prob, g, r, kc):
    """Returns the set of rollouts whose bfloat16 rounding went the other way."""
    d_g = g["delta"][:, :kc, :]
    d_r = r["delta"]
    flipped = set()
    if prob["noise_dtype"] == "bf16":
        bits_g = g["delta_bits"][:, :kc, :]
        bits_r = bf16_bits(d_r)
        diff = bits_g != bits_r
        amb = r["ambig"]
        assert not np.any(diff & ~amb), "bfloat16 noise differs outside rounding ties"
        # where ambiguous, the GPU value must be one of the two neighbours
        if np.any(diff):
            step = np.abs(bits_g.astype(np.int32) - bits_r.astype(np.int32))
            assert np.all(step[diff] == 1)
            flipped = set(np.nonzero(diff.any(axis=(0, 2)))[0].tolist())
    else:
        scale = max(prob["sigma"]) * np.sqrt(prob["c"])
        err = np.abs(d_g - d_r)
        assert np.all(err <= NOISE_RTOL * (np.abs(d_r) + scale)), float(err.max())
    return flipped


def compare_iteration(prob, U_in, g, r, kc=None, check_update=True):
    K = prob["K"]
    kc = K if kc is None else kc
    report = {}
    # 1. jump counts: bit-exact
    np.testing.assert_array_equal(g["counts"][:, :kc], r["counts"])
    report["jumps"] = int(r["counts"].sum())
    # 2. marks
    q = prob["q"]
    if q > 0:
        jg, jr = g["J"][:, :kc, :q], r["J"][:, :, :q]
        scale = max(prob["mark_scale"]) if prob["mark_scale"] else 1.0
        assert np.all(np.abs(jg - jr) <= 1e-5 * (np.abs(jr) + scale))
    # 3. perturbations
    flipped = compare_noise(prob, g, r, kc)
    report["bf16_flips"] = len(flipped)
    # 4. costs
    Sg, Sr = g["S"][:kc], r["S"]
    rel = np.abs(Sg - Sr) / np.maximum(1.0, np.abs(Sr))
    # a rollout may legitimately differ when a float32 and a float64 state
    # fall on opposite sides of the obstacle boundary, or when its bfloat16
    # rounding went the other way; anything else is a failure
    excusable = np.zeros(kc, dtype=bool)
    if prob["system"] == "quadrotor":
        excusable |= r["margin"] < 1e-3
    for k in flipped:
        excusable[k] = True
    bad = rel > S_RTOL
    assert not np.any(bad & ~excusable), (np.nonzero(bad & ~excusable)[0][:10], rel.max())
    report["cost_flips"] = int((bad & excusable).sum())
    assert report["cost_flips"] <= max(2, kc // 200), report
    ok = ~(bad & excusable)
    report["cost_rel_err"] = float(rel[ok].max()) if ok.any() else 0.0
    report["cost_abs_err_over_lambda"] = float((np.abs(Sg - Sr)[ok] / prob["lam"]).max())
    # 5. weights, free energy, update (need all K on the oracle side)
    if check_update and kc == K:
        U0 = np.asarray(U_in, dtype=np.float64)
        dUr = r["U"] - U0
        dUg = g["U"] - U0
        den = max(np.max(np.abs(dUr)), 1e-30)
        report["update_rel_err"] = float(np.max(np.abs(dUg - dUr)) / den)
        report["weight_err"] = float(np.max(np.abs(g["w"] - r["w"])))
        report["free_energy_rel_err"] = float(abs(g["fe"][2] - r["diag"][2]) / max(1, abs(r["diag"][2])))
        assert report["update_rel_err"] <= U_RTOL, report
        assert abs(g["w"].sum() - 1.0) < 1e-5
        # weights and free energy inherit the cost error: to first order
        # |w_gpu / w_ref - 1| <= 2 max|dS| / lambda and |dF| <= 2 max|dS| / lambda
        if report["cost_flips"] == 0:
            dS = float(np.max(np.abs(Sg - Sr))) / prob["lam"]
            big = r["w"] > 1e-6
            wrel = float(np.max(np.abs(g["w"][big] / r["w"][big] - 1.0)))
            report["weight_rel_err"] = wrel
            assert wrel <= 2.0 * dS + 1e-5, (wrel, dS)
            assert abs(g["fe"][2] - r["diag"][2]) <= 2.0 * dS + 1e-5 * max(1.0, abs(r["diag"][2]))
    return report


def run_and_compare(prob, x0, U, it, kc=None, tile=None):
    g = gpu_iteration(prob, x0, U, it, tile=tile)
    r = oracle_iteration(prob, x0, U, it, kc)
    rep = compare_iteration(prob, U, g, r, kc)
    assert g["it"] == it + 1
    return rep
