"""The allocation-free update entry point, for callers that cannot allocate
device memory while they run (a fixed-rate control loop, where a cudaMalloc
may synchronise the device and stall the loop, or a program whose device
memory belongs to another allocator).  It must give what the context's own
update gives from the same costs, perturbations and controls, on two calls
in a row (the second call reuses the shared scratch the first one left
behind).  This file is collected last on purpose."""

import numpy as np
import pytest

import oracle
from paper_1807_06108_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prob", [W.cartpole_k1000(), W.quadrotor_k4096(K=777, T=33, lam=20.0)],
                         ids=["cartpole_K1000_T50", "quadrotor_K777_T33"])
def test_noalloc_update_matches_context_update(cuda, prob):
    torch = cuda
    from paper_1807_06108_gb300 import mppi
    s = mppi.Solver(prob)
    try:
        rng = np.random.default_rng(3)
        x0 = W.random_state(prob, rng, 0.1)
        m, K, T = s.m, prob["K"], prob["T"]
        for call in range(2):
            U_before = s.controls()
            costs = s.rollout_cost(x0)
            noise = s.noise()  # synchronises the solver stream
            S = costs.cpu().numpy()
            s.update()
            s.sync()
            U_after = s.controls()
            with torch.cuda.stream(s.stream):
                c = torch.from_numpy(S).to("cuda")
                d = torch.from_numpy(np.ascontiguousarray(noise, dtype=np.float32)).to("cuda")
                U = torch.from_numpy(np.ascontiguousarray(U_before)).to("cuda")
            s.stream.synchronize()
            mppi.mppi_jump_update_noalloc(c.data_ptr(), d.data_ptr(), K, T, m, prob["lam"],
                                          prob["alpha"], U.data_ptr(), s.stream.cuda_stream)
            s.stream.synchronize()
            got = U.cpu().numpy().astype(np.float64)
            dU_ref = U_after.astype(np.float64) - U_before
            dU = got - U_before
            err = np.max(np.abs(dU - dU_ref)) / max(np.max(np.abs(dU_ref)), 1e-30)
            assert err <= 1e-4, (call, err)
            # and the FP64 oracle's weights and update from the same arrays
            w, _ = oracle.softmin(S.astype(np.float64), prob["lam"])
            U_or = oracle.update(w, noise.astype(np.float64), U_before, prob["alpha"])
            dU_or = U_or - U_before
            err_or = np.max(np.abs(dU - dU_or)) / max(np.max(np.abs(dU_or)), 1e-30)
            assert err_or <= 1e-4, (call, err_or)
    finally:
        s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(cuda):
    from paper_1807_06108_gb300 import mppi
    torch = cuda
    t = torch.zeros(8, device="cuda")
    p = t.data_ptr()
    # ceil(K/1024) * (T*m + 1) + 64 floats must fit in 2^20
    with pytest.raises(mppi.MppiError) as e:
        mppi.mppi_jump_update_noalloc(p, p, 1 << 20, 300, 4, 1.0, 1.0, p)
    assert e.value.code == mppi.ENOMEM
    with pytest.raises(mppi.MppiError) as e:
        mppi.mppi_jump_update_noalloc(p, p, 100, 10, 3, 1.0, 1.0, p)
    assert e.value.code == mppi.EINVAL
    # a horizon beyond 8 * 65535 steps is refused before anything is enqueued,
    # even where its scratch would fit (one chunk of 1024 rollouts, m = 1)
    with pytest.raises(mppi.MppiError) as e:
        mppi.mppi_jump_update_noalloc(p, p, 1000, 8 * 65535 + 1, 1, 1.0, 1.0, p)
    assert e.value.code == mppi.EINVAL
