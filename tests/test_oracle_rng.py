"""Pins for the oracle's random stream: Philox4x32-10 mixing, uniforms,
Box-Muller normals, jump counts (Poisson, Eq. 2; Bernoulli zero-one law,
Algorithm 1) and marks (Normal, Eq. 2; Laplace).  Each test compares the
oracle with a distribution the paper fixes, checked by scipy, or with an
exact property, so that a dropped term, a wrong constant or a swapped word
fails one of them."""

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1807_06108_gb300 import workloads as W


def _philox_py(ctr, key):
    """Philox4x32-10 restated in Python integers (a second, independent
    transcription of the SC'11 round function; a cross-check of the C code's
    integer handling, not a pin of the algorithm itself)."""
    c = [int(v) & 0xFFFFFFFF for v in ctr]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & 0xFFFFFFFF, p1 & 0xFFFFFFFF,
             ((p0 >> 32) ^ c[3] ^ k1) & 0xFFFFFFFF, p0 & 0xFFFFFFFF]
        k0 = (k0 + 0x9E3779B9) & 0xFFFFFFFF
        k1 = (k1 + 0xBB67AE85) & 0xFFFFFFFF
    return c


def test_philox_matches_python_transcription():
    rng = np.random.default_rng(1)
    for _ in range(200):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64)
        assert list(oracle.philox(ctr, key)) == _philox_py(ctr, key)


def test_philox_avalanche():
    """Flipping one input bit flips about half of the 128 output bits (a
    property of the ten-round mixing; a dropped round or multiply breaks it)."""
    rng = np.random.default_rng(2)
    flips = []
    for _ in range(300):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64)
        base = oracle.philox(ctr, key)
        word, bit = rng.integers(0, 6), rng.integers(0, 32)
        c2, k2 = ctr.copy(), key.copy()
        if word < 4:
            c2[word] ^= np.uint64(1 << int(bit))
        else:
            k2[word - 4] ^= np.uint64(1 << int(bit))
        other = oracle.philox(c2, k2)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, other)))
    flips = np.array(flips)
    assert abs(flips.mean() - 64.0) < 1.5
    assert flips.min() > 30


def _uniform_words(n, seed=0):
    out = np.empty((n, 4), dtype=np.uint64)
    for i in range(n):
        out[i] = oracle.philox([i, 7, 3, 1], [seed, 12345])
    return out


def test_philox_words_uniform_bytes_and_uncorrelated():
    w = _uniform_words(20000)
    for col in range(4):
        bytes_ = np.concatenate([(w[:, col] >> s) & 0xFF for s in (0, 8, 16, 24)])
        counts = np.bincount(bytes_.astype(np.int64), minlength=256)
        chi2, p = stats.chisquare(counts)
        assert p > 1e-4, (col, p)
    u = (w.astype(np.float64) + 0.5) / 2**32
    cc = np.corrcoef(u.T)
    assert np.max(np.abs(cc - np.eye(4))) < 0.03
    lag = np.corrcoef(u[:-1, 0], u[1:, 0])[0, 1]
    assert abs(lag) < 0.03


def test_uniform_exact_and_open_interval():
    assert oracle.uniform(0) == 2.0**-24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0**-24
    rng = np.random.default_rng(3)
    for w in rng.integers(0, 2**32, size=1000):
        u = oracle.uniform(int(w))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # exactly representable in float32


def test_box_muller_normals_ks_and_moments():
    rng = np.random.default_rng(4)
    words = rng.integers(0, 2**32, size=(50000, 4), dtype=np.uint64)
    z = np.concatenate([oracle.normals4(w) for w in words])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    n = z.size
    assert abs(z.mean()) < 4 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / n)
    assert abs(stats.skew(z)) < 4 * np.sqrt(6.0 / n)
    # the two normals of one pair are independent
    zz = z.reshape(-1, 4)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 4 / np.sqrt(zz.shape[0])


@pytest.mark.parametrize("nu,dt", [(1.0, 0.02), (2.0, 0.01), (5.0, 0.005), (3.0, 0.02),
                                    (0.5, 0.01), (40.0, 0.02), (0.0, 0.01)])
def test_poisson_threshold_table_matches_scipy_cdf(nu, dt):
    nu32, dt32 = np.float32(nu), np.float32(dt)
    mu = float(nu32) * float(dt32)
    thr, nmax = oracle.count_table(float(nu32), float(dt32), "poisson")
    for n in range(1, nmax + 1):
        ref = 2.0**32 * stats.poisson.cdf(n - 1, mu)
        assert abs(float(thr[n - 1]) - np.ceil(ref)) <= 1.0, (n, thr[n - 1], ref)
    assert np.all(np.diff(thr[:nmax].astype(np.int64)) >= 0)
    # the table ends where the Poisson tail P(N > nmax) drops below 2^-32,
    # and its last entry is still reachable
    assert stats.poisson.sf(nmax, mu) * 2.0**32 < 1.0 + 1e-6
    if nmax > 0:
        assert stats.poisson.sf(nmax - 1, mu) * 2.0**32 > 1.0 - 1e-6
    else:
        assert mu == 0.0


def test_poisson_table_rejects_heavy_tail_and_bad_rates():
    with pytest.raises(oracle.OracleError):
        oracle.count_table(500.0, 0.02, "poisson")  # mu = 10: tail beyond 16 jumps
    with pytest.raises(oracle.OracleError):
        oracle.count_table(-1.0, 0.02, "poisson")
    with pytest.raises(oracle.OracleError):
        oracle.count_table(60.0, 0.02, "bernoulli")  # mu >= 1


def _draws(prob, K=20000, it=0):
    x0 = W.initial_state(prob)
    U = W.initial_controls(prob)
    return oracle.rollouts(prob, x0, U, it, 0, K, counts=True, delta=True, jumps=True)


def test_poisson_counts_match_pmf():
    prob = W.cartpole_k1000(T=50, nu=10.0)  # mu = 0.2 per step
    r = _draws(prob, K=20000)
    mu = prob["nu"] * prob["dt"]
    c = r["counts"].ravel().astype(np.int64)
    n = c.size
    assert abs(c.mean() - mu) < 4 * np.sqrt(mu / n)
    assert abs(c.var() - mu) < 4 * np.sqrt((mu + 2 * mu**2) / n)
    obs = np.bincount(c, minlength=5)[:4]
    exp = n * stats.poisson.pmf(np.arange(4), mu)
    assert np.all(np.abs(obs - exp) < 5 * np.sqrt(exp) + 1)


def test_bernoulli_zero_one_law_rate():
    prob = W.cartpole_k1000(T=50, nu=10.0, count_law="bernoulli")
    r = _draws(prob, K=20000)
    mu = prob["nu"] * prob["dt"]
    c = r["counts"].ravel()
    assert c.max() == 1
    n = c.size
    assert abs(c.mean() - mu) < 4 * np.sqrt(mu * (1 - mu) / n)


def test_zero_rate_draws_no_jumps():
    prob = W.cartpole_k1000(T=30, nu=0.0)
    r = _draws(prob, K=2000)
    assert r["counts"].max() == 0
    assert np.all(r["J"] == 0.0)


@pytest.mark.parametrize("law", ["normal", "laplace"])
def test_compound_poisson_moments(law):
    """Per-step jump J = sum of N marks: E[J] = 0, Var[J] = mu * E[xi^2] with
    E[xi^2] = s^2 (Normal) or 2 b^2 (Laplace)."""
    prob = W.quadrotor_k4096(T=100, nu=20.0, mark_law=law, mark_scale=[0.5, 1.0, 2.0])
    r = _draws(prob, K=4000)
    mu = prob["nu"] * prob["dt"]
    J = r["J"].reshape(-1, 3)
    n = J.shape[0]
    for c, s in enumerate([0.5, 1.0, 2.0]):
        m2 = s**2 if law == "normal" else 2 * s**2
        m4 = 3 * s**4 if law == "normal" else 24 * s**4
        var_th = mu * m2
        # Var of J^2 for a compound Poisson: mu*m4 + 3 (mu*m2)^2 - (mu*m2)^2
        se = np.sqrt((mu * m4 + 2 * (mu * m2) ** 2) / n)
        assert abs(J[:, c].mean()) < 5 * np.sqrt(var_th / n)
        assert abs((J[:, c] ** 2).mean() - var_th) < 5 * se


@pytest.mark.parametrize("law", ["normal", "laplace"])
def test_single_jump_marks_follow_law(law):
    prob = W.quadrotor_k4096(T=100, nu=20.0, mark_law=law, mark_scale=[1.5, 1.5, 1.5])
    r = _draws(prob, K=3000)
    one = r["counts"] == 1
    xi = r["J"][one][:, 0]
    assert xi.size > 5000
    dist = stats.norm(scale=1.5) if law == "normal" else stats.laplace(scale=1.5)
    assert stats.kstest(xi, dist.cdf).pvalue > 1e-3


def test_perturbation_variance_is_c_sigma2():
    prob = W.quadrotor_k4096(T=50, nu=0.0, sigma=[0.2, 0.3, 0.4, 0.5], c=2.0)
    r = _draws(prob, K=4000)
    d = r["delta"].reshape(-1, 4)
    n = d.shape[0]
    for i, s in enumerate([0.2, 0.3, 0.4, 0.5]):
        v = 2.0 * s * s
        assert abs(d[:, i].var() - v) < 5 * v * np.sqrt(2.0 / n)
    cc = np.corrcoef(d.T)
    assert np.max(np.abs(cc - np.eye(4))) < 5 / np.sqrt(n)


def test_counts_independent_of_perturbations():
    prob = W.cartpole_k1000(T=50, nu=10.0)
    r = _draws(prob, K=10000)
    c = r["counts"].ravel().astype(np.float64)
    d = r["delta"].ravel()
    # in state mode delta_eff carries no jump: correlation is zero
    assert abs(np.corrcoef(c, d)[0, 1]) < 5 / np.sqrt(c.size)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32),
                        # exact ties between two bfloat16 neighbours
                        (np.arange(1, 200, dtype=np.float32) * 2.0**-7 + 2.0**-15).astype(np.float32),
                        np.array([1.0 + 2.0**-8, 1.0 + 3 * 2.0**-8, -1.0 - 2.0**-8], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16_round(float(v)) for v in x], dtype=np.float32)
    assert np.array_equal(ref, got)
