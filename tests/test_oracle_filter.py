"""Pins for the oracle's filter: weights, resampling, the ensemble and its rates.

* normalise: scipy's logsumexp; ESS closed forms (uniform -> N, spike -> 1).
* systematic resampling (Alg. 1 step 2b, systematic form): hand-worked
  examples in tests/golden/systematic_worked.txt; offspring counts lie in
  {floor(N w), ceil(N w)}; averaged over a grid of u they equal N w exactly
  up to the grid spacing; ancestors are sorted and never pick a zero weight.
* multinomial resampling (Alg. 1 step 2b as printed): offspring counts are
  Binomial(N, w) in mean and variance.
* kalman: equals conditioning the joint Gaussian of the whole record
  (a different computation of the same posterior and evidence).
* bf_run on the linear-Gaussian model (the case where Sec. 2.2's recursion
  is exact in closed form):
    - the ensemble average converges to the Kalman mean;
    - Lemma 2: E[G_t^N] equals the Kalman evidence p(y_{1:t});
    - Theorem 1: the bias of (f, pi_t^N) decays as 1/N (log-log slope -1);
    - Corollary 1/2: the variance decays as 1/N per filter and as 1/(MN)
      for the average of M independent filters.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_1407_8071_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        yield [f.split() for f in line.split("|")]


# ---------------------------------------------------------------- normalise
def test_normalise_matches_logsumexp():
    rng = np.random.default_rng(0)
    for scale in (0.1, 10.0, 1000.0):
        l = rng.normal(-50.0, scale, size=1000)
        out = oracle.normalise(l)
        assert out["logZ"] == pytest.approx(special.logsumexp(l), rel=1e-14, abs=1e-12)
        w = np.exp(l - l.max())
        assert out["ess"] == pytest.approx(w.sum() ** 2 / (w ** 2).sum(), rel=1e-12)


def test_ess_closed_forms():
    assert oracle.normalise(np.zeros(64))["ess"] == pytest.approx(64.0, rel=1e-15)
    l = np.full(64, -1e4)
    l[5] = 0.0
    assert oracle.normalise(l)["ess"] == 1.0
    assert oracle.normalise(np.array([3.0]))["ess"] == 1.0


# --------------------------------------------------------------- systematic
def test_systematic_golden_worked_examples():
    rows = list(_golden_rows("systematic_worked.txt"))
    assert len(rows) >= 6
    for (n,), w, (u,), a in rows:
        got = oracle.systematic(np.array(w, dtype=float), float(u))
        assert len(got) == int(n)
        assert got.tolist() == [int(v) for v in a], (w, u)


def _offspring(anc, N):
    return np.bincount(anc, minlength=N)


@pytest.mark.parametrize("kind", ["lognormal", "spike", "ties", "sparse", "uniform"])
@pytest.mark.parametrize("N", [1, 7, 64, 1000])
def test_systematic_offspring_floor_ceil(kind, N):
    w = W.random_weights(N, seed=N + len(kind), kind=kind)
    q = oracle.quantise(w)
    what = q / q.sum()
    for u in W.random_uniforms(8, seed=N):
        anc = oracle.systematic(w, float(u))
        assert np.all(np.diff(anc) >= 0)
        assert np.all(q[anc] > 0)
        o = _offspring(anc, N)
        assert o.sum() == N
        lo, hi = np.floor(N * what - 1e-9), np.ceil(N * what + 1e-9)
        assert np.all((o >= lo) & (o <= hi))


@pytest.mark.parametrize("kind", ["lognormal", "ties", "sparse"])
def test_systematic_expected_offspring_over_u_grid(kind):
    N, G = 50, 4000
    w = W.random_weights(N, seed=3, kind=kind)
    q = oracle.quantise(w)
    what = q / q.sum()
    acc = np.zeros(N)
    for g in range(G):
        acc += _offspring(oracle.systematic(w, (g + 0.5) / G), N)
    # each offspring count changes at most twice as u sweeps [0, 1)
    assert np.max(np.abs(acc / G - N * what)) <= 2.0 / G + 1e-12


def test_quantisation_is_exact_integer_form():
    for N in (1, 2, 3, 1000, 1 << 20):
        w = np.array([1.0, 0.5, 1e-3, 0.0][: min(N, 4)])
        q = oracle.quantise(np.resize(w, N))
        L = math.ceil(math.log2(N)) if N > 1 else 0
        assert q[0] == 2.0 ** (52 - L)
        assert np.all(q == np.floor(q)) and q.sum() <= 2.0 ** 52


# -------------------------------------------------------------- multinomial
def test_multinomial_offspring_moments():
    N, R = 20, 4000
    w = W.random_weights(N, seed=9, kind="lognormal")
    q = oracle.quantise(w)
    what = q / q.sum()
    counts = np.empty((R, N))
    for r in range(R):
        U = W.random_uniforms(N, seed=1000 + r)
        counts[r] = _offspring(oracle.multinomial(w, U), N)
    mean, var = counts.mean(0), counts.var(0)
    exp_var = N * what * (1 - what)
    assert np.all(np.abs(mean - N * what) < 4.5 * np.sqrt(exp_var / R) + 1e-12)
    big = exp_var > 0.05
    assert np.all(np.abs(var[big] / exp_var[big] - 1.0) < 0.15)


# ------------------------------------------------------------------- Kalman
def _joint_gaussian_posterior(spec, y):
    """Posterior of x_T and log p(y_{1:T}) by conditioning the joint Gaussian of the record."""
    FK, QK = oracle.lg_transition(spec)
    d, T = spec.dx, len(y)
    H = np.zeros((spec.dy, d))
    H[np.arange(spec.dy), spec.obs_idx] = 1.0
    mus = [np.asarray(spec.x0_mean, float)]
    covs = [spec.sigma0 ** 2 * np.eye(d)]
    for _ in range(T):
        mus.append(FK @ mus[-1])
        covs.append(FK @ covs[-1] @ FK.T + QK)
    # Cov(x_s, x_t) = F^(s-t) Cov(x_t) for s >= t
    def cxx(s, t):
        if s >= t:
            return np.linalg.matrix_power(FK, s - t) @ covs[t]
        return cxx(t, s).T
    R = spec.sigma_obs ** 2 * np.eye(spec.dy)
    Syy = np.block([[H @ cxx(s, t) @ H.T + (R if s == t else 0.0) for t in range(1, T + 1)] for s in range(1, T + 1)])
    Sxy = np.hstack([cxx(T, t) @ H.T for t in range(1, T + 1)])
    muy = np.concatenate([H @ mus[t] for t in range(1, T + 1)])
    yv = np.asarray(y).ravel()
    mean = mus[T] + Sxy @ np.linalg.solve(Syy, yv - muy)
    cov = covs[T] - Sxy @ np.linalg.solve(Syy, Sxy.T)
    ll = stats.multivariate_normal(muy, Syy).logpdf(yv)
    return mean, cov, ll


def test_kalman_equals_joint_gaussian_conditioning():
    spec = W.linear_gaussian(K=10, dt=0.02, sigma=0.8)
    _, y = oracle.simulate(spec, 6, seed=42)
    m, P, ll = oracle.kalman(spec, y)
    for T in (1, 3, 6):
        mean, cov, lj = _joint_gaussian_posterior(spec, y[:T])
        assert np.allclose(m[T - 1], mean, rtol=1e-9, atol=1e-10)
        assert np.allclose(P[T - 1], cov, rtol=1e-8, atol=1e-11)
        assert ll[T - 1] == pytest.approx(lj, rel=1e-10)


# ------------------------------------------------------------ the ensemble
def test_ensemble_converges_to_kalman_mean():
    spec = W.linear_gaussian()
    T = 10
    _, y = oracle.simulate(spec, T, seed=W.SEED_LORENZ_OBS)
    m, _, _ = oracle.kalman(spec, y)
    M, N = 64, 1024
    r = oracle.bf_run(spec, M, N, T, y, seed=5)
    est = r["est"]  # T x M x 3
    se = est.std(axis=1, ddof=1) / math.sqrt(M)
    assert np.all(np.abs(r["ens"] - m) < 4.5 * se + 2e-3)
    # Definition 1: the ensemble value is the plain average of the M estimates
    assert np.allclose(r["ens"], est.mean(axis=1), rtol=0, atol=1e-13)


SCALAR = dict(K=1, dt=0.5, sigma=1.0, sigma_obs=1.0, A=[[0.5]], obs_idx=[0])
Y_SCALAR = np.array([[1.5], [1.8]])


def test_lemma2_unbiased_evidence():
    spec = W.linear_gaussian(**SCALAR)
    _, _, ll = oracle.kalman(spec, Y_SCALAR)
    M = 1 << 16
    for N in (4, 32):
        r = oracle.bf_run(spec, M, N, 2, Y_SCALAR, seed=100 + N)
        for t in range(2):
            ratio = np.exp(r["log_G"][t] - ll[t])
            assert abs(ratio.mean() - 1.0) < 4.5 * ratio.std() / math.sqrt(M), (N, t)


def test_theorem1_bias_rate_and_corollary_variance_rates():
    spec = W.linear_gaussian(**SCALAR)
    m, _, _ = oracle.kalman(spec, Y_SCALAR)
    target = m[-1, 0]
    Ns = np.array([16, 32, 64, 128, 256])
    M = 1 << 17
    bias, se, var = [], [], []
    for N in Ns:
        e = oracle.bf_run(spec, M, int(N), 2, Y_SCALAR, seed=int(N) * 17 + 1)["est"][-1, :, 0]
        bias.append(e.mean() - target)
        se.append(e.std() / math.sqrt(M))
        var.append(e.var())
        # Cor. 2 / eq. eqP1: averaging M' independent filters divides the variance by M'
        for Mg in (16, 256):
            g = e[: (M // Mg) * Mg].reshape(-1, Mg).mean(1)
            assert g.var() / (e.var() / Mg) == pytest.approx(1.0, abs=5.0 * math.sqrt(2.0 / len(g)))
    bias, se, var = map(np.asarray, (bias, se, var))
    assert np.all(np.abs(bias) > 5 * se)  # the bias is resolved at every N
    # Theorem 1: |bias| ~ c / N
    slope_b = np.polyfit(np.log(Ns), np.log(np.abs(bias)), 1, w=np.abs(bias) / se)[0]
    assert -1.2 < slope_b < -0.8, slope_b
    # Corollary 1: Var ~ c / N
    slope_v = np.polyfit(np.log(Ns), np.log(var), 1)[0]
    assert -1.1 < slope_v < -0.9, slope_v


# ------------------------------------------------------------ auxiliary particle filters
def test_apf_ensemble_converges_to_kalman_mean():
    """The ensemble of auxiliary particle filters estimates the same posterior
    (linear-Gaussian model: the Kalman filter)."""
    spec = W.linear_gaussian()
    T = 10
    _, y = oracle.simulate(spec, T, seed=W.SEED_LORENZ_OBS)
    m, _, _ = oracle.kalman(spec, y)
    M, N = 64, 1024
    r = oracle.apf_run(spec, M, N, T, y, seed=6)
    est = r["est"]
    se = est.std(axis=1, ddof=1) / math.sqrt(M)
    assert np.all(np.abs(r["ens"] - m) < 4.5 * se + 2e-3)
    assert np.allclose(r["ens"], est.mean(axis=1), rtol=0, atol=1e-13)


def test_apf_unbiased_evidence():
    """The auxiliary filter's likelihood estimate (first-stage sum times the
    mean second-stage weight) is unbiased, like the bootstrap filter's (the
    remark after Corollary 2 extends Lemma 2 to it): E exp(log G) equals the
    Kalman evidence at every t."""
    spec = W.linear_gaussian(**SCALAR)
    _, _, ll = oracle.kalman(spec, Y_SCALAR)
    M = 1 << 16
    for N in (4, 32):
        r = oracle.apf_run(spec, M, N, 2, Y_SCALAR, seed=200 + N)
        for t in range(2):
            ratio = np.exp(r["log_G"][t] - ll[t])
            assert abs(ratio.mean() - 1.0) < 4.5 * ratio.std() / math.sqrt(M), (N, t)


def test_apf_and_bootstrap_agree_on_lorenz():
    """Both filters target the same posterior: on Lorenz 63 the ensemble means
    of x2 agree within the statistical tolerance."""
    spec = W.lorenz63()
    T = 20
    _, y = oracle.simulate(spec, T, W.SEED_LORENZ_OBS)
    M, N = 64, 512
    a = oracle.apf_run(spec, M, N, T, y, seed=31, est_idx=[1])["est"][:, :, 0]
    b = oracle.bf_run(spec, M, N, T, y, seed=32, est_idx=[1])["est"][:, :, 0]
    for t in (4, 9, 19):
        se = math.sqrt(a[t].var(ddof=1) / M + b[t].var(ddof=1) / M)
        assert abs(a[t].mean() - b[t].mean()) < 4.5 * se, (t, a[t].mean(), b[t].mean(), se)


# ------------------------------------------------------------ resampling only when the ESS is low
def test_sir_always_resampling_is_the_bootstrap_run():
    """With a threshold above 1 every step resamples: the adaptive run is the
    systematic bootstrap run bit for bit (estimates, evidence, ESS)."""
    spec = W.lorenz63()
    T = 8
    _, y = oracle.simulate(spec, T, W.SEED_LORENZ_OBS)
    a = oracle.sir_run(spec, 6, 200, T, y, seed=3, ess_threshold=2.0)
    b = oracle.bf_run(spec, 6, 200, T, y, seed=3)
    assert np.array_equal(a["est"], b["est"]) and np.array_equal(a["log_G"], b["log_G"])
    assert np.array_equal(a["ess"], b["ess"]) and a["resampled"].min() == 1.0


def test_sir_adaptive_converges_to_kalman_and_is_unbiased():
    spec = W.linear_gaussian()
    T = 10
    _, y = oracle.simulate(spec, T, seed=W.SEED_LORENZ_OBS)
    m, _, _ = oracle.kalman(spec, y)
    M, N = 64, 1024
    r = oracle.sir_run(spec, M, N, T, y, seed=8, ess_threshold=0.5)
    assert 0.0 < r["resampled"].mean() < 1.0, r["resampled"].mean()  # some steps skip, some resample
    se = r["est"].std(axis=1, ddof=1) / math.sqrt(M)
    assert np.all(np.abs(r["ens"] - m) < 4.5 * se + 2e-3)
    spec = W.linear_gaussian(**SCALAR)
    _, _, ll = oracle.kalman(spec, Y_SCALAR)
    Mb = 1 << 16
    for N in (4, 32):
        rb = oracle.sir_run(spec, Mb, N, 2, Y_SCALAR, seed=400 + N, ess_threshold=0.5)
        assert 0.0 < rb["resampled"][0].mean() < 1.0
        for t in range(2):
            ratio = np.exp(rb["log_G"][t] - ll[t])
            assert abs(ratio.mean() - 1.0) < 4.5 * ratio.std() / math.sqrt(Mb), (N, t)
