"""Bootstrap filters that resample only when the ESS is low (pf_set_resampling).

* With the threshold at 1 (the adaptive code path, resampling at every step
  in practice) the particles and ancestors equal the default path's bit for
  bit, and estimates and evidence agree to FP64 rounding: the fused one-tile
  resampling kernel against the tile chain.
* At threshold 0.5: statistical parity with the FP64 oracle's adaptive filter
  (oracle.sir_run) on Lorenz 63 and the lattice, including the fraction of
  steps that resample; on the linear-Gaussian model the ensemble converges to
  the Kalman mean and the evidence is unbiased.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(spec, M, N, y, seed, tau, var):
    est, res = np.empty((len(y), M)), []
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        if tau is not None:
            f.set_resampling(tau)
        for t in range(len(y)):
            f.step(y[t])
            est[t] = f.estimate(pf.PF_STAT_MEAN, var=var, per_filter=True)
        out = (est, f.get_state(), f.get_ancestors(), f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True))
    return out


@pytest.mark.parametrize("lattice", [False, True])
def test_threshold_one_matches_the_default_path(lattice):
    spec = W.fhn_lattice(J=8) if lattice else W.lorenz63()
    _, y = oracle.simulate(spec, 5, W.SEED_FHN_OBS if lattice else W.SEED_LORENZ_OBS)
    y = y.astype(np.float32)
    # filters of one tile (<= 1024 particles) and of several: the default path resamples the
    # former in one fused kernel each, the adaptive path takes the tile chain for every filter
    N = np.array([1500, 40, 1024, 2049, 300, 7], dtype=np.int32)
    a = _run(spec, len(N), N, y, 3, None, 1)
    b = _run(spec, len(N), N, y, 3, 1.0, 1)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.allclose(a[0], b[0], rtol=1e-10, atol=1e-12) and np.allclose(a[3], b[3], rtol=1e-12)


@pytest.mark.parametrize("lattice", [False, True])
def test_adaptive_matches_the_oracle(lattice):
    spec = W.fhn_lattice(J=8) if lattice else W.lorenz63()
    T = 12 if lattice else 30
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS if lattice else W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    M, N, var = (64, 64, 9) if lattice else (96, 512, 1)
    est = np.empty((T, M))
    res = np.empty((T, M))
    with pf.EnsembleFilter(spec, M, N, 71) as f:
        f.set_resampling(0.5)
        for t in range(T):
            f.step(y32[t])
            est[t] = f.estimate(pf.PF_STAT_MEAN, var=var, per_filter=True)
            res[t] = f.estimate(pf.PF_STAT_ESS, per_filter=True) < 0.5 * N
    ro = oracle.sir_run(spec, M, N, T, y32.astype(np.float64), seed=72, ess_threshold=0.5, est_idx=[var])
    assert 0.0 < res.mean() < 1.0
    assert abs(res.mean() - ro["resampled"].mean()) < 0.15, (res.mean(), ro["resampled"].mean())
    for t in (0, T // 2, T - 1):
        a, b = est[t], ro["est"][t, :, 0]
        se = math.sqrt(a.var(ddof=1) / M + b.var(ddof=1) / M)
        assert abs(a.mean() - b.mean()) <= 4.5 * se + 1e-9, (t, a.mean(), b.mean(), se)


def test_adaptive_converges_to_kalman_and_is_unbiased():
    spec = W.linear_gaussian()
    T = 12
    _, y = oracle.simulate(spec, T, 3)
    y32 = y.astype(np.float32)
    m, _, _ = oracle.kalman(spec, y32.astype(np.float64))
    M, N = 256, 2048
    with pf.EnsembleFilter(spec, M, N, seed=5) as f:
        f.set_resampling(0.5)
        for t in range(T):
            f.step(y32[t])
            per = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
            ens = f.estimate(pf.PF_STAT_MEAN, var=-1)
            se = per.std(axis=0, ddof=1) / math.sqrt(M)
            assert np.all(np.abs(ens - m[t]) <= 4.5 * se + 1e-3), (t, ens, m[t], se)
    scalar = W.linear_gaussian(K=1, dt=0.5, sigma=1.0, sigma_obs=1.0, A=[[0.5]], obs_idx=[0])
    ys = np.array([[1.5], [1.8]], dtype=np.float32)
    _, _, ll = oracle.kalman(scalar, ys.astype(np.float64))
    M = 1 << 17
    for N in (4, 64):
        with pf.EnsembleFilter(scalar, M, N, seed=500 + N) as f:
            f.set_resampling(0.5)
            for t in range(2):
                f.step(ys[t])
                ratio = np.exp(f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True) - ll[t])
                assert abs(ratio.mean() - 1.0) < 4.5 * ratio.std() / math.sqrt(M), (N, t, ratio.mean())


def test_adaptive_mode_rules():
    spec = W.lorenz63()
    with pf.EnsembleFilter(spec, 2, 64, 1) as f:
        f.set_resampling(0.5)
        with pytest.raises(pf.PFError) as e:
            f.propagate(np.zeros(2, dtype=np.float32))
        assert e.value.status == pf.PF_EUNSUPPORTED
        with pytest.raises(pf.PFError) as e:
            f.set_auxiliary(True)
        assert e.value.status == pf.PF_EUNSUPPORTED
        f.set_resampling(-1.0)
        f.propagate(np.zeros(2, dtype=np.float32))
        f.resample()
