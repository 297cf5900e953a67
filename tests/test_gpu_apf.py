"""The ensemble of auxiliary particle filters on the GPU (pf_set_auxiliary).

* Statistical parity with the FP64 oracle's auxiliary filter (oracle.apf_run):
  Lorenz 63 and the lattice (ragged particle counts), per-filter weighted
  posterior means over R filters, |mean_gpu - mean_orc| <= 4.5 sqrt(s^2_gpu/R
  + s^2_orc/R).
* Linear-Gaussian model: the ensemble average converges to the Kalman mean,
  and the likelihood estimate is unbiased against the Kalman evidence.
* Launch schedules do not change the lattice filter (bit for bit).
* The two-stage step is one unit: pf_propagate is refused, and the mode does
  not combine with the learned proposal.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_apf(spec, M, N, y, seed, var, per_filter_obs=False):
    est = np.empty((len(y), M))
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.set_auxiliary(True)
        for t in range(len(y)):
            f.step(y[t], per_filter=per_filter_obs)
            est[t] = f.estimate(pf.PF_STAT_MEAN, var=var, per_filter=True)
    return est


def z_parity(eg, eo, times):
    for t in times:
        a, b = eg[t], eo[t]
        se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        assert abs(a.mean() - b.mean()) <= 4.5 * se + 1e-9, (t, a.mean(), b.mean(), se)


def test_apf_lorenz_parity_with_oracle():
    spec = W.lorenz63()
    T = 40
    _, y = oracle.simulate(spec, T, W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    M, N = 128, 512
    eg = run_apf(spec, M, N, y32, seed=41, var=1)
    eo = oracle.apf_run(spec, M, N, T, y32.astype(np.float64), seed=42, est_idx=[1])["est"][:, :, 0]
    z_parity(eg, eo, [0, 9, 19, 39])


def test_apf_lattice_parity_with_oracle_ragged():
    spec = W.fhn_lattice(J=8)
    T = 10
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS)
    y32 = y.astype(np.float32)
    N = W.ragged_counts(96, 16, 128, seed=3)
    M, node = len(N), 9
    eg = run_apf(spec, M, N, y32, seed=51, var=node)
    eo = oracle.apf_run(spec, M, N, T, y32.astype(np.float64), seed=52, est_idx=[node])["est"][:, :, 0]
    z_parity(eg, eo, [0, 4, 9])


def test_apf_converges_to_kalman_and_is_unbiased():
    spec = W.linear_gaussian()
    T = 15
    _, y = oracle.simulate(spec, T, 3)
    y32 = y.astype(np.float32)
    m, _, _ = oracle.kalman(spec, y32.astype(np.float64))
    M, N = 256, 2048
    with pf.EnsembleFilter(spec, M, N, seed=2) as f:
        f.set_auxiliary(True)
        for t in range(T):
            f.step(y32[t])
            per = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
            ens = f.estimate(pf.PF_STAT_MEAN, var=-1)
            se = per.std(axis=0, ddof=1) / math.sqrt(M)
            assert np.all(np.abs(ens - m[t]) <= 4.5 * se + 1e-3), (t, ens, m[t], se)
            ess = f.estimate(pf.PF_STAT_ESS, per_filter=True)
            assert np.all((ess > 0) & (ess <= N * (1 + 1e-9)))
    scalar = W.linear_gaussian(K=1, dt=0.5, sigma=1.0, sigma_obs=1.0, A=[[0.5]], obs_idx=[0])
    ys = np.array([[1.5], [1.8]], dtype=np.float32)
    _, _, ll = oracle.kalman(scalar, ys.astype(np.float64))
    M = 1 << 17
    for N in (4, 64):
        with pf.EnsembleFilter(scalar, M, N, seed=300 + N) as f:
            f.set_auxiliary(True)
            for t in range(2):
                f.step(ys[t])
                ratio = np.exp(f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True) - ll[t])
                assert abs(ratio.mean() - 1.0) < 4.5 * ratio.std() / math.sqrt(M), (N, t, ratio.mean())


def test_apf_lattice_schedules_and_graph_replay_identical():
    spec = W.fhn_lattice(J=8)
    T = 4
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS)
    y = y.astype(np.float32)
    N = W.ragged_counts(5, 30, 400, seed=6)
    outs = []
    for sched in ((2, 1, 0), (4, 0, 0), (4, 2, 128), (8, 0, 0)):
        with pf.EnsembleFilter(spec, len(N), N, 8) as f:
            f.set_auxiliary(True)
            f.set_schedule(*sched)
            for t in range(T):
                f.step(y[t])
            outs.append((f.get_state(), f.get_logw(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True),
                         f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True)))
    for x, l, e, g in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(l, outs[0][1])
        assert np.allclose(e, outs[0][2], rtol=1e-12, atol=1e-15) and np.allclose(g, outs[0][3], rtol=1e-12)


def test_apf_mode_rules():
    spec = W.fhn_lattice(J=8)
    with pf.EnsembleFilter(spec, 2, 32, 1) as f:
        f.set_auxiliary(True)
        with pytest.raises(pf.PFError) as e:
            f.propagate(np.zeros(spec.dy, dtype=np.float32))
        assert e.value.status == pf.PF_EUNSUPPORTED
        with pytest.raises(pf.PFError) as e:
            f.set_proposal(mlp.init_params(1), 0.1)
        assert e.value.status == pf.PF_EUNSUPPORTED
        f.set_auxiliary(False)
        f.step(np.zeros(spec.dy, dtype=np.float32))  # the bootstrap filter again
        assert f.t == 1
