"""The learned proposal inside the GPU lattice filter (through the C ABI).

* A network with a zero output layer, and tuple recording without a network,
  reproduce the bootstrap filter bit for bit (same normals, same arithmetic).
* A proposal that ignores the observation collapses the ESS: every filter
  falls back to the transition (PF_STAT_FALLBACK = 1) and the step equals the
  bootstrap filter's bit for bit.
* A non-trivial proposal keeps the posterior: GPU ensemble means agree with the
  FP64 oracle's proposal filter over many independent filters (both use the
  transition's normals and BF16 network weights).
* Recorded tuples: the standardised residuals of the transition's own step
  are the normals it drew (mean 0, variance 1), inputs end with y.
* Training on recorded tuples lowers the held-out loss, and the trained
  proposal still estimates the bootstrap filter's posterior.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1407_8071_gb300 import pf, proposal, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC = W.fhn_lattice(J=8)


@pytest.fixture(scope="module")
def record():
    _, y = oracle.simulate(SPEC, 6, W.SEED_FHN_OBS)
    return y.astype(np.float32)


def _run(spec, M, N, seed, y, theta=None, ess_frac=0.1, record=None):
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        if theta is not None:
            f.set_proposal(theta, ess_frac)
        if record is not None:
            f.record_tuples(*record)
        est, fb = [], []
        for t in range(len(y)):
            f.step(y[t])
            est.append(f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True))
            fb.append(f.estimate(pf.PF_STAT_FALLBACK, per_filter=True))
        return np.array(est), np.array(fb), f.get_state()


def test_zero_network_and_recording_are_the_bootstrap_filter(record):
    M, N, seed = 3, 70, 5
    e0, _, x0 = _run(SPEC, M, N, seed, record)
    e1, fb1, x1 = _run(SPEC, M, N, seed, record, theta=mlp.init_params(1, out_scale=0.0))
    assert np.array_equal(e0, e1) and np.array_equal(x0, x1)
    assert fb1.sum() == 0
    X = torch.empty((10000, 51), dtype=torch.float32, device="cuda")
    R = torch.empty((10000, 2), dtype=torch.float32, device="cuda")
    e2, _, x2 = _run(SPEC, M, N, seed, record, record=(X, R))
    assert np.array_equal(e0, e2) and np.array_equal(x0, x2)


def test_bad_proposal_falls_back_to_the_transition(record):
    th = mlp.unpack(mlp.init_params(3, out_scale=0.0))
    th["b3"] = np.array([40.0, 40.0, -3.0, -3.0])
    M, N, seed = 4, 64, 9
    e0, _, x0 = _run(SPEC, M, N, seed, record)
    e1, fb, x1 = _run(SPEC, M, N, seed, record, theta=mlp.pack(th))
    assert fb.min() == 1.0
    assert np.array_equal(e0, e1) and np.array_equal(x0, x1)


def _moderate_proposal():
    th = mlp.unpack(mlp.init_params(1, out_scale=0.0))
    th["b3"] = np.array([0.15, -0.1, 0.1, 0.05])
    th["W3"][0, :8] = 0.01
    return mlp.pack(th)


def test_proposal_matches_the_oracle_statistically(record):
    theta = _moderate_proposal()
    T = 4
    y = record[:T]
    M, N, node = 1000, 48, 9
    eg, fbg, _ = _run(SPEC, M, N, 31, y, theta=theta, ess_frac=0.0)
    ro = oracle.bf_run_proposal(SPEC, theta, M, N, T, y.astype(np.float64), seed=32, est_idx=[node], ess_frac=0.0)
    assert fbg.sum() == 0
    for t in range(T):
        a, b = eg[t, :, node], ro["est"][t, :, 0]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)


def test_recorded_tuples(record):
    M, N, stride = 4, 100, 3
    kept = sum((N + stride - 1) // stride for _ in range(M))
    cap = 10 ** 6
    X = torch.empty((cap, 51), dtype=torch.float32, device="cuda")
    R = torch.empty((cap, 2), dtype=torch.float32, device="cuda")
    with pf.EnsembleFilter(SPEC, M, N, 2) as f:
        f.record_tuples(X, R, stride=stride)
        for t in range(3):
            f.step(record[t])
            assert f.recorded_tuples() == (t + 1) * kept * SPEC.dy
    n = 3 * kept * SPEC.dy
    Xh, Rh = X[:n].cpu().numpy(), R[:n].cpu().numpy()
    # the last input is y at the node (rounded to BF16 like every input)
    ys = np.concatenate([np.tile(record[t], kept) for t in range(3)])
    assert np.allclose(Xh[:, 50], mlp.bf16(ys), rtol=0, atol=0)
    # bootstrap step: r = (m + h z - m) / h = z up to rounding, posterior-selected
    assert abs(Rh.mean()) < 0.1 and abs(Rh.var() - 1.0) < 0.15


def test_training_lowers_held_out_loss_and_keeps_the_posterior(record):
    y = record
    X, R, n = proposal.collect_tuples(SPEC, 64, 256, y, seed=4, capacity=200_000)
    assert n > 50_000
    cut = int(0.8 * n)
    theta0 = mlp.init_params(11, out_scale=0.0)
    theta, losses = proposal.train(theta0, X[:cut], R[:cut], epochs=3, batch=4096, lr=1e-3)
    l0 = proposal.mean_nll(theta0, X[cut:], R[cut:])
    l1 = proposal.mean_nll(theta, X[cut:], R[cut:])
    assert l1 <= l0 + 1e-3, (l0, l1)
    # the trained proposal estimates the same posterior as the bootstrap filter
    M, N, node = 400, 64, 9
    eb, _, _ = _run(SPEC, M, N, 41, y[:4])
    ep, fb, _ = _run(SPEC, M, N, 42, y[:4], theta=theta)
    for t in range(4):
        a, b = eb[t, :, node], ep[t, :, node]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)


def test_trained_network_gains_where_the_transition_noise_sits_in_the_last_sub_step():
    """What training buys: with one Euler-Maruyama sub-step per observation
    (K = 1) all the transition noise is in the step the network controls, and
    an observation sharper than that noise makes the bootstrap weights uneven.
    The trained proposal moves the observed nodes toward y: the mean ESS
    rises, and the posterior means agree with the bootstrap filter's."""
    spec = W.fhn_lattice(J=8, K=1, sigma=0.05, sigma_obs=0.02)
    T = 24
    _, y_train = oracle.simulate(spec, T, W.SEED_FHN_OBS, record=1)
    _, y_eval = oracle.simulate(spec, T, W.SEED_FHN_OBS, record=2)
    X, R, n = proposal.collect_tuples(spec, 64, 256, y_train.astype(np.float32), seed=6, capacity=400_000, stride=2)
    theta, _ = proposal.train(proposal.initial_theta(12), X, R, epochs=4, batch=4096, lr=2e-3)
    M, N, skip, node = 256, 128, 4, 0
    ess, est = {}, {}
    for name, th in (("bootstrap", None), ("learned", theta)):
        with pf.EnsembleFilter(spec, M, N, 61) as f:
            if th is not None:
                f.set_proposal(th, 0.1)
            e, m = [], []
            for t in range(T):
                f.step(y_eval[t].astype(np.float32))
                e.append(f.estimate(pf.PF_STAT_ESS, per_filter=True))
                m.append(f.estimate(pf.PF_STAT_MEAN, var=node, per_filter=True))
        ess[name], est[name] = np.array(e)[skip:], np.array(m)[skip:]
    gain = ess["learned"].mean() / ess["bootstrap"].mean()
    print(f"mean ESS/N bootstrap {ess['bootstrap'].mean() / N:.3f}, learned {ess['learned'].mean() / N:.3f}, "
          f"gain {gain:.2f}")
    assert gain > 1.15, gain
    for t in range(0, T - skip, 5):
        a, b = est["bootstrap"][t], est["learned"][t]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)
