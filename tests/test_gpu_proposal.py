"""The learned proposal inside the GPU lattice filter (through the C ABI).

* A network with a zero output layer, and tuple recording without a network,
  reproduce the bootstrap filter bit for bit (same normals, same arithmetic).
* A proposal that ignores the observation collapses the ESS: every filter
  falls back to the transition (PF_STAT_FALLBACK = 1) and the step equals the
  bootstrap filter's bit for bit.
* A non-trivial proposal keeps the posterior: GPU ensemble means agree with the
  FP64 oracle's proposal filter over many independent filters (both use the
  transition's normals and BF16 network weights).
* Element-wise parity of one proposal interval from identical states
  (oracle.propagate_proposal): with exact network outputs (W3 = 0) to FP32
  rounding; with a non-trivial network within the bounds derived from the
  network-output bound (tests/_mlp_bounds.py).
* Recorded tuples: the standardised residuals of the transition's own step
  are the normals it drew (mean 0, variance 1), inputs end with y.
* Training on recorded tuples lowers the held-out loss, and the trained
  proposal still estimates the bootstrap filter's posterior.
"""
import math

import numpy as np
import pytest

import oracle
import _mlp_bounds
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


def test_zero_network_on_a_side_the_four_node_kernels_skip():
    """J = 6: the bootstrap filter's sub-steps run in the two-node kernel, whose node pair takes the
    packed FP32 pipes, while the learned path's last sub-step runs in the two-node proposal kernel
    with the scalar helpers and scalar Box-Muller. A zero network must still reproduce the bootstrap
    filter bit for bit: the scalar and the packed forms round alike."""
    spec = W.fhn_lattice(J=6)
    _, y = oracle.simulate(spec, 4, W.SEED_FHN_OBS)
    y = y.astype(np.float32)
    e0, _, x0 = _run(spec, 3, 50, 5, y)
    e1, fb, x1 = _run(spec, 3, 50, 5, y, theta=mlp.init_params(1, out_scale=0.0))
    assert np.array_equal(e0, e1) and np.array_equal(x0, x1)
    assert fb.sum() == 0


def test_bad_proposal_falls_back_to_the_transition(record):
    th = mlp.unpack(mlp.init_params(3, out_scale=0.0))
    th["b3"] = np.array([40.0, 40.0, -3.0, -3.0])
    M, N, seed = 4, 64, 9
    e0, _, x0 = _run(SPEC, M, N, seed, record)
    e1, fb, x1 = _run(SPEC, M, N, seed, record, theta=mlp.pack(th))
    assert fb.min() == 1.0
    assert np.array_equal(e0, e1) and np.array_equal(x0, x1)


@pytest.mark.parametrize("span", [1, 4, SPEC.K])
def test_folded_gather_with_the_learned_proposal(record, span):
    """Learned-proposal steps fold the resampling's gather into the next step's
    ordinary sub-steps (which load each particle's ancestor row themselves) when
    the proposal's span leaves some; the halves pf_propagate / pf_resample copy
    the resampled rows instead, and a read in between writes a pending gather out.
    All three give the same particles, estimates and ancestors bit for bit (a span
    of the whole interval takes the copy in every form)."""
    theta = _moderate_proposal()
    N = np.array([300, 40, 150], dtype=np.int32)
    outs = []
    for mode in ("step", "phases", "step+read"):
        with pf.EnsembleFilter(SPEC, len(N), N, 21) as f:
            f.set_proposal(theta, 0.1)
            f.set_proposal_span(span)
            for t in range(4):
                if mode == "phases":
                    f.propagate(record[t])
                    f.resample()
                else:
                    f.step(record[t])
                    if mode == "step+read" and t % 2 == 0:
                        f.get_state()
            outs.append((f.get_state(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True),
                         f.get_ancestors(), f.estimate(pf.PF_STAT_FALLBACK, per_filter=True)))
    for x, e, a, fb in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(e, outs[0][1])
        assert np.array_equal(a, outs[0][2]) and np.array_equal(fb, outs[0][3])


def test_span_and_recording_changes_between_folded_steps(record):
    """Changing the proposal's span or arming tuple recording between steps switches a
    context between the folded and the copying form while a gather may be pending;
    the results must equal those of the same schedule taken as copying halves."""
    theta = _moderate_proposal()
    N = np.array([260, 33, 128], dtype=np.int32)
    X = torch.empty((20000, 51), dtype=torch.float32, device="cuda")
    R = torch.empty((20000, 2), dtype=torch.float32, device="cuda")
    schedule = [(1, False), (SPEC.K, False), (1, False), (1, True), (1, False), (4, False)]
    outs = []
    for halves in (False, True):
        with pf.EnsembleFilter(SPEC, len(N), N, 33) as f:
            f.set_proposal(theta, 0.1)
            for t, (span, rec) in enumerate(schedule):
                f.set_proposal_span(span)
                if rec:
                    f.record_tuples(X, R)
                if halves:
                    f.propagate(record[t])
                    f.resample()
                else:
                    f.step(record[t])
                if rec:
                    f.record_tuples(None, None)
            outs.append((f.get_state(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True), f.get_ancestors()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


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
    rises, and the posterior means agree with the bootstrap filter's.  The
    posterior comparison runs with many particles per filter (N = 2048): each
    filter's estimate carries a bias of order 1/N (Theorem 1) that differs
    between the two proposals, and at small N it is not small against the
    standard error of a mean over many filters."""
    spec = W.fhn_lattice(J=8, K=1, sigma=0.05, sigma_obs=0.02)
    T = 24
    _, y_train = oracle.simulate(spec, T, W.SEED_FHN_OBS, record=1)
    _, y_eval = oracle.simulate(spec, T, W.SEED_FHN_OBS, record=2)
    X, R, n = proposal.collect_tuples(spec, 64, 256, y_train.astype(np.float32), seed=6, capacity=400_000, stride=2)
    theta, _ = proposal.train(proposal.initial_theta(12), X, R, epochs=4, batch=4096, lr=2e-3)
    skip, node = 4, 0

    def run(M, N, seed):
        ess, est = {}, {}
        for name, th in (("bootstrap", None), ("learned", theta)):
            with pf.EnsembleFilter(spec, M, N, seed) as f:
                if th is not None:
                    f.set_proposal(th, 0.1)
                e, m = [], []
                for t in range(T):
                    f.step(y_eval[t].astype(np.float32))
                    e.append(f.estimate(pf.PF_STAT_ESS, per_filter=True))
                    m.append(f.estimate(pf.PF_STAT_MEAN, var=node, per_filter=True))
            ess[name], est[name] = np.array(e)[skip:], np.array(m)[skip:]
        return ess, est

    M, N = 256, 128
    ess, _ = run(M, N, 61)
    gain = ess["learned"].mean() / ess["bootstrap"].mean()
    print(f"mean ESS/N bootstrap {ess['bootstrap'].mean() / N:.3f}, learned {ess['learned'].mean() / N:.3f}, "
          f"gain {gain:.2f}")
    assert gain > 1.15, gain
    M, N = 48, 2048
    _, est = run(M, N, 62)
    for t in range(0, T - skip, 5):
        a, b = est["bootstrap"][t], est["learned"][t]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)


def _one_proposal_interval(J, K, theta, M, N, seed=77, span=1):
    """From identical FP32 states, one observation interval with the proposal on
    its last `span` sub-steps (no fallback): the GPU's proposed states and
    log-weights, and the oracle's proposal step from the same states."""
    spec = W.fhn_lattice(J=J, K=K)
    _, y = oracle.simulate(spec, 3, W.SEED_FHN_OBS)
    y32 = y.astype(np.float32)
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.step(y32[0])
        x0 = f.get_state()
        f.set_proposal(theta, 0.0)
        f.set_proposal_span(span)
        f.propagate(y32[1])
        xg = f.get_state().astype(np.float64)
        lg = f.get_logw().astype(np.float64)
    pid, fid = np.tile(np.arange(N), M), np.repeat(np.arange(M), N)
    y1 = y32[1].astype(np.float64)
    xo, xb, lw, o, zm, rows = oracle.propagate_proposal(spec, theta, x0.astype(np.float64), pid, fid, 2, seed, y1,
                                                        span=span)
    lo = oracle.loglik(spec, xo, y1) + lw
    return spec, x0, xg, lg, xo, lo, o, zm, rows, y1


def _observed_mask(spec):
    nn = spec.J * spec.J
    obs = np.zeros(spec.dx, dtype=bool)
    obs[np.asarray(spec.obs_idx)] = True
    obs[nn + np.asarray(spec.obs_idx)] = True
    return obs


def _rel(xg, xo):
    rms = np.sqrt(np.mean(xo ** 2, axis=0, keepdims=True))
    return np.abs(xg - xo) / np.maximum(np.abs(xo), rms)


@pytest.mark.parametrize("J,K,N", [(8, 20, 64), (8, 1, 64), (40, 20, 16)])
def test_proposal_step_with_exact_network_outputs(J, K, N):
    """A network whose outputs are its output biases (W3 = 0): both sides then
    have the same o exactly, and the proposal step -- residual mean and scale,
    the draw with the transition's normal, log g + sum (log p - log q) -- differs
    only by FP32 rounding: states within 1e-5 relative everywhere, log-weights
    within the FP32 accumulation bound of their terms."""
    th = mlp.unpack(mlp.init_params(1, out_scale=0.0))
    th["b3"] = np.array([0.35, -0.25, 0.4, -0.3])
    theta = mlp.pack(th).astype(np.float32).astype(np.float64)
    spec, x0, xg, lg, xo, lo, o, zm, rows, y1 = _one_proposal_interval(J, K, theta, 2, N)
    assert np.all(o == th["b3"].astype(np.float32).astype(np.float64))
    assert np.max(_rel(xg, xo)) <= 1e-5
    # the proposal moved every observed component away from the transition's candidate
    xb = oracle.propagate(spec, x0.astype(np.float64), np.tile(np.arange(N), 2), np.repeat(np.arange(2), N), 2, 77)
    assert np.min(np.abs(xo - xb)[:, _observed_mask(spec)]) > 0
    # log-weights: the oracle's log g at the GPU's states plus its own sum of
    # log p - log q; they differ by the FP32 accumulation of the 3 dy terms and
    # the rounding of r = (x' - m) / h if the GPU forms it from x' and m
    h = spec.sigma_dyn * np.sqrt(spec.dt)
    s_ = np.clip(o[..., 2:], -3.0, 3.0)
    r = o[..., :2] + np.exp(s_) * zm[..., :2]
    q = s_ + zm[..., :2] ** 2 / 2.0 - r ** 2 / 2.0
    lw = q.sum(axis=(1, 2))
    lgx = oracle.loglik(spec, xg, y1)
    nn, nodes = spec.J * spec.J, np.asarray(spec.obs_idx)
    xp = np.stack([xg[:, nodes], xg[:, nn + nodes]], axis=2)
    canc = 2.0 ** -22 * (np.abs(zm[..., 2:]) + np.abs(xp)) / h
    tol = (_mlp_bounds.gamma(3 * spec.dy) * (np.abs(lgx) + np.abs(q).sum(axis=(1, 2)))
           + (np.abs(r) * canc + canc ** 2).sum(axis=(1, 2)) + 1e-6)
    assert np.all(np.abs(lg - (lgx + lw)) <= tol), np.max(np.abs(lg - (lgx + lw)) / tol)
    # and the oracle's own weights agree with that reconstruction of them
    assert np.allclose(lo, oracle.loglik(spec, xo, y1) + lw, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("J,K,N", [(8, 20, 64), (8, 1, 64), (40, 20, 16)])
def test_proposal_step_matches_oracle_elementwise(J, K, N):
    """A non-trivial network (non-zero W3 and b3): unobserved components within
    1e-5 relative; observed ones within the bound the network-output bound
    implies (tests/_mlp_bounds.step_bounds), and at most 2 % of them beyond the
    bound without rounding flips; log-weights within their derived bound."""
    p = mlp.unpack(mlp.init_params(5, out_scale=0.3))
    rng = np.random.default_rng(105)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0.0, 0.1, p[k].shape)
    theta = mlp.pack(p).astype(np.float32).astype(np.float64)
    spec, x0, xg, lg, xo, lo, o, zm, rows, y1 = _one_proposal_interval(J, K, theta, 2, N)
    assert np.abs(o[..., :2]).max() > 0.05 and np.abs(o[..., 2:]).max() > 0.05
    obs = _observed_mask(spec)
    assert np.max(_rel(xg, xo)[:, ~obs]) <= 1e-5
    # network inputs: the states after K - 1 sub-steps, known to 1e-5 of their size on the GPU
    if K > 1:
        rms_v = np.sqrt(np.mean(rows[..., :25] ** 2))
        rms_w = np.sqrt(np.mean(rows[..., 25:50] ** 2))
        x_tol = np.concatenate([1e-5 * np.maximum(np.abs(rows[..., :25]), rms_v),
                                1e-5 * np.maximum(np.abs(rows[..., 25:50]), rms_w),
                                np.zeros(rows.shape[:2] + (1,))], axis=2).reshape(-1, 51)
    else:
        x_tol = 0.0
    dx, dx_nf, dl = _mlp_bounds.step_bounds(spec, theta, o, zm, rows, xo, y1, x_tol)
    nn, nodes = spec.J * spec.J, np.asarray(spec.obs_idx)
    d = np.stack([np.abs(xg - xo)[:, nodes], np.abs(xg - xo)[:, nn + nodes]], axis=2)
    assert np.all(d <= dx + 1e-12), np.max(d / dx)
    assert np.mean(d > dx_nf + 1e-12) <= 0.02, np.mean(d > dx_nf)
    assert np.all(np.abs(lg - lo) <= dl + 1e-9), np.max(np.abs(lg - lo) / dl)


def test_zero_network_over_the_whole_interval_is_the_bootstrap_filter(record):
    M, N, seed = 3, 70, 5
    e0, _, x0 = _run(SPEC, M, N, seed, record)
    with pf.EnsembleFilter(SPEC, M, N, seed) as f:
        f.set_proposal(mlp.init_params(1, out_scale=0.0), 0.1)
        f.set_proposal_span(SPEC.K)
        est = []
        for t in range(len(record)):
            f.step(record[t])
            est.append(f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True))
        x1 = f.get_state()
    assert np.array_equal(e0, np.array(est)) and np.array_equal(x0, x1)


@pytest.mark.parametrize("span", [2, 20])
def test_proposal_over_several_sub_steps_with_exact_network_outputs(span):
    """The proposal on the last `span` sub-steps with outputs known exactly on both
    sides (W3 = 0): states within 1e-5 relative, log-weights within the FP32
    accumulation bound of their terms over the span's sub-steps."""
    th = mlp.unpack(mlp.init_params(1, out_scale=0.0))
    th["b3"] = np.array([0.35, -0.25, 0.4, -0.3])
    theta = mlp.pack(th).astype(np.float32).astype(np.float64)
    spec, x0, xg, lg, xo, lo, o, zm, rows, y1 = _one_proposal_interval(8, 20, theta, 2, 64, span=span)
    assert np.max(_rel(xg, xo)) <= 1e-5
    lgx = oracle.loglik(spec, xo, y1)
    lw = lo - lgx  # the oracle's sum over the span of log p - log q
    # Bound: FP32 accumulation of the dy log g terms and of the 2 dy span terms s + z^2/2 - r^2/2, plus,
    # per term, the rounding of r = (x' - m) / h formed from FP32 x' and m: |dr| <= 2^-22 (|m| + |x'|) / h,
    # moving the term by at most (|r| + |dr|) |dr|, with |r| <= |o_mu| + e^s |z| and |z| <= 6.
    h = spec.sigma_dyn * np.sqrt(spec.dt)
    n_terms = 2 * spec.dy * span
    dr = 2.0 ** -22 * 2.0 * np.max(np.abs(xo)) / h
    r_max = np.max(np.abs(th["b3"][:2]) + np.exp(np.clip(th["b3"][2:], -3, 3)) * 6.0)
    q_max = 3.0 + 18.0 + r_max ** 2 / 2.0
    tol = (_mlp_bounds.gamma(spec.dy + n_terms) * (np.abs(lgx) + n_terms * q_max)
           + n_terms * (r_max + dr) * dr + 1e-5 * (np.abs(lgx) + 1.0))
    assert np.all(np.abs(lg - lo) <= tol), np.max(np.abs(lg - lo) / tol)
    # the bound is far below what a wrong term would move: dropping z^2/2 alone shifts by ~ n_terms / 2
    assert np.max(tol) < 0.05 * n_terms


def test_proposal_over_the_whole_interval_matches_the_oracle_statistically(record):
    theta = _moderate_proposal()
    T = 4
    y = record[:T]
    M, N, node = 1000, 48, 9
    with pf.EnsembleFilter(SPEC, M, N, 31) as f:
        f.set_proposal(theta, 0.0)
        f.set_proposal_span(SPEC.K)
        eg = []
        for t in range(T):
            f.step(y[t])
            eg.append(f.estimate(pf.PF_STAT_MEAN, var=node, per_filter=True))
    ro = oracle.bf_run_proposal(SPEC, theta, M, N, T, y.astype(np.float64), seed=32, est_idx=[node], ess_frac=0.0,
                                span=SPEC.K)
    for t in range(T):
        a, b = eg[t], ro["est"][t, :, 0]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)
