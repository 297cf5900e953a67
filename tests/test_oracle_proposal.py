"""Pins for the oracle's learned-proposal filter (lattice model).

* Zero output layer: q equals the transition, log p - log q = 0 exactly, and
  the filter reproduces the bootstrap filter bit for bit.
* Consistency: with a non-trivial proposal the weights carry p g / q, so the
  ensemble mean over many independent filters agrees with the bootstrap
  ensemble's (both estimate the same posterior mean) -- a wrong sign or a
  dropped term in log p - log q shifts it by many standard errors (checked
  by planting a sign error in a copy of the weight formula in the test).
* Fallback: a proposal that ignores the observation and shifts the mean by
  many transition scales collapses the ESS; the filter then takes the
  transition for that step (flag 1) and matches the bootstrap filter.
* The C network forward equals the numpy oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1407_8071_gb300 import workloads as W

SPEC = W.fhn_lattice(J=8)
T = 4


@pytest.fixture(scope="module")
def record():
    _, y = oracle.simulate(SPEC, T, W.SEED_FHN_OBS)
    return y


def test_c_forward_equals_numpy():
    th = mlp.init_params(2, out_scale=0.4)
    X = np.random.default_rng(1).normal(size=(9, mlp.IN))
    assert np.array_equal(oracle.mlp_forward_c(th, X, bf16=True), mlp.forward(th, X, bf16_emulation=True)[0])
    assert np.allclose(oracle.mlp_forward_c(th, X, bf16=False), mlp.forward(th, X)[0], rtol=1e-12, atol=1e-12)


def test_zero_output_proposal_is_the_bootstrap_filter(record):
    r0 = oracle.bf_run(SPEC, 6, 48, T, record, seed=3, est_idx=[9, 70])
    r1 = oracle.bf_run_proposal(SPEC, mlp.init_params(7, out_scale=0.0), 6, 48, T, record, seed=3, est_idx=[9, 70])
    assert np.array_equal(r0["est"], r1["est"]) and np.array_equal(r0["log_G"], r1["log_G"])
    assert r1["fallback"].sum() == 0


def _moderate_proposal(seed):
    # a fixed, observation-dependent proposal: mean pulled by o_mu, scale widened by o_s
    th = mlp.unpack(mlp.init_params(seed, out_scale=0.0))
    th["b3"] = np.array([0.15, -0.1, 0.1, 0.05])
    th["W3"][0, :8] = 0.01
    return mlp.pack(th)


def test_proposal_weights_keep_the_posterior(record):
    M, N = 1000, 48
    node = 9
    rb = oracle.bf_run(SPEC, M, N, T, record, seed=11, est_idx=[node])
    # pure p g / q weights (no fallback), so the check sees the weight formula alone
    rp = oracle.bf_run_proposal(SPEC, _moderate_proposal(1), M, N, T, record, seed=12, est_idx=[node], ess_frac=0.0)
    assert rp["fallback"].sum() == 0
    for t in range(T):
        a, b = rb["est"][t, :, 0], rp["est"][t, :, 0]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)
    # and the evidence estimates agree in mean (Lemma 2 holds for the importance-weighted filter)
    ga, gb = np.exp(rb["log_G"][-1] - rb["log_G"][-1].max()), np.exp(rp["log_G"][-1] - rb["log_G"][-1].max())
    assert abs(ga.mean() - gb.mean()) < 4.5 * math.sqrt(ga.var() / M + gb.var() / M)


def test_a_planted_sign_error_would_be_caught(record):
    """The consistency check above has the power to see a wrong log p - log q:
    reweighting the proposal filter's particles by exp(-2 (log p - log q)) -- what
    a flipped sign gives -- moves the mean of a mean-shifting proposal by many
    standard errors.  Done on one step by hand with the oracle's pieces."""
    rng = np.random.default_rng(0)
    h = SPEC.sigma_dyn * math.sqrt(SPEC.dt)
    n = 200000
    m = 0.0
    mu, sd = m + 3.0 * h, 1.5 * h  # a proposal far from the transition
    x = mu + sd * rng.normal(size=n)
    lw = (-(x - m) ** 2 / (2 * h * h) - math.log(h)) - (-(x - mu) ** 2 / (2 * sd * sd) - math.log(sd))
    good = np.sum(np.exp(lw - lw.max()) * x) / np.sum(np.exp(lw - lw.max()))
    bad = np.sum(np.exp(-lw + lw.min()) * x) / np.sum(np.exp(-lw + lw.min()))
    assert abs(good - m) < 0.05 * h          # importance weights recover the transition's mean
    assert abs(bad - m) > 1.0 * h            # the flipped sign does not


def test_bad_proposal_falls_back_to_the_transition(record):
    th = mlp.unpack(mlp.init_params(3, out_scale=0.0))
    th["b3"] = np.array([40.0, 40.0, -3.0, -3.0])  # mean 40 transition scales away, narrow
    theta = mlp.pack(th)
    M, N = 5, 64
    rp = oracle.bf_run_proposal(SPEC, theta, M, N, T, record, seed=21, est_idx=[9])
    rb = oracle.bf_run(SPEC, M, N, T, record, seed=21, est_idx=[9])
    assert rp["fallback"].min() == 1.0
    assert np.array_equal(rp["est"], rb["est"])


def test_zero_output_proposal_over_the_whole_interval_is_the_bootstrap_filter(record):
    """The proposal acting on every sub-step of the interval (span K): with a zero
    output layer each sub-step draws the transition's own value and log p - log q
    is zero, so the filter is the bootstrap filter bit for bit."""
    r0 = oracle.bf_run(SPEC, 6, 48, T, record, seed=3, est_idx=[9, 70])
    r1 = oracle.bf_run_proposal(SPEC, mlp.init_params(7, out_scale=0.0), 6, 48, T, record, seed=3, est_idx=[9, 70],
                                span=SPEC.K)
    assert np.array_equal(r0["est"], r1["est"]) and np.array_equal(r0["log_G"], r1["log_G"])


@pytest.mark.parametrize("span", [2, 20])
def test_proposal_over_several_sub_steps_keeps_the_posterior(record, span):
    """With the proposal on the last `span` sub-steps, the weights carry the product
    over those sub-steps of p / q, and the ensemble mean agrees with the bootstrap
    ensemble's (no fallback: only a last-sub-step proposal has one)."""
    M, N = 600, 96
    node = 9
    rb = oracle.bf_run(SPEC, M, N, T, record, seed=31, est_idx=[node])
    rp = oracle.bf_run_proposal(SPEC, _moderate_proposal(1), M, N, T, record, seed=32, est_idx=[node], ess_frac=0.5,
                                span=span)
    assert rp["fallback"].sum() == 0  # the threshold is ignored beyond the last sub-step
    for t in range(T):
        a, b = rb["est"][t, :, 0], rp["est"][t, :, 0]
        se = math.sqrt(a.var() / M + b.var() / M)
        assert abs(a.mean() - b.mean()) < 4.5 * se, (t, a.mean(), b.mean(), se)


def test_span_one_is_the_last_sub_step_reading(record):
    theta = _moderate_proposal(2)
    a = oracle.bf_run_proposal(SPEC, theta, 4, 40, T, record, seed=5, est_idx=[9], ess_frac=0.0)
    b = oracle.bf_run_proposal(SPEC, theta, 4, 40, T, record, seed=5, est_idx=[9], ess_frac=0.0, span=1)
    assert np.array_equal(a["est"], b["est"]) and np.array_equal(a["log_G"], b["log_G"])
