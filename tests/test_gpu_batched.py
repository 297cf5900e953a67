"""Ragged batches in one context, the launch autotuner, and the learned
proposal over a ragged batch (through the C ABI).

* The autotuner (pf_autotune) leaves the filter where it was: state, log-weights,
  time and estimates unchanged, and the steps after it give the same particles
  and ancestors as an untuned twin (resampling is exact integer arithmetic, so
  no launch shape can change it); estimates agree to FP64 summation order.
* Filters of a ragged batch are independent: filter m's numbers do not depend
  on the other filters' records or particle counts.
* A ragged batch of lattice filters with the learned proposal agrees with the
  FP64 oracle's proposal filter on the same counts (statistically, over the
  batch: the mixture of per-filter estimates has the same mean on both sides).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _theta():
    th = mlp.unpack(mlp.init_params(2, out_scale=0.0))
    th["b3"] = np.array([0.1, -0.08, 0.05, 0.02])
    th["W3"][1, :6] = 0.01
    return mlp.pack(th)


@pytest.mark.parametrize("spec_name", ["fhn8", "lorenz"])
def test_autotune_preserves_the_filter(spec_name):
    spec = W.fhn_lattice(J=8) if spec_name == "fhn8" else W.lorenz63()
    T = 5
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS if spec_name == "fhn8" else W.SEED_LORENZ_OBS)
    y = y.astype(np.float32)
    N = W.ragged_counts(6, 40, 900, seed=3)
    outs = []
    for tune in (False, True):
        with pf.EnsembleFilter(spec, len(N), N, 17) as f:
            for t in range(2):
                f.step(y[t])
            if tune:
                x0, l0, e0 = f.get_state(), f.get_logw(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
                z0 = f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)
                ppc, threads, nodes = f.autotune()
                assert (ppc >= 1 if spec.kind == W.FHN else ppc == 0) and threads in (64, 128, 256)
                assert nodes in ((2, 4) if spec.kind == W.FHN else (1,))
                assert f.t == 2
                assert np.array_equal(f.get_state(), x0) and np.array_equal(f.get_logw(), l0)
                assert np.array_equal(f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True), e0)
                assert np.array_equal(f.estimate(pf.PF_STAT_LOG_Z, per_filter=True), z0)
                assert f.autotune() == (ppc, threads, nodes)  # cached per shape
            for t in range(2, T):
                f.step(y[t])
            outs.append((f.get_state(), f.get_ancestors(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True),
                         f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)))
    (xa, aa, ea, za), (xb, ab, eb, zb) = outs
    assert np.array_equal(xa, xb) and np.array_equal(aa, ab)
    assert np.allclose(ea, eb, rtol=1e-9, atol=1e-12)
    assert np.allclose(za, zb, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("J,proposal", [(8, False), (20, False), (6, False), (8, True), (20, True)])
def test_lattice_schedules_give_identical_filters(J, proposal):
    """Two, four or eight nodes per thread and any number of particles per CTA: the
    same particles, log-weights and ancestors bit for bit (the four-node
    kernels keep the pair kernels' arithmetic and reduction order), with the
    bootstrap transition and with the learned proposal's last sub-step."""
    spec = W.fhn_lattice(J=J)
    T = 3
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS)
    y = y.astype(np.float32)
    N = W.ragged_counts(4, 30, 300, seed=J)
    scheds = [(2, 1, 0), (2, 0, 0), (0, 0, 0)] + ([(4, 1, 0), (4, 0, 128)] if J % 4 == 0 else []) \
        + ([(8, 1, 0), (8, 0, 0)] if J % 8 == 0 else [])
    outs = []
    for nodes, ppc, rt in scheds:
        with pf.EnsembleFilter(spec, len(N), N, 23) as f:
            f.set_schedule(nodes, ppc, rt)
            if proposal:
                f.set_proposal(_theta(), 0.1)
            for t in range(T):
                f.step(y[t])
            outs.append((f.get_state(), f.get_logw(), f.get_ancestors(),
                         f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)))
    for x, l, a, e in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(l, outs[0][1]) and np.array_equal(a, outs[0][2])
        assert np.allclose(e, outs[0][3], rtol=1e-12, atol=1e-15)
    if J % 4 != 0:
        with pf.EnsembleFilter(spec, 1, 10, 1) as f, pytest.raises(pf.PFError):
            f.set_schedule(4, 0, 0)
    if J % 8 != 0:
        with pf.EnsembleFilter(spec, 1, 10, 1) as f, pytest.raises(pf.PFError):
            f.set_schedule(8, 0, 0)


@pytest.mark.parametrize("proposal", [False, True])
def test_ragged_lattice_filters_are_independent(proposal):
    spec = W.fhn_lattice(J=8)
    T = 3
    N = W.ragged_counts(5, 20, 700, seed=8)
    M = len(N)
    rows = np.stack([oracle.simulate(spec, T, W.SEED_FHN_OBS, record=r)[1].astype(np.float32) for r in range(M)],
                    axis=1)  # T x M x dy

    def run(obs):
        with pf.EnsembleFilter(spec, M, N, 4) as f:
            if proposal:
                f.set_proposal(_theta(), 0.1)
            for t in range(T):
                f.step(obs[t], per_filter=True)
            return f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True), f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)

    e, z = run(rows)
    for m in (0, 3):
        em, zm = run(np.broadcast_to(rows[:, m:m + 1], rows.shape).copy())
        assert np.array_equal(em[m], e[m]) and zm[m] == z[m]


def test_ragged_batch_with_learned_proposal_matches_the_oracle():
    spec = W.fhn_lattice(J=8)
    T = 3
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS)
    y = y.astype(np.float32)
    N = W.ragged_counts(600, 16, 256, seed=5)
    M, node = len(N), 9
    theta = _theta()
    with pf.EnsembleFilter(spec, M, N, 51) as f:
        f.set_proposal(theta, 0.0)
        eg = []
        for t in range(T):
            f.step(y[t])
            eg.append(f.estimate(pf.PF_STAT_MEAN, var=node, per_filter=True))
    eg = np.array(eg)
    ro = oracle.bf_run_proposal(spec, theta, M, N, T, y.astype(np.float64), seed=52, est_idx=[node], ess_frac=0.0)
    for t in range(T):
        a, b = eg[t], ro["est"][t, :, 0]
        se = math.sqrt(a.var(ddof=1) / M + b.var(ddof=1) / M)
        assert abs(a.mean() - b.mean()) <= 4.5 * se, (t, a.mean(), b.mean(), se)


def test_user_stream_and_graph_branches_give_the_same_filter():
    """A context on a caller stream (pf_set_stream) with filters of one tile and of several (the
    step graph forks the fused one-tile resampling onto the context's second stream and joins it
    back): the same particles, ancestors and estimates as on the context's own stream, step by
    step, through graph replays and asynchronous estimate reads."""
    spec = W.lorenz63()
    _, y = oracle.simulate(spec, 6, W.SEED_LORENZ_OBS)
    y = y.astype(np.float32)
    N = np.array([3000, 700, 1024, 64, 5000, 1], dtype=np.int32)
    outs = []
    for use_stream in (False, True):
        st = torch.cuda.Stream() if use_stream else None
        with pf.EnsembleFilter(spec, len(N), N, 12) as f:
            if st is not None:
                f.set_stream(st.cuda_stream)
            ens = []
            for t in range(6):
                f.step(y[t])
                ens.append(f.estimate_async(pf.PF_STAT_MEAN, var=-1).wait())
            outs.append((f.get_state(), f.get_ancestors(), np.array(ens),
                         f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True)))
    a, b = outs
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])

