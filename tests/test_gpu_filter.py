"""End-to-end GPU filters against the oracle and against the mathematics.

* Statistical parity (Lorenz 63 at the oracle size, the FHN lattice at reduced
  size): per-filter posterior-mean estimates of the GPU and of the oracle over
  R independent filters on the same record agree in mean within
  4 sqrt(s_gpu^2 / R + s_orc^2 / R) (trajectories cannot agree element-wise
  beyond one interval: Lorenz is chaotic and FP32 vs FP64 rounding flips
  resampling decisions).
* Linear-Gaussian model, where the exact filter is the Kalman filter:
  the ensemble average converges to the Kalman mean; Lemma 2 (E G_t^N equals
  the Kalman evidence); Theorem 1 (|bias| ~ 1/N); Corollary 2 (variance of the
  M-average ~ 1/(MN)).
* Checkpoint / resume is bit-identical; host and device observation paths
  agree bit for bit; argument and ordering errors.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_gpu(spec, M, N, y, seed, var):
    est = np.empty((len(y), M))
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        for t in range(len(y)):
            f.step(y[t])
            est[t] = f.estimate(pf.PF_STAT_MEAN, var=var, per_filter=True)
    return est


def z_parity(eg, eo, times):
    for t in times:
        a, b = eg[t], eo[t]
        se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        assert abs(a.mean() - b.mean()) <= 4.0 * se + 1e-9, (t, a.mean(), b.mean(), se)


def test_lorenz_statistical_parity_with_oracle():
    spec = W.lorenz63()
    T = 60
    _, y = oracle.simulate(spec, T, W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    M, N = 128, 512
    eg = run_gpu(spec, M, N, y32, seed=11, var=1)
    eo = oracle.bf_run(spec, M, N, T, y32.astype(np.float64), seed=12, est_idx=[1])["est"][:, :, 0]
    z_parity(eg, eo, [0, 9, 29, 59])


def test_fhn_statistical_parity_with_oracle():
    spec = W.fhn_lattice(J=8, K=20)
    T = 12
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS)
    y32 = y.astype(np.float32)
    M, N = 64, 64
    node = 9  # a v-variable near the stimulated corner
    eg = run_gpu(spec, M, N, y32, seed=21, var=node)
    eo = oracle.bf_run(spec, M, N, T, y32.astype(np.float64), seed=22, est_idx=[node])["est"][:, :, 0]
    z_parity(eg, eo, [0, 5, 11])


def test_ensemble_converges_to_kalman_mean():
    spec = W.linear_gaussian()
    T = 20
    _, y = oracle.simulate(spec, T, 3)
    y32 = y.astype(np.float32)
    m, _, _ = oracle.kalman(spec, y32.astype(np.float64))
    M, N = 256, 4096
    with pf.EnsembleFilter(spec, M, N, seed=1) as f:
        for t in range(T):
            f.step(y32[t])
            per = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
            ens = f.estimate(pf.PF_STAT_MEAN, var=-1)
            se = per.std(axis=0, ddof=1) / math.sqrt(M)
            assert np.all(np.abs(ens - m[t]) <= 4.5 * se + 1e-3), (t, ens, m[t], se)
            assert np.allclose(ens, per.mean(axis=0), rtol=1e-13, atol=1e-13)


SCALAR = dict(K=1, dt=0.5, sigma=1.0, sigma_obs=1.0, A=[[0.5]], obs_idx=[0])
Y_SCALAR = np.array([[1.5], [1.8]], dtype=np.float32)


def test_lemma2_unbiased_evidence():
    spec = W.linear_gaussian(**SCALAR)
    _, _, ll = oracle.kalman(spec, Y_SCALAR.astype(np.float64))
    M = 1 << 18
    for N in (4, 64):
        with pf.EnsembleFilter(spec, M, N, seed=N) as f:
            for t in range(2):
                f.step(Y_SCALAR[t])
                lg = f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True)
                ratio = np.exp(lg - ll[t])
                assert abs(ratio.mean() - 1.0) < 4.5 * ratio.std() / math.sqrt(M), (N, t, ratio.mean())


def test_theorem1_bias_and_corollary2_variance_rates():
    spec = W.linear_gaussian(**SCALAR)
    m, _, _ = oracle.kalman(spec, Y_SCALAR.astype(np.float64))
    target = m[-1, 0]
    Ns = np.array([16, 32, 64, 128, 256, 512])
    M = 1 << 19
    bias, se, var = [], [], []
    for N in Ns:
        with pf.EnsembleFilter(spec, M, int(N), seed=int(N) + 7) as f:
            for t in range(2):
                f.step(Y_SCALAR[t])
            e = f.estimate(pf.PF_STAT_MEAN, var=0, per_filter=True)
        bias.append(e.mean() - target)
        se.append(e.std() / math.sqrt(M))
        var.append(e.var())
        for Mg in (16, 1024):  # eq. eqP1: the M-average divides the variance by M
            g = e[: (M // Mg) * Mg].reshape(-1, Mg).mean(1)
            assert g.var() / (e.var() / Mg) == pytest.approx(1.0, abs=5.0 * math.sqrt(2.0 / len(g)))
    bias, se, var = map(np.asarray, (bias, se, var))
    assert np.all(np.abs(bias) > 4 * se)
    slope_b = np.polyfit(np.log(Ns), np.log(np.abs(bias)), 1, w=np.abs(bias) / se)[0]
    assert -1.15 < slope_b < -0.85, slope_b
    slope_v = np.polyfit(np.log(Ns), np.log(var), 1)[0]
    assert -1.08 < slope_v < -0.92, slope_v


def test_checkpoint_resume_is_bit_identical():
    spec = W.lorenz63()
    _, y = oracle.simulate(spec, 6, W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    M, N, seed = 4, 3000, 9
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        for t in range(3):
            f.step(y32[t])
        ckpt = f.get_state()
        for t in range(3, 6):
            f.step(y32[t])
        a = f.get_state()
        ea = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
    with pf.EnsembleFilter(spec, M, N, seed) as g:
        g.set_state(ckpt, 3)
        for t in range(3, 6):
            g.step(y32[t])
        b = g.get_state()
        eb = g.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
        assert g.t == 6
    assert np.array_equal(a, b) and np.array_equal(ea, eb)


def test_step_equals_propagate_then_resample_and_device_obs():
    spec = W.fhn_lattice(J=8)
    _, y = oracle.simulate(spec, 3, W.SEED_FHN_OBS)
    y32 = y.astype(np.float32)
    outs = []
    for mode in ("step", "phases", "device"):
        with pf.EnsembleFilter(spec, 3, 100, 5) as f:
            for t in range(3):
                if mode == "step":
                    f.step(y32[t])
                elif mode == "phases":
                    f.propagate(y32[t])
                    f.resample()
                else:
                    f.step_device(torch.from_numpy(y32[t]).cuda())
            outs.append((f.get_state(), f.estimate(pf.PF_STAT_MEAN, var=-1)))
    for x, e in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(e, outs[0][1])


def test_asynchronous_estimates_equal_synchronous():
    """pf_estimate_async read one step late (step t+1 already enqueued) gives the
    values pf_estimate gives right after step t, for every statistic it offers."""
    spec = W.lorenz63()
    _, y = oracle.simulate(spec, 6, W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    N = W.ragged_counts(9, 16, 600, seed=2)
    kinds = [(pf.PF_STAT_MEAN, -1, False), (pf.PF_STAT_MEAN, 1, False), (pf.PF_STAT_MEAN, -1, True),
             (pf.PF_STAT_MEAN, 2, True), (pf.PF_STAT_LOG_EVIDENCE, -1, True), (pf.PF_STAT_ESS, -1, True)]
    sync_vals = []
    with pf.EnsembleFilter(spec, len(N), N, 4) as f:
        for t in range(6):
            f.step(y32[t])
            sync_vals.append([f.estimate(k, var=v, per_filter=p) for k, v, p in kinds])
    with pf.EnsembleFilter(spec, len(N), N, 4) as f:
        with pytest.raises(pf.PFError) as e:
            f.estimate_async()
        assert e.value.status == pf.PF_ESTATE  # no step yet
        pending = None
        for t in range(7):
            if t < 6:
                f.step(y32[t])
            if pending is not None:  # step t is enqueued: read step t-1's statistic
                k = (t - 1) % len(kinds)
                assert np.array_equal(pending.wait(), sync_vals[t - 1][k]), (t, kinds[k])
            if t < 6:
                k, v, p = kinds[t % len(kinds)]
                pending = f.estimate_async(k, var=v, per_filter=p)
    with pf.EnsembleFilter(spec, len(N), N, 4) as f:
        pending = None
        for t in range(6):
            f.step(y32[t])
            if pending is not None:
                got = pending.wait()
                assert np.array_equal(got, sync_vals[t - 1][2]), t
            pending = f.estimate_async(pf.PF_STAT_MEAN, var=-1, per_filter=True)
        assert np.array_equal(pending.wait(), sync_vals[5][2])
        with pytest.raises(pf.PFError) as e:
            f.estimate_async(pf.PF_STAT_ESS)
        assert e.value.status == pf.PF_EUNSUPPORTED  # the M-average of ESS is formed by pf_estimate


def test_per_filter_observation_streams():
    spec = W.lorenz63()
    M, N, T = 4, 256, 3
    ys = [oracle.simulate(spec, T, W.SEED_LORENZ_OBS, record=r)[1].astype(np.float32) for r in range(M)]
    rows = np.stack(ys, axis=1)  # T x M x dy
    with pf.EnsembleFilter(spec, M, N, 3) as f:
        for t in range(T):
            f.step(rows[t], per_filter=True)
        per = f.estimate(pf.PF_STAT_MEAN, var=1, per_filter=True)
    # filter m alone on record m gives the same numbers (filters are independent)
    for m in range(M):
        with pf.EnsembleFilter(spec, M, N, 3) as g:
            for t in range(T):
                g.step(np.broadcast_to(rows[t, m], (M, 2)).copy(), per_filter=True)
            assert g.estimate(pf.PF_STAT_MEAN, var=1, per_filter=True)[m] == per[m]


def test_order_and_argument_errors():
    spec = W.lorenz63()
    with pf.EnsembleFilter(spec, 2, 64, 1) as f:
        with pytest.raises(pf.PFError) as e:
            f.resample()
        assert e.value.status == pf.PF_ESTATE
        with pytest.raises(pf.PFError) as e:
            f.estimate()
        assert e.value.status == pf.PF_ESTATE  # no step yet
        f.propagate(np.zeros(2))
        with pytest.raises(pf.PFError) as e:
            f.step(np.zeros(2))
        assert e.value.status == pf.PF_ESTATE
        f.resample()
        with pytest.raises(pf.PFError) as e:
            f.estimate(pf.PF_STAT_MEAN, var=7)
        assert e.value.status == pf.PF_EINVAL
        assert f.t == 1


def test_torch_allocator_and_injected_allocation_failure():
    spec = W.lorenz63()
    pf.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        with pf.EnsembleFilter(spec, 8, 4096, 1) as f:
            assert torch.cuda.memory_allocated() > before + 8 * 4096 * 12
            f.step(np.zeros(2))
            f.estimate()
        assert torch.cuda.memory_allocated() == before
    finally:
        pf.use_torch_allocator(False)
    # an allocator that fails on its third request -> PF_ENOMEM, nothing leaks
    calls = {"n": 0}
    import ctypes

    def alloc(nbytes, stream, user):
        calls["n"] += 1
        if calls["n"] == 3:
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)

    def free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (pf.PF_ALLOC_FN(alloc), pf.PF_FREE_FN(free))
    pf.lib().pf_set_allocator(hooks[0], hooks[1], None)
    try:
        before = torch.cuda.memory_allocated()
        with pytest.raises(pf.PFError) as e:
            pf.EnsembleFilter(spec, 2, 64, 1)
        assert e.value.status == pf.PF_ENOMEM
        assert torch.cuda.memory_allocated() == before
    finally:
        pf.use_torch_allocator(False)


@pytest.mark.parametrize("code", [pf.PF_ETIMEOUT, pf.PF_ENUMERIC])
def test_device_failure_flags_reach_the_caller(code):
    """The error word a bounded device wait (or a degenerate normaliser) sets is
    turned into the status code on both read paths, and the context refuses
    further steps.  The word is written from the host (pf_inject_error): making
    a tensor-core wait expire with MMAs in flight is not a safe test."""
    spec = W.lorenz63()
    _, y = oracle.simulate(spec, 3, W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    for path in ("sync", "async"):
        with pf.EnsembleFilter(spec, 3, 128, 21) as f:
            f.step(y32[0])
            assert np.isfinite(f.estimate(pf.PF_STAT_MEAN, var=1)).all()  # healthy before
            f.inject_error(code, filter=2)
            with pytest.raises(pf.PFError) as e:
                if path == "sync":
                    f.estimate(pf.PF_STAT_MEAN, var=1)
                else:
                    f.estimate_async(pf.PF_STAT_MEAN, var=1).wait()
            assert e.value.status == code
            if code == pf.PF_ENUMERIC:
                assert "filter 2" in str(e.value)
            else:
                assert "wait" in str(e.value)
            with pytest.raises(pf.PFError) as e2:
                f.step(y32[1])
            assert e2.value.status == pf.PF_ESTATE
    with pf.EnsembleFilter(spec, 3, 128, 21) as f:
        with pytest.raises(pf.PFError) as e:
            f.inject_error(pf.PF_EINVAL)
        assert e.value.status == pf.PF_EINVAL


def test_fhn_20x20_statistical_parity_with_oracle():
    """The ragged batch's lattice size (20 x 20, 800 variables) over ten observations."""
    spec = W.fhn_lattice(J=20, K=20)
    T = 10
    _, y = oracle.simulate(spec, T, W.SEED_FHN_OBS)
    y32 = y.astype(np.float32)
    M, N = 64, 64
    node = 21  # a v-variable inside the stimulated corner block
    eg = run_gpu(spec, M, N, y32, seed=23, var=node)
    eo = oracle.bf_run(spec, M, N, T, y32.astype(np.float64), seed=24, est_idx=[node])["est"][:, :, 0]
    z_parity(eg, eo, [0, 4, 9])


@pytest.mark.parametrize("model", ["lorenz63", "fhn", "fhn_paper"])
def test_folded_gather_equals_the_copied_state(model):
    """Bootstrap steps fold the resampling's gather into the next propagation
    (which loads each particle's ancestor itself); the two halves
    pf_propagate / pf_resample copy the resampled particles instead, and a
    read of the state in between writes a pending gather out.  All three give
    the same particles and estimates bit for bit, on ragged filters of one and
    of several tiles."""
    spec = {"lorenz63": W.lorenz63, "fhn": lambda: W.fhn_lattice(J=8),
            "fhn_paper": lambda: W.fhn_paper(J=8, zones=4)}[model]()
    _, y = oracle.simulate(spec, 4, W.SEED_LORENZ_OBS if model == "lorenz63" else W.SEED_FHN_OBS)
    y32 = y.astype(np.float32)
    N = np.array([1500, 40, 700], dtype=np.int32)
    outs = []
    for mode in ("step", "phases", "step+read"):
        with pf.EnsembleFilter(spec, len(N), N, 13) as f:
            for t in range(4):
                if mode == "phases":
                    f.propagate(y32[t])
                    f.resample()
                else:
                    f.step(y32[t])
                    if mode == "step+read" and t % 2 == 0:
                        f.get_state()
            outs.append((f.get_state(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True),
                         f.get_ancestors()))
    for x, e, a in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(e, outs[0][1]) and np.array_equal(a, outs[0][2])


def test_timed_step_is_a_step():
    """pf_step_timed advances the filter exactly as pf_step_device does and
    reports two positive device times (propagation, resampling)."""
    spec = W.lorenz63()
    _, y = oracle.simulate(spec, 3, W.SEED_LORENZ_OBS)
    d_y = torch.from_numpy(y.astype(np.float32)).cuda()
    outs = []
    for timed in (False, True):
        with pf.EnsembleFilter(spec, 3, np.array([1500, 40, 700], dtype=np.int32), 4) as f:
            for t in range(3):
                if timed:
                    a, b = f.step_timed(d_y[t])
                    assert a > 0 and b > 0
                else:
                    f.step_device(d_y[t])
            outs.append((f.get_state(), f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
