"""GPU resampling and normalisation against the FP64 oracle (through the C ABI).

* Stateless systematic resampling: ancestors bit-exact against the oracle
  given identical FP64 weights and uniforms, for ragged filters spanning
  several tiles (1024 particles), ties, zeros, spikes and N = 1.
* In-context resampling from FP32 log-weights: the GPU computes the weights
  with FP32 exp, so ancestors are compared with the oracle's (FP64 exp)
  allowing the rare boundary moved by one FP32 rounding; offspring counts obey
  the floor/ceil invariant; log Z, ESS and log G match within 1e-6 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["lognormal", "spike", "ties", "sparse", "uniform"]


def run_stateless(N_list, kind_of, seed):
    N_list = np.asarray(N_list, dtype=np.int32)
    ws = [W.random_weights(int(n), seed=seed + i, kind=kind_of(i)) for i, n in enumerate(N_list)]
    us = W.random_uniforms(len(N_list), seed=seed)
    w = np.concatenate(ws)
    d_w = torch.from_numpy(w).cuda()
    d_u = torch.from_numpy(us).cuda()
    d_anc = torch.empty(len(w), dtype=torch.int32, device="cuda")
    nbytes = pf.pf_systematic_scratch_bytes(len(N_list), len(w))
    d_scr = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    pf.pf_systematic_resample(N_list, d_w, d_u, d_anc, d_scr)
    torch.cuda.synchronize()
    got = d_anc.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(N_list)])
    for i, n in enumerate(N_list):
        exp = oracle.systematic(ws[i], float(us[i]))
        assert np.array_equal(got[off[i]:off[i + 1]], exp), (i, n, kind_of(i))


@pytest.mark.parametrize("kind", KINDS)
def test_systematic_bit_exact_ragged(kind):
    run_stateless([1, 2, 3, 1023, 1024, 1025, 3000, 4096, 17, 64], lambda i: kind, seed=10 + len(kind))


def test_systematic_bit_exact_mixed_many_filters():
    N = W.ragged_counts(256, 64, 4096)
    run_stateless(N, lambda i: KINDS[i % len(KINDS)], seed=500)


def test_systematic_bit_exact_one_big_filter():
    run_stateless([1 << 20], lambda i: "lognormal", seed=7)
    run_stateless([(1 << 20) - 3], lambda i: "sparse", seed=8)


def test_systematic_bit_exact_at_the_maximum_size():
    """N_m = 2^24, the largest particle count the ABI accepts (q below 2^28 each), next to N = 1."""
    run_stateless([1 << 24, 1], lambda i: "lognormal", seed=9)


def test_context_at_the_maximum_size():
    """One Lorenz filter of 2^24 particles in a context with a small one: resampling against the
    oracle, gather, normaliser; one particle more is refused.  The context's weights are FP32
    exp(l - max) against the oracle's FP64 exp: their roundings add up along the 2^24-term prefix,
    so more grid points change sides than at 2^20 (0.11 % of the ancestors here); the exact
    arithmetic itself is pinned bit for bit at this size by the stateless test above, and here the
    offspring counts must stay within one of floor / ceil of N times the FP64 weights."""
    spec = W.lorenz63()
    N = np.array([1 << 24, 300], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(N)])
    seed = 31
    rng = np.random.default_rng(4)
    logw = rng.normal(-10.0, 2.0, size=int(off[-1])).astype(np.float32)
    with pf.EnsembleFilter(spec, 2, N, seed) as f:
        f.propagate(np.zeros(spec.dy, dtype=np.float32))
        xbar = f.get_state()
        f.set_logw(logw)
        f.resample()
        anc = f.get_ancestors()
        x = f.get_state()
        logZ = f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)
    for m in range(2):
        a, b = off[m], off[m + 1]
        l = logw[a:b].astype(np.float64)
        nrm = oracle.normalise(l)
        assert logZ[m] == pytest.approx(nrm["logZ"], rel=1e-6)
        exp = oracle.systematic(np.exp(l - nrm["max"]), oracle.resample_u(seed, m, 1))
        got = anc[a:b]
        assert np.sum(got != exp) <= max(2, (b - a) // 200)
        assert np.all(np.diff(got) >= 0) and got.min() >= 0 and got.max() < b - a
        w = np.exp(l - nrm["max"])
        o = np.bincount(got, minlength=b - a)
        nw = (b - a) * w / w.sum()
        assert np.all(o >= np.floor(nw) - 1) and np.all(o <= np.ceil(nw) + 1)
        sample = np.random.default_rng(m).choice(b - a, size=min(b - a, 4096), replace=False)
        assert np.array_equal(x[a + sample], xbar[a + got[sample]])
    with pytest.raises(pf.PFError) as e:
        pf.EnsembleFilter(spec, 1, (1 << 24) + 1, 1)
    assert e.value.status == pf.PF_EINVAL


def test_systematic_golden_worked_examples():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "systematic_worked.txt")
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        n, w, u, a = [f.split() for f in line.split("|")]
        w = np.array(w, dtype=np.float64)
        d_w = torch.from_numpy(w).cuda()
        d_u = torch.tensor([float(u[0])], dtype=torch.float64, device="cuda")
        d_anc = torch.empty(len(w), dtype=torch.int32, device="cuda")
        d_scr = torch.empty(pf.pf_systematic_scratch_bytes(1, len(w)), dtype=torch.uint8, device="cuda")
        pf.pf_systematic_resample([len(w)], d_w, d_u, d_anc, d_scr)
        torch.cuda.synchronize()
        assert d_anc.cpu().tolist() == [int(v) for v in a]


def _filter_with_logw(spec, M, N, seed, logw):
    f = pf.EnsembleFilter(spec, M, N, seed)
    f.propagate(np.zeros(spec.dy, dtype=np.float32))
    f.set_logw(logw)
    f.resample()
    return f


@pytest.mark.parametrize("N", [1, 100, 512, 1024, 2500])
def test_context_resampling_and_normaliser(N):
    spec = W.lorenz63()
    M, seed = 5, 4242
    rng = np.random.default_rng(N)
    logw = rng.normal(-30.0, 4.0, size=M * N).astype(np.float32)
    f = _filter_with_logw(spec, M, N, seed, logw)
    anc = f.get_ancestors()
    logZ = f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)
    ess = f.estimate(pf.PF_STAT_ESS, per_filter=True)
    logG = f.estimate(pf.PF_STAT_LOG_EVIDENCE, per_filter=True)
    f.close()
    const = -0.5 * spec.dy * math.log(2 * math.pi * spec.sigma_obs ** 2)
    mismatched = 0
    for m in range(M):
        l = logw[m * N:(m + 1) * N].astype(np.float64)
        nrm = oracle.normalise(l)
        assert logZ[m] == pytest.approx(nrm["logZ"], rel=1e-6)
        assert ess[m] == pytest.approx(nrm["ess"], rel=1e-5)
        assert logG[m] == pytest.approx(nrm["logZ"] - math.log(N) + const, rel=1e-6)
        w = np.exp(l - nrm["max"])
        exp = oracle.systematic(w, oracle.resample_u(seed, m, 1))
        a = anc[m * N:(m + 1) * N]
        mismatched += int(np.sum(a != exp))
        assert np.all(np.diff(a) >= 0)
        o = np.bincount(a, minlength=N)
        q = oracle.quantise(w)
        what = q / q.sum()
        assert np.all(o >= np.floor(N * what) - 1) and np.all(o <= np.ceil(N * what) + 1)
    # FP32 exp moves a systematic boundary only when a t_i falls within ~1e-7 of a C_k
    assert mismatched <= max(2, M * N // 1000)


def test_context_size_classes_in_one_context():
    """Filters on both sides of every boundary of the fused kernel's size classes (128, 256, 512
    threads x 4 particles) and of the tile (1024) in one context: each filter's resampling
    against the oracle, the gather, the per-filter means and the normaliser."""
    spec = W.lorenz63()
    N = np.array([1, 2, 127, 128, 129, 255, 256, 257, 511, 512, 513, 1023, 1024, 1025, 2048, 3000],
                 dtype=np.int32)
    M, seed = len(N), 77
    off = np.concatenate([[0], np.cumsum(N)])
    rng = np.random.default_rng(11)
    logw = rng.normal(-20.0, 3.0, size=int(off[-1])).astype(np.float32)
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.propagate(np.zeros(spec.dy, dtype=np.float32))
        xbar = f.get_state()
        f.set_logw(logw)
        f.resample()
        anc = f.get_ancestors()
        x = f.get_state()
        logZ = f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)
        ess = f.estimate(pf.PF_STAT_ESS, per_filter=True)
        est = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
    mismatched = 0
    for m in range(M):
        a, b = off[m], off[m + 1]
        l = logw[a:b].astype(np.float64)
        nrm = oracle.normalise(l)
        assert logZ[m] == pytest.approx(nrm["logZ"], rel=1e-6)
        assert ess[m] == pytest.approx(nrm["ess"], rel=1e-5)
        got = anc[a:b]
        exp = oracle.systematic(np.exp(l - nrm["max"]), oracle.resample_u(seed, m, 1))
        mismatched += int(np.sum(got != exp))
        assert np.all(np.diff(got) >= 0) and got.min() >= 0 and got.max() < b - a
        src = xbar[a + got]
        assert np.array_equal(x[a:b], src)
        ref = src.astype(np.float64).mean(axis=0)
        assert np.all(np.abs(est[m] - ref) <= 1e-6 * np.abs(src).astype(np.float64).mean(axis=0) + 1e-12)
    assert mismatched <= max(2, int(off[-1]) // 1000)


def test_step_kernel_counts():
    """pf_step_kernels: the kernels of the captured step graph for each resampling layout."""
    spec = W.lorenz63()
    y = np.zeros(spec.dy, dtype=np.float32)
    # small model: propagate + the tile chain (weights, scan, ancestors) + ensemble
    for N, want in (([4096, 2048], 5),
                    # propagate + one fused launch per size class present + finish + ensemble
                    ([256, 300, 1024], 1 + 3 + 1 + 1),
                    # both: propagate, chain (3), fused classes (1), finish, ensemble
                    ([2048, 100], 1 + 3 + 1 + 1 + 1)):
        with pf.EnsembleFilter(spec, len(N), N, 1) as f:
            with pytest.raises(pf.PFError):
                f.step_kernels()  # nothing captured yet
            f.step(y)
            assert f.step_kernels() == want, (N, f.step_kernels())
    lat = W.fhn_lattice(J=8)
    with pf.EnsembleFilter(lat, 2, 64, 1) as f:  # propagate, fused, finish, gather + means, ensemble
        f.step(np.zeros(lat.dy, dtype=np.float32))
        assert f.step_kernels() == 5


def test_context_gather_is_exact_and_estimate_within_fp32_partials():
    spec = W.lorenz63()
    M, N, seed = 3, 2000, 5
    rng = np.random.default_rng(3)
    f = pf.EnsembleFilter(spec, M, N, seed)
    f.propagate(np.zeros(2, dtype=np.float32))
    xbar = f.get_state()
    f.set_logw(rng.normal(0.0, 2.0, M * N).astype(np.float32))
    f.resample()
    anc = f.get_ancestors()
    x = f.get_state()
    est = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
    ens = f.estimate(pf.PF_STAT_MEAN, var=-1)
    f.close()
    for m in range(M):
        src = xbar[m * N + anc[m * N:(m + 1) * N]]
        assert np.array_equal(x[m * N:(m + 1) * N], src)
        ref = src.astype(np.float64).mean(axis=0)
        # each thread sums its 4 particles in FP32 (error <= 3 2^-24 of their
        # absolute sum), the rest is FP64
        assert np.all(np.abs(est[m] - ref) <= 1e-6 * np.abs(src).astype(np.float64).mean(axis=0))
    assert np.allclose(ens, est.mean(axis=0), rtol=1e-13, atol=1e-13)


def test_degenerate_filter_is_reported():
    spec = W.lorenz63()
    M, N = 2, 64
    logw = np.zeros(M * N, dtype=np.float32)
    logw[N:] = -np.inf
    f = _filter_with_logw(spec, M, N, 1, logw)
    with pytest.raises(pf.PFError) as e:
        f.estimate(pf.PF_STAT_MEAN, var=1)
    assert e.value.status == pf.PF_ENUMERIC and "filter 1" in str(e.value)
    with pytest.raises(pf.PFError) as e:
        f.step(np.zeros(2))
    assert e.value.status == pf.PF_ESTATE
    f.close()
