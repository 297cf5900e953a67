"""GPU parity of the filter's building blocks against the FP64 oracle (through the C ABI).

Tolerances (FP32 state on the GPU vs FP64 in the oracle):
* Philox words: bit-exact.
* Box-Muller normals: |z_gpu - z| <= 1e-5 (|z| + 1): the uniforms are exact;
  FP32 -2 ln u1 (range reduction + artanh series, a few ulp), v rsqrt(v) (about
  2 ulp) and the hardware sine/cosine
  on [-pi, pi) (absolute error below 2^-21, plus pi 2^-24 from rounding the
  angle) times R <= sqrt(48 ln 2) = 5.77 bound the error by ~4e-6 + 1e-6 |z|.
* Propagated states after a full observation interval from identical inputs:
  |x_gpu - x| <= 1e-5 max(|x|, rms of the component over the batch).
* Log-weights: |l_gpu - l| <= 1e-5 max(|l|, 1), with l the oracle's likelihood
  at the GPU's propagated states (so the check isolates the weight step; the
  states are checked on their own above).
"""
import numpy as np
import pytest

import oracle
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATE_RTOL = 1e-5


def assert_state_close(xg, xo, rtol=STATE_RTOL):
    xg = np.asarray(xg, dtype=np.float64)
    rms = np.sqrt(np.mean(xo ** 2, axis=0, keepdims=True))
    scale = np.maximum(np.abs(xo), rms)
    err = np.abs(xg - xo) / np.maximum(scale, 1e-30)
    assert np.max(err) <= rtol, f"max scaled error {np.max(err):.3e} at {np.unravel_index(np.argmax(err), err.shape)}"


def ids(N, M):
    pid = np.concatenate([np.arange(n) for n in np.broadcast_to(N, (M,))]).astype(np.int32)
    fid = np.repeat(np.arange(M), np.broadcast_to(N, (M,))).astype(np.int32)
    return pid, fid


# ------------------------------------------------------------------ generator
def test_philox_bit_exact():
    ctr = W.random_counters(1 << 16, seed=1)
    ctr[:64] = 0
    ctr[64:128] = 0xFFFFFFFF
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_out = torch.empty_like(d_ctr)
    for key in [(0, 0), (0xDEADBEEF, 0x12345678), (0xFFFFFFFF, 0xFFFFFFFF)]:
        pf.pf_rng_philox(d_ctr, key[0], key[1], d_out)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.philox(ctr, *key))


def test_philox_known_answers_on_the_device():
    """The device generator reproduces the published Philox4x32-10 known-answer vectors."""
    from test_oracle_rng import philox_kat

    for c, k, o in philox_kat():
        d_ctr = torch.from_numpy(c[None, :].view(np.int32).copy()).cuda()
        d_out = torch.empty_like(d_ctr)
        pf.pf_rng_philox(d_ctr, int(k[0]), int(k[1]), d_out)
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy().view(np.uint32)[0], o), (c, k)


def test_normals_match_oracle():
    ctr = W.random_counters(1 << 20, seed=2)  # 4M normals: u1 within 2^-20 of 1 is sampled
    seed = 0x0123456789ABCDEF
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_z = torch.empty((len(ctr), 4), dtype=torch.float32, device="cuda")
    pf.pf_rng_normals(d_ctr, seed, d_z)
    torch.cuda.synchronize()
    z = oracle.normals(ctr, seed)
    err = np.abs(d_z.cpu().numpy() - z) / (np.abs(z) + 1.0)
    assert err.max() <= 1e-5, err.max()


def test_propagation_noise_is_the_stateless_normals_bit_for_bit():
    """The small-model propagation draws its normals two particles per packed FP32 instruction;
    pf_rng_normals draws them one at a time. With zero drift, unit noise scale (sigma sqrt(dt) = 1),
    one sub-step and a zero state, a propagated particle is exactly the normal it drew
    (fma(1, z, 0) = z), so the two generators must agree bit for bit at the propagation's counters
    (particle, t = 1, filter, dynamics stream << 24 | block 0), on ragged filters whose threads
    carry two particles each (and repeat the last one past a sub-tile's end)."""
    spec = W.linear_gaussian(K=1, dt=1.0, sigma=1.0, A=[[0.0]], obs_idx=[0])
    N = np.array([257, 64, 1000, 3], dtype=np.int32)
    seed = 0x5EED0F00D
    with pf.EnsembleFilter(spec, len(N), N, seed) as f:
        f.set_state(np.zeros(int(N.sum()), dtype=np.float32), 0)
        f.propagate(np.zeros(1, dtype=np.float32))
        x = f.get_state().reshape(-1)
    fid = np.repeat(np.arange(len(N)), N).astype(np.uint32)
    pid = np.concatenate([np.arange(n) for n in N]).astype(np.uint32)
    ctr = np.stack([pid, np.ones_like(pid), fid, np.full_like(pid, 3 << 24)], axis=1).astype(np.uint32)
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_z = torch.empty((len(ctr), 4), dtype=torch.float32, device="cuda")
    pf.pf_rng_normals(d_ctr, seed, d_z)
    torch.cuda.synchronize()
    z = d_z.cpu().numpy()[:, 0]
    assert np.array_equal(x.view(np.uint32), z.view(np.uint32))


# ------------------------------------------------------------------ prior and propagation
SMALL_SPECS = {
    "lorenz63": lambda: W.lorenz63(),
    "lg1": lambda: W.linear_gaussian(A=[[0.3]], obs_idx=[0]),
    "lg2": lambda: W.linear_gaussian(A=[[0.5, -1.0], [1.0, 0.5]], obs_idx=[1]),
    "lg3": lambda: W.linear_gaussian(),
    "lg4": lambda: W.linear_gaussian(A=np.diag([0.1, 0.2, 0.3, 0.4]).tolist(), obs_idx=[0, 3]),
}


@pytest.mark.parametrize("name", list(SMALL_SPECS))
def test_prior_matches_oracle(name):
    spec = SMALL_SPECS[name]()
    M, N, seed = 3, 777, 0xC0FFEE
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        xg = f.get_state()
    pid, fid = ids(N, M)
    xo = oracle.prior(spec, pid, fid, seed)
    # x0 = mean + sigma0 z: the normals' error bound 1e-5 (|z| + 1) carries over
    assert_state_close(xg, xo, rtol=1e-5)


@pytest.mark.parametrize("name", list(SMALL_SPECS))
@pytest.mark.parametrize("t", [1, 7])
def test_propagate_and_weights_match_oracle(name, t):
    spec = SMALL_SPECS[name]()
    M, N, seed = 3, 1500, 77  # ragged tail: 1500 = 1024 + 476
    x0 = W.random_states(spec, M * N, seed=5).astype(np.float32)
    y = np.linspace(-2.0, 3.0, spec.dy).astype(np.float32)
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.set_state(x0, t - 1)
        f.propagate(y)
        xg = f.get_state()
        lg = f.get_logw()
    pid, fid = ids(N, M)
    xo = oracle.propagate(spec, x0.astype(np.float64), pid, fid, t, seed)
    assert_state_close(xg, xo)
    # a3 on its own: the oracle's likelihood at the GPU's propagated states
    lo = oracle.loglik(spec, xg.astype(np.float64), y.astype(np.float64))
    assert np.max(np.abs(lg - lo) / np.maximum(np.abs(lo), 1.0)) <= 1e-5


def test_lorenz_full_size_sampled():
    """Lorenz at M * N = 2^20 (the bench launch), sampled particles vs the oracle one by one."""
    spec = W.lorenz63()
    M, N, seed = 64, 1 << 14, 2024
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        x0 = f.get_state()
        f.propagate(np.array([1.0, 20.0], dtype=np.float32))
        xg = f.get_state()
    rng = np.random.default_rng(0)
    sample = rng.choice(M * N, size=3000, replace=False)
    pid, fid = (sample % N).astype(np.int32), (sample // N).astype(np.int32)
    xo = oracle.propagate(spec, x0[sample].astype(np.float64), pid, fid, 1, seed)
    assert_state_close(xg[sample], xo)


def test_lorenz_sweep_one_context_sampled():
    """The timed launch configuration: the seven M*N = 2^20 rows of the sweep as one context of
    5461 filters (N from 2^20 down to 256; the tile chain for filters of several tiles, the fused
    kernel for the others).  Sampled particles of the propagation against the oracle one by one;
    for one filter of every size, the resampling against the oracle's systematic resampling of
    the GPU's log-weights, the gather, the per-filter means and the normaliser."""
    spec = W.lorenz63()
    N = np.concatenate([np.full(M, n, dtype=np.int32) for M, n in W.lorenz_sweep()])
    off = np.concatenate([[0], np.cumsum(N)])
    seed = 2025
    y = oracle.simulate(spec, 1, W.SEED_LORENZ_OBS)[1][0].astype(np.float32)
    with pf.EnsembleFilter(spec, len(N), N, seed) as f:
        x0 = f.get_state()
        f.propagate(y)
        xg = f.get_state()
        lg = f.get_logw()
        f.resample()
        anc = f.get_ancestors()
        x1 = f.get_state()
        logZ = f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)
        est = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
        ens = f.estimate(pf.PF_STAT_MEAN, var=-1)
    rng = np.random.default_rng(5)
    sample = rng.choice(int(off[-1]), size=2000, replace=False)
    fid = (np.searchsorted(off, sample, side="right") - 1).astype(np.int32)
    pid = (sample - off[fid]).astype(np.int32)
    xo = oracle.propagate(spec, x0[sample].astype(np.float64), pid, fid, 1, seed)
    assert_state_close(xg[sample], xo)
    lo = oracle.loglik(spec, xg[sample].astype(np.float64), y.astype(np.float64))
    assert np.max(np.abs(lg[sample] - lo) / np.maximum(np.abs(lo), 1.0)) <= 1e-5
    first = np.concatenate([[0], np.cumsum([M for M, _ in W.lorenz_sweep()])[:-1]])
    for m in list(first) + [len(N) - 1]:  # the first filter of each row and the very last one
        a, b = off[m], off[m + 1]
        l = lg[a:b].astype(np.float64)
        nrm = oracle.normalise(l)
        assert logZ[m] == pytest.approx(nrm["logZ"], rel=1e-6)
        w = np.exp(l - nrm["max"])
        exp = oracle.systematic(w, oracle.resample_u(seed, int(m), 1))
        got = anc[a:b]
        assert np.all(np.diff(got) >= 0) and got.min() >= 0 and got.max() < b - a
        # FP32 exp moves a systematic boundary only when a grid point falls within ~1e-7 of a C_k
        assert np.sum(got != exp) <= max(2, (b - a) // 1000), (m, b - a)
        src = xg[a + got]
        assert np.array_equal(x1[a:b], src)
        ref = src.astype(np.float64).mean(axis=0)
        assert np.all(np.abs(est[m] - ref) <= 1e-6 * np.abs(src).astype(np.float64).mean(axis=0) + 1e-12)
    assert np.allclose(ens, est.mean(axis=0), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ lattice
def fhn_spec(J, **kw):
    return W.fhn_lattice(J=J, **kw)


@pytest.mark.parametrize("J,M,N", [(2, 2, 5), (2, 3, 17), (4, 3, 11), (8, 3, 40), (20, 2, 9), (40, 1, 3)])
def test_fhn_prior_and_propagate_match_oracle(J, M, N):
    spec = fhn_spec(J)
    seed = 99
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        x_init = f.get_state()
        pid, fid = ids(N, M)
        assert_state_close(x_init, oracle.prior(spec, pid, fid, seed), rtol=1e-5)
        x0 = W.random_states(spec, M * N, seed=J).astype(np.float32)
        y = np.random.default_rng(J).uniform(0.0, 1.0, spec.dy).astype(np.float32)
        for t in (1, 9):  # t = 9 crosses the end of the stimulus (200 sub-steps)
            f.set_state(x0, t - 1)
            f.propagate(y)
            xg = f.get_state()
            lg = f.get_logw()
            xo = oracle.propagate(spec, x0.astype(np.float64), pid, fid, t, seed)
            assert_state_close(xg, xo)
            lo = oracle.loglik(spec, xg.astype(np.float64), y.astype(np.float64))
            assert np.max(np.abs(lg - lo) / np.maximum(np.abs(lo), 1.0)) <= 1e-5
            f.resample()


def test_fhn_full_size_sampled():
    """The 40 x 40 lattice at M = 32, N = 1024 (the full workload) in the schedule
    the autotuner picks, as the bench runs it; sampled particles."""
    spec = fhn_spec(40)
    M, N, seed = 32, 1024, 31
    _, y = oracle.simulate(spec, 1, W.SEED_FHN_OBS)
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.autotune()
        x0 = f.get_state()
        f.propagate(y[0].astype(np.float32))
        xg = f.get_state()
        lg = f.get_logw()
    rng = np.random.default_rng(1)
    sample = rng.choice(M * N, size=24, replace=False)
    pid, fid = (sample % N).astype(np.int32), (sample // N).astype(np.int32)
    xo = oracle.propagate(spec, x0[sample].astype(np.float64), pid, fid, 1, seed)
    assert_state_close(xg[sample], xo)
    lo = oracle.loglik(spec, xg[sample].astype(np.float64), y[0].astype(np.float32).astype(np.float64))
    assert np.max(np.abs(lg[sample] - lo) / np.maximum(np.abs(lo), 1.0)) <= 1e-5


def test_ragged_full_size_sampled():
    """The ragged batch at full size -- 256 filters of the 20 x 20 lattice, N log-uniform in
    [64, 4096], 250,979 particles in one context -- in the layout and the autotuned schedule the
    bench runs it in: one bootstrap interval from the prior, sampled particles against the oracle."""
    spec = fhn_spec(W.RAGGED["J"])
    N = W.ragged_counts(W.RAGGED["n_filters"], W.RAGGED["n_lo"], W.RAGGED["n_hi"])
    M, seed = len(N), 41
    _, y = oracle.simulate(spec, 1, W.SEED_FHN_OBS)
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.autotune()
        x0 = f.get_state()
        f.propagate(y[0].astype(np.float32))
        xg = f.get_state()
        lg = f.get_logw()
    pid, fid = ids(N, M)
    rng = np.random.default_rng(4)
    sample = rng.choice(int(N.sum()), size=32, replace=False)
    xo = oracle.propagate(spec, x0[sample].astype(np.float64), pid[sample], fid[sample], 1, seed)
    assert_state_close(xg[sample], xo)
    lo = oracle.loglik(spec, xg[sample].astype(np.float64), y[0].astype(np.float32).astype(np.float64))
    assert np.max(np.abs(lg[sample] - lo) / np.maximum(np.abs(lo), 1.0)) <= 1e-5


# ------------------------------------------------------------------ record simulator
@pytest.mark.parametrize("name", ["lorenz63", "lg3"])
def test_simulate_matches_oracle_small(name):
    spec = SMALL_SPECS[name]()
    T, seed = 200, W.SEED_LORENZ_OBS
    xg, yg = pf.pf_simulate(spec, T, seed, record=3)
    xo, yo = oracle.simulate(spec, T, seed, record=3)
    # FP64 on both sides; Lorenz amplifies rounding differences chaotically
    assert np.max(np.abs(xg - xo) / (np.abs(xo) + 1.0)) <= 1e-7
    assert np.max(np.abs(yg - yo.astype(np.float32)) / (np.abs(yo) + 1.0)) <= 1e-6


def test_simulate_matches_oracle_lattice():
    spec = fhn_spec(12)
    T, seed = 12, W.SEED_FHN_OBS
    xg, yg = pf.pf_simulate(spec, T, seed)
    xo, yo = oracle.simulate(spec, T, seed)
    assert np.max(np.abs(xg - xo)) <= 1e-10
    assert np.max(np.abs(yg - yo.astype(np.float32)) / (np.abs(yo) + 1.0)) <= 1e-6


@pytest.mark.parametrize("N", [64, 1024])
def test_fhn_full_size_one_step(N):
    """One complete step of the 40 x 40 lattice (K = 20) from identical states:
    propagated states and log-weights against the oracle, the per-filter log Z,
    the ancestors against the oracle's systematic resampling of the GPU's own
    log-weights (an FP32 exp moves a boundary only where a grid point lies
    within ~1e-7 of a prefix value), the gather fused with the per-filter means
    bit for bit, and the means within 1e-6."""
    spec = fhn_spec(40)
    M, seed = 2, 57
    _, y = oracle.simulate(spec, 1, W.SEED_FHN_OBS)
    y32 = y[0].astype(np.float32)
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        x0 = f.get_state()
        f.propagate(y32)
        xg = f.get_state()
        lg = f.get_logw()
        f.resample()
        anc = f.get_ancestors()
        x1 = f.get_state()
        logZ = f.estimate(pf.PF_STAT_LOG_Z, per_filter=True)
        est = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)
        ens = f.estimate(pf.PF_STAT_MEAN, var=-1)
    rng = np.random.default_rng(8)
    sample = np.arange(M * N) if N <= 64 else np.sort(rng.choice(M * N, size=96, replace=False))
    pid, fid = (sample % N).astype(np.int32), (sample // N).astype(np.int32)
    xo = oracle.propagate(spec, x0[sample].astype(np.float64), pid, fid, 1, seed)
    assert_state_close(xg[sample], xo)
    lo = oracle.loglik(spec, xg.astype(np.float64), y32.astype(np.float64))
    assert np.max(np.abs(lg - lo) / np.maximum(np.abs(lo), 1.0)) <= 1e-5
    for m in range(M):
        a, b = m * N, (m + 1) * N
        l = lg[a:b].astype(np.float64)
        nrm = oracle.normalise(l)
        assert logZ[m] == pytest.approx(nrm["logZ"], rel=1e-6)
        exp = oracle.systematic(np.exp(l - nrm["max"]), oracle.resample_u(seed, m, 1))
        got = anc[a:b]
        assert np.all(np.diff(got) >= 0) and got.min() >= 0 and got.max() < N
        assert np.sum(got != exp) <= max(2, N // 1000), (m, np.sum(got != exp))
        src = xg[a + got]
        assert np.array_equal(x1[a:b], src)
        ref = src.astype(np.float64).mean(axis=0)
        assert np.all(np.abs(est[m] - ref) <= 1e-6 * np.abs(src).astype(np.float64).mean(axis=0) + 1e-12)
    assert np.allclose(ens, est.mean(axis=0), rtol=1e-12, atol=1e-12)
