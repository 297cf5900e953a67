"""Pins for the oracle's state-space models (prior, Euler-Maruyama kernels, likelihood).

* Lorenz 63 (Sec. 4.1): the drift vanishes at the three fixed points; with the
  noise off, Euler's method converges to scipy's ODE solution at first order.
* Linear-Gaussian: the K-step Euler-Maruyama kernel has mean F^K x and
  covariance Q_K (checked against numpy's matrix power and scipy's discrete
  Lyapunov solver, then against the oracle's propagation by Monte Carlo).
* FHN lattice (Sec. 5.1, Rogers-McCulloch form): the zero-flux 5-point
  Laplacian has the cosine (DCT-II) eigenmodes with eigenvalues
  -4 sin^2(pi k / 2J) - 4 sin^2(pi l / 2J); pure diffusion conserves sum v;
  a single node converges to scipy's ODE solution; the stimulus acts only on
  the corner block and only for stim_steps sub-steps.
"""
import math

import numpy as np
import pytest
from scipy import integrate, linalg, stats

import oracle
from paper_1407_8071_gb300 import workloads as W


# ----------------------------------------------------------------- Lorenz 63
def test_lorenz_fixed_points():
    spec = W.lorenz63()
    s, r, b = spec.params
    c = math.sqrt(b * (r - 1.0))
    for p in ([0.0, 0.0, 0.0], [c, c, r - 1.0], [-c, -c, r - 1.0]):
        f = oracle.drift(spec, np.array(p))
        assert np.max(np.abs(f)) < 1e-12


def _lorenz_rhs(_, x, s, r, b):
    return [s * (x[1] - x[0]), r * x[0] - x[1] - x[0] * x[2], x[0] * x[1] - b * x[2]]


def test_lorenz_euler_converges_to_ode():
    x0 = np.array(W.LORENZ_X_STAR)
    horizon = 0.2
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        K = int(round(horizon / dt))
        spec = W.lorenz63(K=K, dt=dt, sigma=0.0)
        xe = oracle.propagate(spec, x0[None], [0], [0], t=1, seed=1)[0]
        sol = integrate.solve_ivp(_lorenz_rhs, (0.0, horizon), x0, args=tuple(spec.params), rtol=1e-12,
                                  atol=1e-12)
        errs.append(np.linalg.norm(xe - sol.y[:, -1]))
    # first-order global error: halving dt halves the error
    assert 1.7 < errs[0] / errs[1] < 2.3
    assert 1.7 < errs[1] / errs[2] < 2.3


def test_lorenz_noise_increment_moments():
    # with s = r = b = 0 the drift vanishes except -x2 in f2; at x = 0 one step
    # of the kernel is pure noise sigma sqrt(dt) z
    spec = W.lorenz63(K=1, dt=1e-2, sigma=0.5)
    spec.params = [0.0, 0.0, 0.0]
    n = 20000
    x = np.zeros((n, 3))
    xs = oracle.propagate(spec, x, np.arange(n), np.zeros(n, dtype=np.int32), t=1, seed=99)
    sd = 0.5 * math.sqrt(1e-2)
    assert np.all(np.abs(xs.mean(0)) < 4 * sd / math.sqrt(n))
    assert np.all(np.abs(xs.std(0) / sd - 1.0) < 4.0 / math.sqrt(2 * n))
    c = np.corrcoef(xs.T)
    assert np.max(np.abs(c - np.eye(3))) < 4.0 / math.sqrt(n)


# ----------------------------------------------------------- linear-Gaussian
def test_lg_transition_matches_library():
    spec = W.linear_gaussian()
    FK, QK = oracle.lg_transition(spec)
    A = np.array(spec.params).reshape(3, 3)
    F = np.eye(3) - spec.dt * A
    assert np.allclose(FK, np.linalg.matrix_power(F, spec.K), rtol=1e-13, atol=1e-15)
    # Q_K solves Q = F Q F^T + sigma^2 dt (I - F^K F^K^T)
    C = spec.sigma_dyn ** 2 * spec.dt * (np.eye(3) - FK @ FK.T)
    Q = linalg.solve_discrete_lyapunov(F, C)
    assert np.allclose(QK, Q, rtol=1e-9, atol=1e-15)


def test_lg_propagation_moments():
    spec = W.linear_gaussian(K=40, dt=1e-2, sigma=0.7)
    FK, QK = oracle.lg_transition(spec)
    x0 = np.array([1.5, -2.0, 0.5])
    n = 40000
    xs = oracle.propagate(spec, np.repeat(x0[None], n, 0), np.arange(n), np.full(n, 3), t=2, seed=4)
    mean = FK @ x0
    se = np.sqrt(np.diag(QK) / n)
    assert np.all(np.abs(xs.mean(0) - mean) < 4.5 * se)
    emp = np.cov(xs.T)
    # entrywise standard error of a sample covariance ~ sqrt((Q_ii Q_jj + Q_ij^2) / n)
    se_c = np.sqrt((np.outer(np.diag(QK), np.diag(QK)) + QK ** 2) / n)
    assert np.all(np.abs(emp - QK) < 4.5 * se_c)


def test_prior_moments_and_independence():
    spec = W.lorenz63()
    n = 20000
    x = oracle.prior(spec, np.arange(n) % 5000, np.arange(n) // 5000, seed=8)
    assert np.all(np.abs(x.mean(0) - np.array(spec.x0_mean)) < 4.0 / math.sqrt(n))
    assert np.all(np.abs(x.std(0) - 1.0) < 4.0 / math.sqrt(2 * n))
    # particles of different filters differ (the filter index is part of the counter)
    assert not np.allclose(x[:5000], x[5000:10000])


def test_loglik_is_gaussian_log_density():
    spec = W.lorenz63()
    x = W.random_states(spec, 50, seed=3)
    y = np.array([1.0, -3.0])
    l = oracle.loglik(spec, x, y)
    ref = stats.norm.logpdf(y[0], x[:, 0], spec.sigma_obs) + stats.norm.logpdf(y[1], x[:, 2], spec.sigma_obs)
    const = -spec.dy * 0.5 * math.log(2 * math.pi * spec.sigma_obs ** 2)
    assert np.allclose(l + const, ref, rtol=1e-13, atol=1e-12)


# ------------------------------------------------------------------ FHN lattice
def _fhn_diffusion_only(J, D=0.1):
    return W.fhn_lattice(J=J, sigma=0.0, c1=0.0, c2=0.0, b=0.0, stim_amp=0.0, D=D)


@pytest.mark.parametrize("k,l", [(0, 1), (1, 1), (2, 5), (7, 3)])
def test_fhn_laplacian_eigenmodes(k, l):
    J, D = 8, 0.1
    spec = _fhn_diffusion_only(J, D)
    i = np.arange(J)
    mode = np.outer(np.cos(np.pi * k * (i + 0.5) / J), np.cos(np.pi * l * (i + 0.5) / J)).ravel()
    x = np.concatenate([mode, np.zeros(J * J)])
    f = oracle.drift(spec, x)
    lam = -4.0 * math.sin(math.pi * k / (2 * J)) ** 2 - 4.0 * math.sin(math.pi * l / (2 * J)) ** 2
    assert np.allclose(f[: J * J], D * lam * mode, atol=1e-13)
    assert np.all(f[J * J:] == 0.0)


def test_fhn_diffusion_conserves_mass():
    J = 10
    spec = _fhn_diffusion_only(J)
    spec.K = 50
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.random(J * J), np.zeros(J * J)])
    xs = oracle.propagate(spec, x[None], [0], [0], t=1, seed=0)[0]
    assert abs(xs[: J * J].sum() - x[: J * J].sum()) < 1e-11
    assert xs[: J * J].std() < x[: J * J].std()  # and smooths


def test_fhn_single_node_converges_to_ode():
    p = W.FHN_PARAMS

    def rhs(_, u):
        v, w = u
        return [p["c1"] * v * (v - p["a"]) * (1 - v) - p["c2"] * v * w, p["b"] * (v - p["d"] * w)]

    u0 = np.array([0.4, 0.05])
    horizon = 20.0
    errs = []
    for dt in (0.1, 0.05, 0.025):
        K = int(round(horizon / dt))
        spec = W.fhn_lattice(J=1, K=K, dt=dt, sigma=0.0, stim_amp=0.0)
        xe = oracle.propagate(spec, u0[None], [0], [0], t=1, seed=0)[0]
        sol = integrate.solve_ivp(rhs, (0.0, horizon), u0, rtol=1e-12, atol=1e-12)
        errs.append(np.linalg.norm(xe - sol.y[:, -1]))
    assert 1.7 < errs[0] / errs[1] < 2.3
    assert 1.7 < errs[1] / errs[2] < 2.3


def test_fhn_stimulus_region_and_duration():
    J = 6
    spec = W.fhn_lattice(J=J, sigma=0.0, c1=0.0, c2=0.0, b=0.0, D=0.0, stim_amp=0.3, stim_steps=4)
    x = np.zeros(2 * J * J)
    for n, on in [(1, True), (4, True), (5, False)]:
        f = oracle.drift(spec, x, step=n)
        grid = f[: J * J].reshape(J, J)
        expect = np.zeros((J, J))
        if on:
            expect[:3, :3] = 0.3
        assert np.array_equal(grid, expect)


def test_fhn_noise_is_per_variable_and_scaled():
    J = 4
    spec = W.fhn_lattice(J=J, K=1, dt=0.05, sigma=0.01, c1=0.0, c2=0.0, b=0.0, D=0.0, stim_amp=0.0)
    n = 4000
    xs = oracle.propagate(spec, np.zeros((n, 2 * J * J)), np.arange(n), np.zeros(n, dtype=np.int32), t=1,
                          seed=5)
    sd = 0.01 * math.sqrt(0.05)
    assert np.all(np.abs(xs.std(0) / sd - 1.0) < 5.0 / math.sqrt(2 * n))
    c = np.corrcoef(xs.T)
    assert np.max(np.abs(c - np.eye(2 * J * J))) < 5.0 / math.sqrt(n)


def test_simulate_observation_noise():
    spec = W.lorenz63()
    T = 400
    x, y = oracle.simulate(spec, T, W.SEED_LORENZ_OBS)
    assert np.array_equal(x[0], np.array(W.LORENZ_X_STAR))
    e = y - x[1:][:, spec.obs_idx]
    assert abs(e.mean()) < 4.0 / math.sqrt(e.size)
    assert abs(e.std() - 1.0) < 4.0 / math.sqrt(2 * e.size)
    # trajectory matches propagating the truth with the truth stream
    x1 = oracle.propagate(spec, x[0][None], [0], [0], t=1, seed=W.SEED_LORENZ_OBS, stream=W.STREAM_TRUTH)
    assert np.array_equal(x1[0], x[1])


def test_workload_constants_are_the_papers():
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            vals[k] = [float(x) for x in v]
    spec = W.lorenz63()
    assert spec.params == pytest.approx(vals["lorenz_s"] + vals["lorenz_r"] + vals["lorenz_b"], rel=1e-15)
    assert spec.x0_mean == vals["x_star"]
    assert spec.dt == vals["lorenz_dt"][0]


# ------------------------------------------------------------ the paper's own lattice (Sec. 5.1-5.2)
def _paper(J=4, **over):
    base = dict(coupling=0.0, F=0.0, eps=0.0, F_psi=0.0)
    base.update(over)
    return W.fhn_paper(J=J, sigma=0.0, **base)


def test_paper_lattice_rest_state_is_a_fixed_point():
    """Uncoupled, unforced, unstimulated, noise-free: the resting point of
    p3(u) = v, b0 u + b1 v + b2 = 0 does not move, and S stays at l0 (pins the
    cubic's sign and the recovery equation)."""
    spec = _paper()
    x0 = np.array(spec.x0_mean)[None, :]
    x = oracle.propagate(spec, x0, [0], [0], 1, seed=1)
    for t in range(2, 40):
        x = oracle.propagate(spec, x, [0], [0], t, seed=1)
    assert np.allclose(x, x0, rtol=0, atol=1e-12)


def test_paper_lattice_node_matches_the_ode():
    """A single uncoupled node from (1, 0) follows du = p3(u) - v, dv = b0 u + b1 v + b2
    (scipy's integrator) to first order in the step."""
    from scipy.integrate import solve_ivp
    p = W.FHNP_PARAMS
    errs = []
    for dt in (1e-3, 5e-4):
        spec = _paper(J=2)
        spec.dt = dt
        nn = 4
        x = np.array([1.0] * nn + [0.0] * nn + [25.0] * nn)[None, :]
        steps = int(round(0.5 / dt))
        for t in range(1, steps + 1):
            x = oracle.propagate(spec, x, [0], [0], t, seed=1)

        def rhs(_, s):
            u, v = s
            return [-u ** 3 + p["a1"] * u - v, p["b0"] * u + p["b1"] * v + p["b2"]]
        ref = solve_ivp(rhs, (0.0, 0.5), [1.0, 0.0], rtol=1e-11, atol=1e-12).y[:, -1]
        errs.append(max(abs(x[0, 0] - ref[0]), abs(x[0, nn] - ref[1])))
    assert errs[0] < 5e-3 and 1.6 < errs[0] / errs[1] < 2.4, errs


def test_paper_lattice_forcing_pulse_and_stimulus_hold():
    """Forcing acts on the first column during the first `width` sub-steps of each
    period; a stimulus counter started at 0 keeps Psi on for l0 - 1 more steps."""
    spec = _paper(J=4, F=200.0, period_steps=30, width_steps=5, F_psi=200.0, l0=7)
    nn = 16
    u0, v0 = W.fhnp_rest_state()
    x = np.array([u0] * nn + [v0] * nn + [7.0] * nn)
    x[2 * nn + 5] = 0.0  # node (1, 1): S = 0
    ref = np.array([u0] * nn + [v0] * nn + [7.0] * nn)
    du_forced, du_psi = [], []
    xs, rs = x[None, :], ref[None, :]
    for t in range(1, 12):
        xn = oracle.propagate(spec, xs, [0], [0], t, seed=1)
        rn = oracle.propagate(_paper(J=4), rs, [0], [0], t, seed=1)  # nothing applied
        du_forced.append(xn[0, 4] - xs[0, 4] - (rn[0, 4] - rs[0, 4]))   # node (1, 0): forced column
        du_psi.append(xn[0, 5] - xs[0, 5] - (rn[0, 5] - rs[0, 5]))     # node (1, 1): stimulated
        xs, rs = xn, rn
    kick = 200.0 * spec.dt
    forced = [abs(d - kick) < 0.3 * kick for d in du_forced]
    assert forced[:5] == [True] * 5 and not any(forced[5:8])
    held = [d > 0.5 * kick for d in du_psi]
    assert held[:6] == [True] * 6 and not any(held[6:])
    assert xs[0, 2 * nn + 5] == 7.0 and xs[0, 2 * nn + 0] == 7.0


def test_paper_lattice_stimulus_picks_the_region_uniformly():
    """One node in the band (u-, u+): the stimulus region is it and its neighbours;
    with epsilon = 1 every step hits one of them, chosen uniformly (chi-square
    over seeds), together with its neighbours (S restarts at 0 on a plus shape)."""
    from scipy.stats import chisquare
    J, nn = 8, 64
    spec = _paper(J=J, eps=1.0 - 2.0 ** -30)
    u0, v0 = W.fhnp_rest_state()
    x = np.array([u0] * nn + [v0] * nn + [25.0] * nn)
    i0, j0 = 3, 4
    x[i0 * J + j0] = -1.7
    region = [(i0, j0), (i0 - 1, j0), (i0 + 1, j0), (i0, j0 - 1), (i0, j0 + 1)]
    counts = dict.fromkeys(region, 0)
    R = 2000
    for seed in range(R):
        xn = oracle.propagate(spec, x[None, :], [0], [0], 1, seed=seed)[0]
        zero = {(q // J, q % J) for q in range(nn) if xn[2 * nn + q] == 0.0}
        centre = [c for c in region if zero == {c, (c[0] - 1, c[1]), (c[0] + 1, c[1]), (c[0], c[1] - 1),
                                                (c[0], c[1] + 1)} & {(a, b) for a in range(J) for b in range(J)}]
        assert len(centre) == 1, zero
        counts[centre[0]] += 1
    assert chisquare(list(counts.values())).pvalue > 1e-3, counts
