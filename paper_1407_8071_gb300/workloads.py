"""Workload definitions and seeded input generators.

Plain data only: model constants, problem sizes, seeds, and numpy generators
for synthetic inputs (ragged particle counts, random log-weights, random
particle states).  Nothing here performs any step of the filter; the CUDA
path and the CPU oracle each compute from these inputs independently.

Workloads (arXiv:1407.8071, Secs. 4-5, in the synthetic form used here):

* LG      -- a 3-D linear-Gaussian SDE observed in x1 and x3; its exact filter is
             the Kalman filter, so it pins the particle filters (Sec. 2.2).
* LORENZ  -- stochastic Lorenz 63, Sec. 4.1: (s, r, b) = (10, 28, 8/3),
             Euler-Maruyama step 1e-3, noise 0.5 * sqrt(dt) per component,
             x1 and x3 observed every 40 steps with N(0, 1) noise,
             200 observations, prior N(x_*, I) with x_* the paper's mean.
* FHN     -- 40 x 40 lattice of stochastic FitzHugh-Nagumo nodes (Sec. 5.1,
             Rogers-McCulloch form), v observed at every 4th node in both
             axes (100 nodes) with N(0, 0.1^2) noise every 20 steps.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

LG, LORENZ63, FHN, FHN_PAPER = 0, 1, 2, 3
KIND_NAMES = {LG: "linear_gaussian", LORENZ63: "lorenz63", FHN: "fhn_lattice", FHN_PAPER: "fhn_paper_lattice"}

# Philox stream identifiers, the last counter word's top byte (both sides use
# these numbers; each side implements the generator itself).
STREAM_TRUTH, STREAM_OBS, STREAM_INIT, STREAM_DYN, STREAM_RESAMPLE, STREAM_PROPOSAL, STREAM_MISC = range(7)

# Observation-record seeds for the synthetic workloads.
SEED_LORENZ_OBS = 0x0B5E0001
SEED_FHN_OBS = 0x0F4E0003
SEED_RAGGED = 0x0A66ED05


@dataclasses.dataclass
class ModelSpec:
    """State-space model in the paper's notation: prior tau_0 = N(x0_mean, sigma0^2 I),
    kernel tau_t = K Euler-Maruyama sub-steps of the drift with noise sigma_dyn,
    likelihood g_t = N(y; x[obs_idx], sigma_obs^2 I)."""

    kind: int
    dx: int
    K: int
    dt: float
    sigma_dyn: float
    sigma0: float
    sigma_obs: float
    params: List[float]
    x0_mean: List[float]
    obs_idx: List[int]
    J: int = 0
    truth_init_random: bool = False  # truth X_0 drawn from the prior (else X_0 = x0_mean)

    @property
    def dy(self) -> int:
        return len(self.obs_idx)


# x_* of Sec. 4.1: "chosen from a typical trajectory of the deterministic Lorenz 63 model".
LORENZ_X_STAR = [-10.2410, -1.3984, -23.6752]


def lorenz63(K: int = 40, dt: float = 1e-3, sigma: float = 0.5, sigma_obs: float = 1.0,
             sigma0: float = 1.0) -> ModelSpec:
    return ModelSpec(kind=LORENZ63, dx=3, K=K, dt=dt, sigma_dyn=sigma, sigma0=sigma0, sigma_obs=sigma_obs,
                     params=[10.0, 28.0, 8.0 / 3.0], x0_mean=list(LORENZ_X_STAR), obs_idx=[0, 2])


LG_A = [[0.5, -1.0, 0.0],
        [1.0, 0.5, 0.0],
        [0.0, 0.0, 1.0]]


def linear_gaussian(K: int = 40, dt: float = 1e-3, sigma: float = 0.5, sigma_obs: float = 1.0,
                    A: Optional[list] = None, obs_idx=(0, 2), sigma0: float = 1.0) -> ModelSpec:
    A = LG_A if A is None else A
    d = len(A)
    flat = [float(a) for row in A for a in row]
    return ModelSpec(kind=LG, dx=d, K=K, dt=dt, sigma_dyn=sigma, sigma0=sigma0, sigma_obs=sigma_obs,
                     params=flat, x0_mean=[0.0] * d, obs_idx=list(obs_idx), truth_init_random=True)


# Rogers-McCulloch FitzHugh-Nagumo constants and the corner stimulus.
FHN_PARAMS = dict(a=0.13, b=0.013, c1=0.26, c2=0.1, d=1.0, D=0.1,
                  stim_amp=0.1, stim_steps=200, stim_block=3)


def fhn_obs_nodes(J: int, every: int = 4) -> List[int]:
    """Observed v-variables: nodes (i, j) with i % every == 0 and j % every == 0."""
    return [i * J + j for i in range(0, J, every) for j in range(0, J, every)]


def fhn_lattice(J: int = 40, K: int = 20, dt: float = 0.05, sigma: float = 0.01, sigma_obs: float = 0.1,
                sigma0: float = 0.05, obs_every: int = 4, **over) -> ModelSpec:
    p = dict(FHN_PARAMS)
    p.update(over)
    params = [p["a"], p["b"], p["c1"], p["c2"], p["d"], p["D"], p["stim_amp"], float(p["stim_steps"]),
              float(p["stim_block"])]
    dx = 2 * J * J
    return ModelSpec(kind=FHN, dx=dx, K=K, dt=dt, sigma_dyn=sigma, sigma0=sigma0, sigma_obs=sigma_obs,
                     params=params, x0_mean=[0.0] * dx, obs_idx=fhn_obs_nodes(J, obs_every), J=J,
                     truth_init_random=True)


# The paper's own lattice (Sec. 5.1-5.2): p3(u) = -u (u + sqrt(18/5)) (u - sqrt(18/5)),
# (b0, b1, b2) = (2.1, -0.6, 0.6), 1/D = 4.5e-3, T_d = 5e-3, forcing pulses of
# amplitude 200 every 20 time units, random stimuli of amplitude 200 held for
# l0 = 25 steps, thresholds (-1.8, -1.6), epsilon = 1e-3, noise variance 1/2 on
# U, observation variance 1/2.  Readings where the text is silent or garbled:
# the cubic's sign (as printed it makes U blow up), a 25-step forcing pulse on
# the first column, the stimulus held while any event lies in the last l0 steps.
FHNP_PARAMS = dict(a3=-1.0, a2=0.0, a1=18.0 / 5.0, a0=0.0, b0=2.1, b1=-0.6, b2=0.6, coupling=4.5e-3, F=200.0,
                   period_steps=4000, width_steps=25, forced_cols=1, u_lo=-1.8, u_hi=-1.6, eps=1e-3,
                   F_psi=200.0, l0=25)


def fhnp_rest_state(p=FHNP_PARAMS):
    """The node's resting point: p3(u) = v and b0 u + b1 v + b2 = 0 (the real root)."""
    # p3(u) + (b0 u + b2) / b1 = 0
    c = [p["a3"], p["a2"], p["a1"] + p["b0"] / p["b1"], p["a0"] + p["b2"] / p["b1"]]
    roots = np.roots(c)
    u = float(min(roots, key=lambda r: abs(r.imag)).real)
    return u, -(p["b0"] * u + p["b2"]) / p["b1"]


def fhnp_obs_nodes(J: int = 32, zones: int = 5, size: int = 2) -> List[int]:
    """5 x 5 equally spaced zones of 2 x 2 nodes (Sec. 5.2, Fig. 3): zone corners at
    offset + k * spacing, spacing = J / zones rounded down, centred."""
    sp = J // zones
    off = (J - sp * (zones - 1) - size) // 2
    out = []
    for a in range(zones):
        for b in range(zones):
            for di in range(size):
                for dj in range(size):
                    out.append((off + a * sp + di) * J + off + b * sp + dj)
    return out


def fhn_paper(J: int = 32, K: int = 1, dt: float = 5e-3, sigma: float = math.sqrt(0.5),
              sigma_obs: float = math.sqrt(0.5), sigma0: float = 0.05, zones: int = 5, **over) -> ModelSpec:
    p = dict(FHNP_PARAMS)
    p.update(over)
    params = [p["a3"], p["a2"], p["a1"], p["a0"], p["b0"], p["b1"], p["b2"], p["coupling"], p["F"],
              float(p["period_steps"]), float(p["width_steps"]), float(p["forced_cols"]), p["u_lo"], p["u_hi"],
              float(round(p["eps"] * (1 << 24))), p["F_psi"], float(p["l0"])]
    u0, v0 = fhnp_rest_state(p)
    nn = J * J
    x0 = [u0] * nn + [v0] * nn + [float(p["l0"])] * nn
    obs = fhnp_obs_nodes(J, zones) if J >= 2 * zones else list(range(nn))
    return ModelSpec(kind=FHN_PAPER, dx=3 * nn, K=K, dt=dt, sigma_dyn=sigma, sigma0=sigma0, sigma_obs=sigma_obs,
                     params=params, x0_mean=x0, obs_idx=obs, J=J, truth_init_random=True)


# ---------------------------------------------------------------------------
# Problem sizes
# ---------------------------------------------------------------------------
LORENZ_SMALL = dict(M=4, N=512, T=200)                     # CPU-oracle size
LORENZ_SWEEP_M = [1, 4, 16, 64, 256, 1024, 4096]           # M * N = 2^20
LORENZ_BUDGET = 1 << 20
FHN_FULL = dict(M=32, N=1024, T=100, J=40)
RAGGED = dict(n_filters=256, J=20, n_lo=64, n_hi=4096)


def lorenz_sweep():
    return [(m, LORENZ_BUDGET // m) for m in LORENZ_SWEEP_M]


def ragged_counts(n_filters: int = 256, lo: int = 64, hi: int = 4096, seed: int = SEED_RAGGED) -> np.ndarray:
    """N_m = round(2^U), U ~ Uniform(log2 lo, log2 hi): log-uniform particle counts."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log2(lo), math.log2(hi), size=n_filters)
    return np.clip(np.rint(2.0 ** u), lo, hi).astype(np.int32)


# ---------------------------------------------------------------------------
# Seeded synthetic inputs for component tests
# ---------------------------------------------------------------------------
def random_weights(N: int, seed: int, kind: str = "lognormal") -> np.ndarray:
    """Unnormalised weights in [0, 1] with max 1, in several shapes (ties, zeros, spikes)."""
    rng = np.random.default_rng(seed)
    if kind == "lognormal":
        l = rng.normal(0.0, 3.0, size=N)
    elif kind == "spike":
        l = rng.normal(-60.0, 5.0, size=N)
        l[rng.integers(0, N)] = 0.0
    elif kind == "ties":
        l = rng.integers(-3, 1, size=N).astype(np.float64)
    elif kind == "sparse":
        l = np.where(rng.random(N) < 0.1, rng.normal(0.0, 1.0, size=N), -800.0)
        l[rng.integers(0, N)] = 0.0
    elif kind == "uniform":
        l = np.zeros(N)
    else:
        raise ValueError(kind)
    w = np.exp(l - l.max())
    return w


def random_uniforms(n: int, seed: int) -> np.ndarray:
    """u in [0, 1) on the 2^-32 grid (the form the filters draw)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.float64) * 2.0 ** -32


def random_counters(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)


def random_states(spec: ModelSpec, n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """n x dx particle states spread around the prior mean."""
    rng = np.random.default_rng(seed)
    x0 = np.asarray(spec.x0_mean, dtype=np.float64)
    if spec.kind == FHN:
        v = rng.uniform(-0.1, 1.0, size=(n, spec.dx // 2))
        w = rng.uniform(0.0, 0.3, size=(n, spec.dx // 2))
        return np.concatenate([v, w], axis=1) * scale
    return x0[None, :] + scale * rng.normal(0.0, 3.0, size=(n, spec.dx))
