"""FP64 CPU oracle for the ensemble of independent bootstrap filters (arXiv:1407.8071).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1407_8071_gb300``): the two sides meet only in the
seeded input generators of ``paper_1407_8071_gb300.workloads``, which hold
plain data and no step of the method.

Contents and what pins each (the pins live in ``tests/test_oracle_*.py``):

=====================  =============================================  ==========================================
function               paper passage                                  pinned by
=====================  =============================================  ==========================================
philox / normals       counter-based generator (Salmon et al. 2011),  Weyl constants from their definitions;
                       Box-Muller (1958)                              inverse-round round trip; chi^2, moment
                                                                      and avalanche tests
prior / propagate      Alg. 1 steps 1, 2a; eqs. eqDiscreteLorenz-1..3 LG: exact transition moments F^K x and
                       (Sec. 4.1); Sec. 5.1 lattice (Rogers-McCulloch Q_K; Lorenz: fixed points, deterministic
                       form)                                          ODE limit vs scipy; FHN: Neumann-Laplacian
                                                                      eigenmodes, mass conservation, ODE limit
loglik / normalise     Alg. 1 step 2a weights; eq. eqGtN              scipy.stats.norm / logsumexp
systematic             Alg. 1 step 2b (systematic form)               offspring counts in {floor, ceil}(N w);
                                                                      E over a u-grid of o_k = N w_k; worked
                                                                      example in tests/golden
multinomial            Alg. 1 step 2b                                 offspring mean and variance (binomial)
bf_run                 Alg. 1 x M, Def. 1, eq. eqGtN                  LG: converges to the Kalman mean; Lemma 2
                                                                      (E G = Kalman evidence); Thm. 1 bias
                                                                      ~ 1/N; Cor. 2 variance ~ 1/(MN)
apf_run                auxiliary particle filters (Pitt & Shephard),  LG: converges to the Kalman mean; E G =
                       the filter of Sec. 5.3; remark after Cor. 2    Kalman evidence (unbiased, as Lemma 2);
                                                                      Lorenz: same posterior as bf_run
sir_run                Alg. 1 with step 2b only when ESS < tau N      tau > 1: bf_run bit for bit; LG: Kalman
                       (the adaptive form of the resampling step)     mean and unbiased evidence at tau = 0.5
bf_run_proposal        Alg. 1 step 2a with an importance function     zero network = bf_run bit for bit; p g / q
                       (remark after Alg. 1; Sec. 6 footnote)         weights keep the bootstrap posterior
mlp (oracle/mlp.py)    the proposal's network                         finite-difference gradients; BF16 rounding
                                                                      against its definition
kalman                 exact filter of the LG case (Sec. 2.2)         joint-Gaussian conditioning of the whole
                                                                      record (a different method)
simulate               record generator (Sec. 4.2)                    same model code as propagate; obs noise
                                                                      moments
=====================  =============================================  ==========================================

No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None


class _OrcModel(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("dx", ctypes.c_int32), ("J", ctypes.c_int32), ("K", ctypes.c_int32),
        ("dt", ctypes.c_double), ("sigma_dyn", ctypes.c_double), ("sigma0", ctypes.c_double),
        ("sigma_obs", ctypes.c_double),
        ("dy", ctypes.c_int32), ("n_params", ctypes.c_int32),
        ("params", ctypes.POINTER(ctypes.c_double)),
        ("x0_mean", ctypes.POINTER(ctypes.c_double)),
        ("obs_idx", ctypes.POINTER(ctypes.c_int32)),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _lib.orc_resample_u.restype = ctypes.c_double
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class _Model:
    """Keeps the numpy buffers alive for as long as the ctypes struct is used."""

    def __init__(self, spec):
        self.spec = spec
        self.params = np.ascontiguousarray(spec.params, dtype=np.float64)
        self.x0 = np.ascontiguousarray(spec.x0_mean, dtype=np.float64)
        self.idx = np.ascontiguousarray(spec.obs_idx, dtype=np.int32)
        self.s = _OrcModel(spec.kind, spec.dx, spec.J, spec.K, spec.dt, spec.sigma_dyn, spec.sigma0,
                           spec.sigma_obs, len(self.idx), len(self.params),
                           _p(self.params, ctypes.c_double), _p(self.x0, ctypes.c_double),
                           _p(self.idx, ctypes.c_int32))

    @property
    def ref(self):
        return ctypes.byref(self.s)


# --------------------------------------------------------------------------
# Generator
# --------------------------------------------------------------------------
def philox(ctr: np.ndarray, key0: int, key1: int) -> np.ndarray:
    """Philox4x32-10 of each row of ctr (n x 4 uint32) under key (key0, key1)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().orc_philox_batch(ctypes.c_int64(len(ctr)), _p(ctr, ctypes.c_uint32), ctypes.c_uint32(key0),
                           ctypes.c_uint32(key1), _p(out, ctypes.c_uint32))
    return out


def normals(ctr: np.ndarray, seed: int) -> np.ndarray:
    """Four Box-Muller normals per counter row (key = seed's low and high words)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    z = np.empty((len(ctr), 4), dtype=np.float64)
    lib().orc_normals_batch(ctypes.c_int64(len(ctr)), _p(ctr, ctypes.c_uint32), ctypes.c_uint64(seed),
                            _p(z, ctypes.c_double))
    return z


def box_muller(ab: np.ndarray) -> np.ndarray:
    """Box-Muller pair of each row (a, b) of 32-bit words."""
    ab = np.ascontiguousarray(ab, dtype=np.uint32).reshape(-1, 2)
    z = np.empty((len(ab), 2), dtype=np.float64)
    lib().orc_box_muller_batch(ctypes.c_int64(len(ab)), _p(ab, ctypes.c_uint32), _p(z, ctypes.c_double))
    return z


def resample_u(seed: int, m: int, t: int) -> float:
    return lib().orc_resample_u(ctypes.c_uint64(seed), ctypes.c_int32(m), ctypes.c_int32(t))


# --------------------------------------------------------------------------
# Model steps
# --------------------------------------------------------------------------
def prior(spec, pid: Sequence[int], fid: Sequence[int], seed: int) -> np.ndarray:
    md = _Model(spec)
    pid = np.ascontiguousarray(pid, dtype=np.int32)
    fid = np.ascontiguousarray(fid, dtype=np.int32)
    x = np.empty((len(pid), spec.dx), dtype=np.float64)
    lib().orc_prior(md.ref, ctypes.c_int64(len(pid)), _p(pid, ctypes.c_int32), _p(fid, ctypes.c_int32),
                    ctypes.c_uint64(seed), _p(x, ctypes.c_double))
    return x


def propagate(spec, x: np.ndarray, pid, fid, t: int, seed: int, stream: int = 3) -> np.ndarray:
    """K Euler-Maruyama sub-steps from observation t-1 to t for each particle row of x."""
    md = _Model(spec)
    x = np.array(x, dtype=np.float64, order="C", copy=True).reshape(-1, spec.dx)
    pid = np.ascontiguousarray(pid, dtype=np.int32)
    fid = np.ascontiguousarray(fid, dtype=np.int32)
    lib().orc_propagate(md.ref, ctypes.c_int64(len(x)), _p(pid, ctypes.c_int32), _p(fid, ctypes.c_int32),
                        ctypes.c_int32(t), ctypes.c_uint64(seed), ctypes.c_int32(stream), _p(x, ctypes.c_double))
    return x


def em_step(spec, x: np.ndarray, z: np.ndarray, step: int = 1) -> np.ndarray:
    """One Euler-Maruyama step with given normals (rows of z)."""
    md = _Model(spec)
    x = np.array(x, dtype=np.float64, order="C", copy=True).reshape(-1, spec.dx)
    z = np.ascontiguousarray(z, dtype=np.float64).reshape(-1, spec.dx)
    lib().orc_em_step(md.ref, ctypes.c_int64(len(x)), ctypes.c_int64(step), _p(x, ctypes.c_double),
                      _p(z, ctypes.c_double))
    return x


def drift(spec, x: np.ndarray, step: int = 1) -> np.ndarray:
    md = _Model(spec)
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.empty_like(x)
    lib().orc_drift(md.ref, ctypes.c_int64(step), _p(x, ctypes.c_double), _p(f, ctypes.c_double))
    return f


def loglik(spec, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    md = _Model(spec)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, spec.dx)
    y = np.ascontiguousarray(y, dtype=np.float64)
    l = np.empty(len(x), dtype=np.float64)
    lib().orc_loglik(md.ref, ctypes.c_int64(len(x)), _p(x, ctypes.c_double), _p(y, ctypes.c_double),
                     _p(l, ctypes.c_double))
    return l


def normalise(l: np.ndarray) -> dict:
    l = np.ascontiguousarray(l, dtype=np.float64)
    out = np.empty(5, dtype=np.float64)
    lib().orc_normalise(ctypes.c_int64(len(l)), _p(l, ctypes.c_double), _p(out, ctypes.c_double))
    return dict(max=out[0], logZ=out[1], sum_w=out[2], sum_w2=out[3], ess=out[4])


def quantise(w: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    q = np.empty_like(w)
    lib().orc_quantise(ctypes.c_int64(len(w)), _p(w, ctypes.c_double), _p(q, ctypes.c_double))
    return q


def systematic(w: np.ndarray, u: float) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    a = np.empty(len(w), dtype=np.int32)
    lib().orc_systematic(ctypes.c_int64(len(w)), _p(w, ctypes.c_double), ctypes.c_double(u),
                         _p(a, ctypes.c_int32))
    return a


def multinomial(w: np.ndarray, U: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    a = np.empty(len(w), dtype=np.int32)
    lib().orc_multinomial(ctypes.c_int64(len(w)), _p(w, ctypes.c_double), _p(U, ctypes.c_double),
                          _p(a, ctypes.c_int32))
    return a


def simulate(spec, T: int, seed: int, record: int = 0):
    """Truth X_0..X_T (at observation times) and observations y_1..y_T."""
    md = _Model(spec)
    x = np.empty((T + 1, spec.dx), dtype=np.float64)
    y = np.empty((T, spec.dy), dtype=np.float64)
    lib().orc_simulate(md.ref, ctypes.c_int32(T), ctypes.c_uint64(seed), ctypes.c_int32(record),
                       ctypes.c_int32(1 if spec.truth_init_random else 0), _p(x, ctypes.c_double),
                       _p(y, ctypes.c_double))
    return x, y


def bf_run(spec, M: int, N, T: int, obs: np.ndarray, seed: int, resampler: str = "systematic",
           est_idx: Optional[Sequence[int]] = None, obs_per_filter: bool = False, want_pre: bool = False,
           want_final: bool = False, threads: int = 0) -> dict:
    """M independent bootstrap filters (Alg. 1) on one record, and their average (Def. 1)."""
    md = _Model(spec)
    N = np.ascontiguousarray(np.broadcast_to(np.asarray(N, dtype=np.int32), (M,)), dtype=np.int32)
    est_idx = np.ascontiguousarray(range(spec.dx) if est_idx is None else est_idx, dtype=np.int32)
    ne = len(est_idx)
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    post = np.empty((T, M, ne))
    pre = np.empty((T, M, ne)) if want_pre else None
    logG = np.empty((T, M))
    ess = np.empty((T, M))
    ens = np.empty((T, ne))
    xf = np.empty((int(N.sum()), spec.dx)) if want_final else None
    nullp = ctypes.POINTER(ctypes.c_double)()
    lib().orc_bf_run(md.ref, ctypes.c_int32(M), _p(N, ctypes.c_int32), ctypes.c_int32(T), _p(obs, ctypes.c_double),
                     ctypes.c_int32(1 if obs_per_filter else 0), ctypes.c_uint64(seed),
                     ctypes.c_int32(1 if resampler == "multinomial" else 0), ctypes.c_int32(ne),
                     _p(est_idx, ctypes.c_int32), _p(post, ctypes.c_double),
                     _p(pre, ctypes.c_double) if pre is not None else nullp,
                     _p(logG, ctypes.c_double), _p(ess, ctypes.c_double), _p(ens, ctypes.c_double),
                     _p(xf, ctypes.c_double) if xf is not None else nullp, ctypes.c_int32(threads))
    return dict(est=post, est_pre=pre, log_G=logG, ess=ess, ens=ens, x_final=xf)


class _OrcProposal(ctypes.Structure):
    _fields_ = [("theta", ctypes.POINTER(ctypes.c_float)), ("bf16", ctypes.c_int32), ("ess_frac", ctypes.c_double),
                ("span", ctypes.c_int32)]


def mlp_forward_c(theta: np.ndarray, rows: np.ndarray, bf16: bool = True) -> np.ndarray:
    """The C oracle's network forward (the one its filter uses)."""
    th = np.ascontiguousarray(theta, dtype=np.float32)
    rows = np.ascontiguousarray(rows, dtype=np.float64).reshape(-1, 51)
    out = np.empty((len(rows), 4))
    pr = _OrcProposal(_p(th, ctypes.c_float), 1 if bf16 else 0, 0.1, 1)
    lib().orc_mlp_forward(ctypes.byref(pr), ctypes.c_int64(len(rows)), _p(rows, ctypes.c_double),
                          _p(out, ctypes.c_double))
    return out


def propagate_proposal(spec, theta, x: np.ndarray, pid, fid, t: int, seed: int, y: np.ndarray, bf16: bool = True,
                       span: int = 1):
    """One interval of the learned-proposal filter for each particle row of x (lattice), the proposal
    acting on the last `span` sub-steps: returns (proposed x, the transition's candidates xb from the
    state before the last sub-step, sum of log p - log q per row,
    network outputs o [n, dy, 4], normals and transition means zm [n, dy, 4], network
    inputs rows [n, dy, 51])."""
    md = _Model(spec)
    x = np.array(x, dtype=np.float64, order="C", copy=True).reshape(-1, spec.dx)
    n = len(x)
    pid = np.ascontiguousarray(pid, dtype=np.int32)
    fid = np.ascontiguousarray(fid, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float32)
    pr = _OrcProposal(_p(th, ctypes.c_float), 1 if bf16 else 0, 0.0, int(span))
    xb, lw = np.empty_like(x), np.empty(n)
    o, zm, rows = np.empty((n, spec.dy, 4)), np.empty((n, spec.dy, 4)), np.empty((n, spec.dy, 51))
    lib().orc_propagate_proposal(md.ref, ctypes.byref(pr), ctypes.c_int64(n), _p(pid, ctypes.c_int32),
                                 _p(fid, ctypes.c_int32), ctypes.c_int32(t), ctypes.c_uint64(seed),
                                 _p(y, ctypes.c_double), _p(x, ctypes.c_double), _p(xb, ctypes.c_double),
                                 _p(lw, ctypes.c_double), _p(o, ctypes.c_double), _p(zm, ctypes.c_double),
                                 _p(rows, ctypes.c_double))
    return x, xb, lw, o, zm, rows


def patch_row_c(spec, x: np.ndarray, node: int, y: float) -> np.ndarray:
    md = _Model(spec)
    x = np.ascontiguousarray(x, dtype=np.float64)
    row = np.empty(51)
    lib().orc_patch_row(md.ref, _p(x, ctypes.c_double), ctypes.c_int32(node), ctypes.c_double(y),
                        _p(row, ctypes.c_double))
    return row


def apf_run(spec, M: int, N, T: int, obs: np.ndarray, seed: int, est_idx: Optional[Sequence[int]] = None,
            obs_per_filter: bool = False, threads: int = 0) -> dict:
    """M independent auxiliary particle filters (Pitt & Shephard) and their average (Def. 1):
    look-ahead by the noise-free Euler prediction, first-stage systematic resampling,
    second-stage weights g(y | x) / g(y | mu), weighted estimates."""
    md = _Model(spec)
    N = np.ascontiguousarray(np.broadcast_to(np.asarray(N, dtype=np.int32), (M,)), dtype=np.int32)
    est_idx = np.ascontiguousarray(range(spec.dx) if est_idx is None else est_idx, dtype=np.int32)
    ne = len(est_idx)
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    est, logG, ess, ens = np.empty((T, M, ne)), np.empty((T, M)), np.empty((T, M)), np.empty((T, ne))
    lib().orc_apf_run(md.ref, ctypes.c_int32(M), _p(N, ctypes.c_int32), ctypes.c_int32(T), _p(obs, ctypes.c_double),
                      ctypes.c_int32(1 if obs_per_filter else 0), ctypes.c_uint64(seed), ctypes.c_int32(ne),
                      _p(est_idx, ctypes.c_int32), _p(est, ctypes.c_double), _p(logG, ctypes.c_double),
                      _p(ess, ctypes.c_double), _p(ens, ctypes.c_double), ctypes.c_int32(threads))
    return dict(est=est, log_G=logG, ess=ess, ens=ens)


def sir_run(spec, M: int, N, T: int, obs: np.ndarray, seed: int, ess_threshold: float,
            est_idx: Optional[Sequence[int]] = None, obs_per_filter: bool = False, threads: int = 0) -> dict:
    """M bootstrap filters that resample only when ESS < ess_threshold N (carried weights between
    resamplings; weighted estimates), and their average (Def. 1)."""
    md = _Model(spec)
    N = np.ascontiguousarray(np.broadcast_to(np.asarray(N, dtype=np.int32), (M,)), dtype=np.int32)
    est_idx = np.ascontiguousarray(range(spec.dx) if est_idx is None else est_idx, dtype=np.int32)
    ne = len(est_idx)
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    est, logG, ess, res, ens = (np.empty((T, M, ne)), np.empty((T, M)), np.empty((T, M)), np.empty((T, M)),
                                np.empty((T, ne)))
    lib().orc_sir_run(md.ref, ctypes.c_int32(M), _p(N, ctypes.c_int32), ctypes.c_int32(T), _p(obs, ctypes.c_double),
                      ctypes.c_int32(1 if obs_per_filter else 0), ctypes.c_uint64(seed), ctypes.c_double(ess_threshold),
                      ctypes.c_int32(ne), _p(est_idx, ctypes.c_int32), _p(est, ctypes.c_double),
                      _p(logG, ctypes.c_double), _p(ess, ctypes.c_double), _p(res, ctypes.c_double),
                      _p(ens, ctypes.c_double), ctypes.c_int32(threads))
    return dict(est=est, log_G=logG, ess=ess, resampled=res, ens=ens)


def bf_run_proposal(spec, theta, M: int, N, T: int, obs: np.ndarray, seed: int, est_idx=None, bf16: bool = True,
                    ess_frac: float = 0.1, obs_per_filter: bool = False, threads: int = 0, span: int = 1) -> dict:
    """M filters with the learned proposal (lattice) acting on the last `span` sub-steps of each
    interval (the fallback to the transition only for span 1); theta None = bootstrap."""
    md = _Model(spec)
    N = np.ascontiguousarray(np.broadcast_to(np.asarray(N, dtype=np.int32), (M,)), dtype=np.int32)
    est_idx = np.ascontiguousarray(range(spec.dx) if est_idx is None else est_idx, dtype=np.int32)
    ne = len(est_idx)
    obs = np.ascontiguousarray(obs, dtype=np.float64)
    post, logG, ess = np.empty((T, M, ne)), np.empty((T, M)), np.empty((T, M))
    ens, fb = np.empty((T, ne)), np.empty((T, M))
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
    pr = None if th is None else _OrcProposal(_p(th, ctypes.c_float), 1 if bf16 else 0, ess_frac, int(span))
    nullp = ctypes.POINTER(ctypes.c_double)()
    lib().orc_bf_run_proposal(md.ref, ctypes.byref(pr) if pr is not None else None, ctypes.c_int32(M),
                              _p(N, ctypes.c_int32), ctypes.c_int32(T), _p(obs, ctypes.c_double),
                              ctypes.c_int32(1 if obs_per_filter else 0), ctypes.c_uint64(seed), ctypes.c_int32(0),
                              ctypes.c_int32(ne), _p(est_idx, ctypes.c_int32), _p(post, ctypes.c_double), nullp,
                              _p(logG, ctypes.c_double), _p(ess, ctypes.c_double), _p(ens, ctypes.c_double), nullp,
                              _p(fb, ctypes.c_double), ctypes.c_int32(threads))
    return dict(est=post, log_G=logG, ess=ess, ens=ens, fallback=fb)


# --------------------------------------------------------------------------
# Kalman filter: the exact filter of the linear-Gaussian case (Sec. 2.2)
# --------------------------------------------------------------------------
def lg_transition(spec):
    """Observation-time transition of K Euler-Maruyama steps of dx = -A x dt + sigma dW:
    x_{t} = F^K x_{t-1} + e, e ~ N(0, Q_K), F = I - dt A, Q_K = sigma^2 dt sum_{j<K} F^j F^j^T."""
    d = spec.dx
    A = np.asarray(spec.params, dtype=np.float64).reshape(d, d)
    F = np.eye(d) - spec.dt * A
    FK = np.eye(d)
    Q = np.zeros((d, d))
    for _ in range(spec.K):
        Q += FK @ FK.T
        FK = F @ FK
    return FK, spec.sigma_dyn ** 2 * spec.dt * Q


def kalman(spec, y: np.ndarray):
    """Posterior means m_t, covariances P_t (t = 1..T) and log p(y_{1:t}) for the LG model."""
    d = spec.dx
    FK, Q = lg_transition(spec)
    H = np.zeros((spec.dy, d))
    for j, i in enumerate(spec.obs_idx):
        H[j, i] = 1.0
    R = spec.sigma_obs ** 2 * np.eye(spec.dy)
    m = np.asarray(spec.x0_mean, dtype=np.float64)
    P = spec.sigma0 ** 2 * np.eye(d)
    T = len(y)
    means = np.empty((T, d))
    covs = np.empty((T, d, d))
    ll = np.empty(T)
    acc = 0.0
    for t in range(T):
        m = FK @ m
        P = FK @ P @ FK.T + Q
        S = H @ P @ H.T + R
        e = y[t] - H @ m
        Si = np.linalg.inv(S)
        acc += -0.5 * (e @ Si @ e) - 0.5 * np.linalg.slogdet(2.0 * np.pi * S)[1]
        G = P @ H.T @ Si
        m = m + G @ e
        P = (np.eye(d) - G @ H) @ P
        means[t], covs[t], ll[t] = m, P, acc
    return means, covs, ll
