"""Accuracy studies on the GPU: the MSE of the ensemble estimator against a
reference posterior, and the wall time needed to reach a given MSE.

* Lorenz 63 at a fixed budget M N = 2^20 (Corollary 2 and the remark after it:
  the MSE of the averaged estimator keeps the 1/(MN) rate while N >= M; for
  N < M the 1/N^2 bias term takes over).  R independent ensembles per M run
  side by side in one context (R M filters; ensemble r = filters
  [r M, (r + 1) M)), so one launch per step serves all of them.
* The lattice: MSE of the averaged v-estimates against a reference posterior,
  plain bootstrap vs learned proposal vs auxiliary filters vs the centralised
  filter at several sizes, and the time-error index of Sec. 3.4 (wall time x MSE), so they can
  be compared at equal MSE.

The Lorenz reference posterior is a bootstrap filter with many more particles
(M = 1), averaged over a few seeds; the lattice reference is a large ensemble
(see lattice_time_to_mse).  Everything runs through the C ABI; this
module only orders the calls and does FP64 bookkeeping on the host.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import pf
from . import workloads as W


def _var_index(spec: W.ModelSpec):
    """The statistics a study scores: x2 for Lorenz 63, every v-node for the lattice."""
    if spec.kind == W.LORENZ63:
        return np.array([1])
    return np.arange(spec.J * spec.J)


def filter_estimates(spec: W.ModelSpec, M: int, N, seed: int, d_y, theta=None, ess_frac: float = 0.1,
                     want_ess: bool = False, aux: bool = False, tau: float = -1.0, span: int = 1):
    """Per-filter posterior means of the scored statistics at every observation
    time: array (T, M, n_stat); optionally the per-filter ESS (T, M)."""
    idx = _var_index(spec)
    T = d_y.shape[0]
    out = np.empty((T, M, len(idx)))
    ess = np.empty((T, M)) if want_ess else None
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        if theta is not None:
            f.set_proposal(theta, ess_frac)
            f.set_proposal_span(span)
        if aux:
            f.set_auxiliary(True)
        f.set_resampling(tau)
        for t in range(T):
            f.step_device(d_y[t])
            if len(idx) == 1:
                out[t, :, 0] = f.estimate(pf.PF_STAT_MEAN, var=int(idx[0]), per_filter=True)
            else:
                out[t] = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)[:, idx]
            if want_ess:
                ess[t] = f.estimate(pf.PF_STAT_ESS, per_filter=True)
    return out, ess


def reference_posterior(spec: W.ModelSpec, N_ref: int, seeds, d_y):
    """Posterior means from a bootstrap filter with N_ref particles (M = 1),
    averaged over the seeds: array (T, n_stat)."""
    acc = None
    for s in seeds:
        e, _ = filter_estimates(spec, 1, N_ref, s, d_y)
        acc = e[:, 0, :] if acc is None else acc + e[:, 0, :]
    return acc / len(seeds)


def step_time(spec: W.ModelSpec, M: int, N, d_y, theta=None, steps: int = 20, warmup: int = 3,
              aux: bool = False, tau: float = -1.0, span: int = 1) -> float:
    """Device seconds per observation step of one M-filter context (CUDA events)."""
    import torch
    st = torch.cuda.Stream()
    with pf.EnsembleFilter(spec, M, N, 99) as f:
        f.set_stream(st.cuda_stream)
        if theta is not None:
            f.set_proposal(theta, 0.1)
            f.set_proposal_span(span)
        if aux:
            f.set_auxiliary(True)
        f.set_resampling(tau)
        for t in range(warmup):
            f.step_device(d_y[t % d_y.shape[0]])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for t in range(steps):
            f.step_device(d_y[(warmup + t) % d_y.shape[0]])
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / steps


def ensemble_mse(per_filter: np.ndarray, M: int, ref: np.ndarray, skip: int = 0):
    """MSE of the M-averages (Def. 1) of R = n_filters / M ensembles against ref,
    averaged over times >= skip and statistics; also its variance and squared
    bias parts (bias^2 = |mean_r Phi - ref|^2 - var / R)."""
    T, F, S = per_filter.shape
    R = F // M
    phi = per_filter[:, :R * M, :].reshape(T, R, M, S).mean(axis=2)  # (T, R, S), FP64
    err = phi[skip:] - ref[skip:, None, :]
    mse = float(np.mean(err ** 2))
    var = float(np.mean(phi[skip:].var(axis=1, ddof=1)))
    bias2 = float(np.mean((phi[skip:].mean(axis=1) - ref[skip:]) ** 2)) - var / R
    return mse, var, bias2, R


def lorenz_sweep_mse(R: int = 64, T: int = 200, N_ref: int = 1 << 24, ref_seeds=(901, 902, 903, 904, 905, 906,
                                                                                    907, 908), log=None):
    """MSE of the averaged x2 estimator over R seeds for each M of the 2^20 sweep."""
    import torch
    spec = W.lorenz63()
    _, y = pf.pf_simulate(spec, T, W.SEED_LORENZ_OBS)
    d_y = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    t0 = time.perf_counter()
    ref = reference_posterior(spec, N_ref, ref_seeds, d_y)
    if log:
        log(f"reference posterior ({len(ref_seeds)} x {N_ref} particles): {time.perf_counter() - t0:.1f} s")
    rows = []
    for tau in (-1.0, 0.5):  # resampling at every step (Algorithm 1), and only when ESS < N / 2
        for M, N in W.lorenz_sweep():
            est, _ = filter_estimates(spec, R * M, N, 1000 + M, d_y, tau=tau)
            mse, var, bias2, _ = ensemble_mse(est, M, ref, skip=1)
            dt = step_time(spec, M, N, d_y, tau=tau)
            rows.append({"M": M, "N": N, "ess_threshold": tau, "mse": mse, "var": var, "bias2": bias2,
                         "s_per_step": dt, "s_per_run": dt * T, "time_error_index": dt * T * mse})
            if log:
                log(f"tau={tau:+.1f} M={M:5d} N={N:8d}  MSE {mse:.3e} (var {var:.3e}, bias^2 {bias2:+.2e})  "
                    f"{dt * 1e3:.3f} ms/step")
    return {"workload": "lorenz63 M*N = 2^20 sweep", "R": R, "T": T, "N_ref": N_ref,
            "ref_seeds": len(ref_seeds), "rows": rows}


def ensemble_reference(spec: W.ModelSpec, M: int, N: int, seeds, d_y):
    """Reference posterior means from large ensembles (Def. 1): the library's
    FP64 M-average, averaged over the seeds: array (T, n_stat)."""
    idx = _var_index(spec)
    T = d_y.shape[0]
    acc = np.zeros((T, len(idx)))
    for s in seeds:
        with pf.EnsembleFilter(spec, M, N, s) as f:
            for t in range(T):
                f.step_device(d_y[t])
                acc[t] += f.estimate(pf.PF_STAT_MEAN, var=-1)[idx]
    return acc / len(seeds)


ALL_METHODS = ("plain", "learned", "auxiliary", "adaptive", "centralised")


def lattice_time_to_mse(theta, Ns=(128, 256, 512, 1024), M: int = 32, R: int = 8, T: int = 40, M_ref: int = 1024,
                        N_ref: int = 1024, ref_seeds=(951, 952), skip: int = 5, log=None, methods=ALL_METHODS,
                        theta_interval=None):
    """Plain bootstrap vs learned proposal on the 40 x 40 lattice: MSE of the
    averaged v-estimates (every node) against a reference posterior, wall time
    per run, and the wall time the learned form needs to reach the plain
    filter's MSE at the largest N (log-log interpolation).  Also the
    centralised filter (M = 1) with the same total particles M N (Sec. 3.4).

    The reference is a large ensemble, not one large filter: on this
    3200-variable lattice a single bootstrap filter's estimate of the
    unobserved nodes keeps a variance that falls far more slowly than 1/N
    (resampling duplicates whole lattices and the small dynamic noise
    re-diversifies them slowly), while independent filters average it away."""
    import torch
    spec = W.fhn_lattice()
    _, y = pf.pf_simulate(spec, T, W.SEED_FHN_OBS)
    d_y = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    ref = ensemble_reference(spec, M_ref, N_ref, ref_seeds, d_y)
    out = {}
    runs = [("plain", None, M, False, -1.0, 1), ("learned", theta, M, False, -1.0, 1),
            ("auxiliary", None, M, True, -1.0, 1), ("adaptive", None, M, False, 0.5, 1),
            ("centralised", None, 1, False, -1.0, 1)]
    if theta_interval is not None:  # the proposal over the whole interval (every sub-step)
        runs.insert(2, ("learned_interval", theta_interval, M, False, -1.0, spec.K))
    for name, th, m_run, aux, tau, span in runs:
        if name not in methods and not (name == "learned_interval" and theta_interval is not None):
            continue
        rows = []
        for N in Ns:
            n_run = N * M // m_run
            est, ess = filter_estimates(spec, R * m_run, n_run, 2000 + N + 7 * m_run, d_y, theta=th, want_ess=True,
                                        aux=aux, tau=tau, span=span)
            mse, var, bias2, _ = ensemble_mse(est, m_run, ref, skip=skip)
            dt = step_time(spec, m_run, n_run, d_y, theta=th, aux=aux, tau=tau, span=span)
            rows.append({"M": m_run, "N": n_run, "mse": mse, "var": var, "bias2": bias2, "s_per_step": dt,
                         "s_per_run": dt * T, "mean_ess_frac": float(np.mean(ess[skip:]) / n_run),
                         "time_error_index": dt * T * mse})
            if log:
                log(f"{name:11s} M={m_run:3d} N={n_run:6d}  MSE {mse:.3e} (var {var:.2e}, bias^2 {bias2:+.1e})  "
                    f"ESS/N {rows[-1]['mean_ess_frac']:.3f}  {dt * 1e3:.2f} ms/step")
        out[name] = rows
    target = out["plain"][-1]["mse"]

    def time_at(rows, mse):
        # wall time per run where the MSE curve crosses `mse` (log-log; None if outside the runs)
        for a, b in zip(rows, rows[1:]):
            if (a["mse"] - mse) * (b["mse"] - mse) <= 0 and a["mse"] != b["mse"]:
                u = (math.log(mse) - math.log(a["mse"])) / (math.log(b["mse"]) - math.log(a["mse"]))
                return math.exp(math.log(a["s_per_run"]) + u * (math.log(b["s_per_run"]) - math.log(a["s_per_run"])))
        return None

    return {"workload": "fhn 40x40, M=32", "R": R, "T": T, "M_ref": M_ref, "N_ref": N_ref,
            "ref_seeds": len(ref_seeds), "skip": skip, "rows": out, "target_mse": target,
            "plain_s_at_target": out["plain"][-1]["s_per_run"],
            **{f"{k}_s_at_target": time_at(out[k], target) for k in out if k != "plain"}}


def paper_lattice_mse(Ns=(100, 500, 1000, 2000, 5000), M: int = 10, records=(0, 1, 2, 3), T: int = 200,
                      skip: int = 20, log=None):
    """The paper's Sec. 5.3 experiment on its own lattice (32 x 32, random
    re-entry stimuli), synthetic records: empirical MSE per node of the
    posterior-mean U against the true U, for an ensemble of M auxiliary
    filters with N particles each and for the centralised auxiliary filter
    with K = M N particles, averaged over the records; device time per step."""
    import torch
    spec = W.fhn_paper()
    nn = spec.J * spec.J
    rows = {"ensemble": [], "centralised": []}
    for N in Ns:
        for name, m_run, n_run in (("ensemble", M, N), ("centralised", 1, M * N)):
            errs = []
            for r in records:
                x, y = pf.pf_simulate(spec, T, W.SEED_FHN_OBS, record=r)
                d_y = torch.from_numpy(np.ascontiguousarray(y)).cuda()
                with pf.EnsembleFilter(spec, m_run, n_run, 4000 + 17 * r + N) as f:
                    f.set_auxiliary(True)
                    for t in range(T):
                        f.step_device(d_y[t])
                        if t >= skip:
                            u = f.estimate(pf.PF_STAT_MEAN, var=-1)[:nn]
                            errs.append(np.mean((u - x[t + 1, :nn]) ** 2))
            dt = step_time(spec, m_run, n_run, d_y, aux=True)
            rows[name].append({"M": m_run, "N": n_run, "mse_per_node": float(np.mean(errs)), "s_per_step": dt})
            if log:
                log(f"paper lattice {name:11s} M={m_run:3d} N={n_run:6d}  MSE/node {np.mean(errs):.4f}  "
                    f"{dt * 1e3:.3f} ms/step")
    return {"workload": "paper's 32x32 lattice, auxiliary filters", "M": M, "records": len(records), "T": T,
            "skip": skip, "rows": rows}


def _ragged_records(spec: W.ModelSpec, n_filters: int, T: int):
    """One synthetic record per filter of the ragged batch: truth (T+1, M, dx) and y (T, M, dy)."""
    xs, ys = [], []
    for m in range(n_filters):
        x, y = pf.pf_simulate(spec, T, W.SEED_RAGGED, record=m)
        xs.append(x)
        ys.append(y)
    return np.stack(xs, axis=1), np.stack(ys, axis=1)


def _time_at(rows, mse, key="s_per_run"):
    """Wall time where the MSE curve of `rows` (ordered by size) crosses `mse`, by
    log-log interpolation between the two runs that bracket it (None if none do)."""
    for a, b in zip(rows, rows[1:]):
        if (a["mse"] - mse) * (b["mse"] - mse) <= 0 and a["mse"] != b["mse"]:
            u = (math.log(mse) - math.log(a["mse"])) / (math.log(b["mse"]) - math.log(a["mse"]))
            return math.exp(math.log(a[key]) + u * (math.log(b[key]) - math.log(a[key])))
    return None


def ragged_time_error(theta, T: int = 20, R: int = 2, M_ref: int = 8, N_ref: int = 2048, skip: int = 4,
                      scales=(0.5, 1.0, 2.0), log=None):
    """The ragged batch (256 lattices of 20 x 20, N log-uniform in [64, 4096], a
    record per filter) with the learned proposal in one context -- the batched
    form -- against the same filters with the bootstrap proposal as 256
    separate contexts, and the two mixed forms: the MSE of each filter's
    v-estimates against its own record's reference posterior (an ensemble of
    M_ref x N_ref bootstrap filters per record, Def. 1), the wall time per run,
    the time-error index of Sec. 3.4 (wall time x MSE), and the wall time the
    batched learned form needs to reach the separate bootstrap filters' MSE
    (its particle counts scaled by `scales`, log-log interpolation)."""
    import torch
    spec = W.fhn_lattice(J=W.RAGGED["J"])
    counts = W.ragged_counts(W.RAGGED["n_filters"], W.RAGGED["n_lo"], W.RAGGED["n_hi"])
    nf = len(counts)
    idx = _var_index(spec)
    _, y = _ragged_records(spec, nf, T)
    d_y = torch.from_numpy(np.ascontiguousarray(y)).cuda()  # (T, nf, dy)
    # reference: M_ref filters per record, filter r nf + m observing record m
    d_y_ref = torch.from_numpy(np.ascontiguousarray(np.tile(y, (1, M_ref, 1)))).cuda()
    ref = np.zeros((T, nf, len(idx)))
    with pf.EnsembleFilter(spec, M_ref * nf, N_ref, 777) as f:
        for t in range(T):
            f.step_device(d_y_ref[t], per_filter=True)
            e = f.estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)[:, idx]
            ref[t] = e.reshape(M_ref, nf, len(idx)).mean(axis=0)
    if log:
        log(f"ragged reference: {M_ref} x {N_ref} particles per record")

    def contexts(batched, learned, scale, seed, st=None):
        n = np.maximum(1, np.round(counts * scale)).astype(np.int32)
        ctxs = [pf.EnsembleFilter(spec, nf, n, seed)] if batched else \
            [pf.EnsembleFilter(spec, 1, int(k), seed + m) for m, k in enumerate(n)]
        for f in ctxs:
            if st is not None:
                f.set_stream(st.cuda_stream)
            if learned:
                f.set_proposal(theta, 0.1)
        return ctxs, int(n.sum())

    def step_all(batched, ctxs, t):
        if batched:
            ctxs[0].step_device(d_y[t % T], per_filter=True)
        else:
            for m, f in enumerate(ctxs):
                f.step_device(d_y[t % T, m])

    def estimates(batched, learned, scale, seed):
        out = np.empty((T, nf, len(idx)))
        ctxs, _ = contexts(batched, learned, scale, seed)
        try:
            for t in range(T):
                step_all(batched, ctxs, t)
                if batched:
                    out[t] = ctxs[0].estimate(pf.PF_STAT_MEAN, var=-1, per_filter=True)[:, idx]
                else:
                    for m, f in enumerate(ctxs):
                        out[t, m] = f.estimate(pf.PF_STAT_MEAN, var=-1)[idx]
        finally:
            for f in ctxs:
                f.close()
        return out

    def seconds_per_step(batched, learned, scale, steps=10):
        st = torch.cuda.Stream()
        ctxs, _ = contexts(batched, learned, scale, 99, st)
        try:
            for t in range(3):
                step_all(batched, ctxs, t)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for t in range(steps):
                step_all(batched, ctxs, 3 + t)
            b.record(st)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / 1e3 / steps
        finally:
            for f in ctxs:
                f.close()

    forms = [(True, True, sc) for sc in scales] + [(False, False, 1.0), (True, False, 1.0), (False, True, 1.0)]
    rows = []
    for batched, learned, scale in forms:
        mse = float(np.mean([np.mean((estimates(batched, learned, scale, 5000 + 311 * r)[skip:] - ref[skip:]) ** 2)
                             for r in range(R)]))
        dt = seconds_per_step(batched, learned, scale)
        row = {"form": "batched" if batched else "separate", "proposal": "learned" if learned else "bootstrap",
               "scale": scale, "N_total": int(np.maximum(1, np.round(counts * scale)).sum()), "mse": mse,
               "s_per_step": dt, "s_per_run": dt * T, "time_error_index": dt * T * mse}
        rows.append(row)
        if log:
            log(f"ragged {row['form']:8s} {row['proposal']:9s} x{scale:<4g} MSE {mse:.3e}  {dt * 1e3:.2f} ms/step")
    plain_sep = next(r for r in rows if r["form"] == "separate" and r["proposal"] == "bootstrap")
    learned_b = sorted([r for r in rows if r["form"] == "batched" and r["proposal"] == "learned"],
                       key=lambda r: r["scale"])
    t_learned = _time_at(learned_b, plain_sep["mse"])
    return {"workload": "256 fhn 20x20 lattices, N log-uniform in [64, 4096], a record per filter",
            "T": T, "R": R, "skip": skip, "M_ref": M_ref, "N_ref": N_ref, "N_total": int(counts.sum()), "rows": rows,
            "target_mse": plain_sep["mse"], "plain_separate_s": plain_sep["s_per_run"],
            "learned_batched_s_at_target": t_learned,
            "learned_batched_vs_plain_separate": (t_learned / plain_sep["s_per_run"]) if t_learned else None}
