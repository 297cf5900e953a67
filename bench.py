"""Throughput benchmark of the GPU ensemble particle filter.

Workload (default): the Lorenz 63 ensemble with a total budget of M * N = 2^20
particles swept over M in {1, 4, 16, 64, 256, 1024, 4096}, N = 2^20 / M; the
seven configurations (5461 filters, 7 x 2^20 particles) run as one ragged batch
in one context, so every launch covers all of them and each step is one CUDA
graph.  One bench step is one observation time: K = 40 Euler-Maruyama
sub-steps of every particle, Gaussian weights, FP64 normalisation, systematic
resampling with the gather, and the per-filter and ensemble means.  The metric
is particle-steps/s (one Euler-Maruyama sub-step of one particle).
`--workload lorenz-sweep-7ctx` runs the seven configurations as seven contexts
on seven streams instead.

`--workload fhn` runs the 40 x 40 FitzHugh-Nagumo lattice at M = 32, N = 1024;
`--workload fhn-learned` the same with the learned proposal (network trained,
untimed, on tuples the plain filter records); `--workload ragged` 256 lattice
filters of 20 x 20 nodes with N log-uniform in [64, 4096], independent records
and the learned proposal, in one autotuned context -- and, beside it, the same
batch as 256 separate contexts.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the plain restatement of the method this project checks against) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1407_8071_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128

# Algorithmic ALU operations per Lorenz particle-step (one Euler-Maruyama
# sub-step of one particle), counting the minimal work of each published step:
#   Philox4x32-10: 10 rounds x (2 wide multiplies + 2 three-input XORs) = 40,
#                  0.75 calls per sub-step (3 blocks per 4 sub-steps)       -> 30
#   Box-Muller pair: 4 (uniforms) + 8 (log) + 2 (sqrt) + 12 (sincospi)
#                  + 3 (scalings) = 29, 1.5 pairs per sub-step               -> 43.5
#   drift 7 + Euler-Maruyama update 6                                      -> 13
LORENZ_OPS_PER_PARTICLE_STEP = 86.5
# Algorithmic HBM bytes of a resampling step per particle: its log-weight read
# and its ancestor index written, plus, per state variable, the gather (one
# read, one write; the per-filter means are taken from the gathered values) --
# or, where the gather is folded into the next propagation, the read alone.
# The prefix and the markers of the tile chain are implementation traffic.
RESAMPLE_BYTES_PER_PARTICLE = 4 + 4
RESAMPLE_BYTES_PER_VARIABLE = 4 + 4
RESAMPLE_BYTES_PER_VARIABLE_FOLDED = 4

# Algorithmic ALU operations per lattice node-step (one Euler-Maruyama
# sub-step of one node, both planes): Philox4x32-10 40 per 4 normals -> 20,
# one Box-Muller pair 29, Laplacian 4 (three adds, one fused -4v), drift of
# v 9 (cubic, coupling, D times the Laplacian), of w 2, two Euler-Maruyama
# updates 4 -> 68.
FHN_OPS_PER_NODE_STEP = 68
# The auxiliary filter's noise-free look-ahead: Laplacian 4, drift 9 + 2,
# two Euler updates 2 -> 17 per node-step.
FHN_LOOKAHEAD_OPS_PER_NODE_STEP = 17
# The paper's lattice per node-step: Philox 40 / 2 nodes (the U normal takes
# half a Box-Muller pair's block) -> 20, Box-Muller pair / 2 -> 14.5,
# neighbour sum 3 + coupling 1, cubic 3, drift of U 4 and V 2, stimulus
# counter 2, two updates 2 -> 51.5 (look-ahead without the generator: 17).
FHNP_OPS_PER_NODE_STEP = 51.5
# With one Euler step per observation the auxiliary step on the paper's lattice
# moves each particle's state four times (see the roofline below).
FHNP_STATE_PASSES = 4


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r for r in csv.reader(io.StringIO(out)) if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def source_digest(unit: str = "k_filter.cu", root: str = None):
    """Digest of the CUDA translation unit `unit` and every local header it
    includes (directly or through another header), with comments and blank
    lines removed, so that a recorded measurement stays attached to the code
    it was taken on."""
    import re
    root = root or ROOT
    dirs = [os.path.join(root, "paper_1407_8071_gb300", "csrc"), os.path.join(root, "include")]
    found, todo = {}, [unit]
    while todo:
        name = todo.pop()
        if name in found:
            continue
        path = next((os.path.join(d, name) for d in dirs if os.path.exists(os.path.join(d, name))), None)
        if path is None:
            continue
        with open(path, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        found[name] = "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip()) + "\n"
        todo.extend(re.findall(r'#include\s+"([^"]+)"', text))
    h = hashlib.sha256()
    for name in sorted(found):
        h.update(name.encode() + b"\n" + found[name].encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` (a kernel of k_filter.cu) from the
    committed ncu summary, if its sources have not changed since it was taken
    (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = source_digest()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
            return float(parts[2])
    return None


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
WORKLOAD_TEXT = {
    "lorenz-sweep": ("lorenz63 ensemble, the seven M*N = 2^20 configurations of the sweep (M in {1,4,16,64,256,"
                     "1024,4096}) as one ragged batch of 5461 filters in one context: every kernel launch covers "
                     "all of them, one CUDA graph per step (one observation, K=40 Euler-Maruyama sub-steps)"),
    "lorenz-sweep-7ctx": ("lorenz63 ensemble, M*N = 2^20 swept over M in {1,4,16,64,256,1024,4096}, the seven "
                          "configurations as seven contexts on seven streams; one step = one observation of each"),
    "fhn": "fhn 40x40 lattice (3200 variables), M=32 x N=1024, K=20, bootstrap proposal",
    "fhn-learned": "fhn 40x40 lattice, M=32 x N=1024, K=20, learned proposal (network trained untimed)",
    "fhn-apf": "fhn 40x40 lattice, M=32 x N=1024, K=20, auxiliary particle filters (the paper's Sec. 5.3 filter)",
    "fhn-paper": ("the paper's own 32x32 FitzHugh-Nagumo lattice with random re-entry stimuli (3072 variables), "
                  "M=10 x N=5000 auxiliary particle filters, one Euler step per observation (the paper's Sec. 5.3 "
                  "set-up)"),
    "ragged": ("256 fhn 20x20 lattices, N log-uniform in [64, 4096], independent records, learned proposal, "
               "one autotuned context (all filters in each launch, CUDA graph)"),
}


class Workload:
    def __init__(self, name, seed_base):
        import torch
        from paper_1407_8071_gb300 import pf, proposal
        self.name = name
        self.filters, self.streams = [], []
        self.pending, self.last_estimate = [], None
        self.per_filter_obs = False
        self.choice = None
        self.N_list = None
        if name == "lorenz-sweep-7ctx":
            self.spec = W.lorenz63()
            self.rows = W.lorenz_sweep()
            rec_seed, T = W.SEED_LORENZ_OBS, 200
        elif name == "lorenz-sweep":
            self.spec = W.lorenz63()
            self.N_list = np.concatenate([np.full(M, N, dtype=np.int32) for M, N in W.lorenz_sweep()])
            self.rows = [(len(self.N_list), self.N_list)]
            rec_seed, T = W.SEED_LORENZ_OBS, 200
        elif name in ("fhn", "fhn-learned", "fhn-apf"):
            self.spec = W.fhn_lattice()
            self.rows = [(W.FHN_FULL["M"], W.FHN_FULL["N"])]
            rec_seed, T = W.SEED_FHN_OBS, W.FHN_FULL["T"]
        elif name == "fhn-paper":
            self.spec = W.fhn_paper()
            self.rows = [(10, 5000)]
            rec_seed, T = W.SEED_FHN_OBS, 400
        elif name == "ragged":
            self.spec = W.fhn_lattice(J=W.RAGGED["J"])
            self.N_list = W.ragged_counts(W.RAGGED["n_filters"], W.RAGGED["n_lo"], W.RAGGED["n_hi"])
            self.rows = [(len(self.N_list), self.N_list)]
            rec_seed, T = W.SEED_RAGGED, 50
            self.per_filter_obs = True
        else:
            raise ValueError(name)
        self.T = T
        if self.per_filter_obs:  # an independent record per filter: T x M x dy
            y = np.stack([pf.pf_simulate(self.spec, T, rec_seed, record=m)[1] for m in range(len(self.N_list))],
                         axis=1)
            train_record = pf.pf_simulate(self.spec, 20, rec_seed, record=1 << 20)[1]
        else:
            y = pf.pf_simulate(self.spec, T, rec_seed)[1]
            train_record = y
        self.y_host = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
        self.y_dev = self.y_host.cuda()
        torch.cuda.synchronize()
        self.theta = None
        self.aux = name in ("fhn-apf", "fhn-paper")
        if name in ("fhn-learned", "ragged"):
            self.theta = proposal.trained_theta(self.spec, train_record[:20], seed=seed_base + 77)
        # one stream per context: the configurations are independent, so their
        # kernels may overlap; `stream` is where the timed region starts and ends
        self.stream = torch.cuda.Stream()
        for i, (M, N) in enumerate(self.rows):
            f = pf.EnsembleFilter(self.spec, M, N, seed=seed_base + i)
            st = torch.cuda.Stream()
            f.set_stream(st.cuda_stream)
            if self.theta is not None:
                f.set_proposal(self.theta, 0.1)
            self.choice = f.autotune()
            if self.aux:
                f.set_auxiliary(True)
            self.filters.append(f)
            self.streams.append(st)
        self.particles = int(sum(int(np.sum(N)) if np.ndim(N) else M * N for M, N in self.rows))
        self.particle_steps_per_step = self.particles * self.spec.K
        self.t = 0

    def row(self, src):
        return src[self.t % self.T]

    def step_device(self):
        r = self.row(self.y_dev)
        for f in self.filters:
            f.step_device(r, per_filter=self.per_filter_obs)
        self.t += 1

    def launches_per_step(self):
        """Kernels one step of every context launches, counted from the contexts' captured step graphs."""
        return sum(f.step_kernels() for f in self.filters)

    def step_host(self):
        """Through the public API with host buffers: H2D of y_t, D2H of each ensemble estimate
        (pipelined: the copy of step t's estimate is enqueued behind step t and read once
        step t+1 has been enqueued; the timed region ends after the last copy)."""
        from paper_1407_8071_gb300 import pf
        y = self.row(self.y_host).numpy()
        for f in self.filters:
            f.step(y, per_filter=self.per_filter_obs)
        # step t-1's estimates are read while step t runs
        for p in self.pending:
            self.last_estimate = p.wait()
        var = 1 if self.spec.kind == W.LORENZ63 else 0
        self.pending = [f.estimate_async(pf.PF_STAT_MEAN, var=var) for f in self.filters]
        self.t += 1

    def obs_bytes(self):
        """Observation bytes one step copies host to device."""
        per = int(np.prod(self.y_host.shape[1:])) * 4
        return per * len(self.filters)

    def close(self):
        for f in self.filters:
            f.close()


def separate_contexts(torch, wl, steps):
    """The ragged batch as one context per filter, stepped one after another on
    one stream (the alternative to batching all filters in each launch)."""
    from paper_1407_8071_gb300 import pf
    st = torch.cuda.Stream()
    ctxs = []
    for m, n in enumerate(wl.N_list):
        f = pf.EnsembleFilter(wl.spec, 1, int(n), seed=7000 + m)
        f.set_stream(st.cuda_stream)
        if wl.theta is not None:
            f.set_proposal(wl.theta, 0.1)
        ctxs.append(f)

    def step(t):
        for m, f in enumerate(ctxs):
            f.step_device(wl.y_dev[t % wl.T, m])

    for t in range(3):
        step(t)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for t in range(steps):
        step(t)
    b.record(st)
    torch.cuda.synchronize()
    el = a.elapsed_time(b) / 1e3
    launches = steps * sum(f.step_kernels() for f in ctxs)
    for f in ctxs:
        f.close()
    return {"value": wl.particle_steps_per_step * steps / el, "unit": METRIC, "ms_per_step": el / steps * 1e3,
            "contexts": len(ctxs), "gpu_launches": launches}


def time_region(torch, wl, fn, K, barrier=None):
    torch.cuda.synchronize()
    if barrier:
        barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(wl.stream)
    for st in wl.streams:
        st.wait_stream(wl.stream)
    for _ in range(K):
        fn()
    for st in wl.streams:
        wl.stream.wait_stream(st)
    end.record(wl.stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return start.elapsed_time(end) / 1e3


def phase_times(torch, wl, reps=5):
    """Average device time of the propagate+weight half and of the resampling
    half of a step, per launch, as the step runs them (pf_step_timed: CUDA
    events between the halves on the filters' stream; the auxiliary filter
    steps as one unit, so its whole step is the first figure)."""
    prop, res = [], []
    if wl.aux:
        for f, st in zip(wl.filters, wl.streams):
            for _ in range(reps):
                e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                e0.record(st)
                f.step_device(wl.y_dev[wl.t % wl.T])
                e1.record(st)
                torch.cuda.synchronize()
                prop.append(e0.elapsed_time(e1) / 1e3)
                wl.t += 1
        return float(np.mean(prop)), 0.0, prop
    for f in wl.filters:
        for _ in range(reps):
            a, b = f.step_timed(wl.y_dev[wl.t % wl.T], per_filter=wl.per_filter_obs)
            prop.append(a / 1e3)
            res.append(b / 1e3)
            wl.t += 1
    return float(np.mean(prop)), float(np.mean(res)), prop


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def resample_roofline(wl, t_res, peaks, peak_src, folded):
    """HBM roofline of the resampling chain (normaliser, systematic resampling,
    gather, per-filter means), per context step, on algorithmic bytes: with
    the gather folded into the next propagation only the ancestors' values are
    read (for the means), else they are also written as the new state."""
    nf = len(wl.filters)
    per_ctx = wl.particles / nf
    per_var = RESAMPLE_BYTES_PER_VARIABLE_FOLDED if folded else RESAMPLE_BYTES_PER_VARIABLE
    bytes_ = per_ctx * (RESAMPLE_BYTES_PER_PARTICLE + wl.spec.dx * per_var)
    hbm = float(peaks["hbm_gbs"])
    achieved = bytes_ / t_res / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "bytes_per_launch": bytes_, "avg_chain_s": t_res, "peak_source": f"{peak_src} copy bandwidth",
            "note": ("working set below the 129 MB L2 per context" if bytes_ < 129e6 else "larger than L2")}


def oracle_case(workload: str, M: int, n_scale: int, T: int, theta=None):
    """A bounded sample of `workload` for the FP64 oracle: (spec, M, N, y, per-filter obs, theta)."""
    import oracle
    if workload.startswith("lorenz-sweep"):  # filters of the M = 64, N = 16384 row of the sweep
        spec = W.lorenz63()
        return spec, M, (1 << 14) // n_scale, oracle.simulate(spec, T, W.SEED_LORENZ_OBS)[1], False, None
    if workload in ("fhn", "fhn-learned", "fhn-apf"):
        spec = W.fhn_lattice()
        y = oracle.simulate(spec, T, W.SEED_FHN_OBS)[1]
        if workload == "fhn-learned" and theta is None:
            from paper_1407_8071_gb300 import proposal
            theta = proposal.initial_theta(1)
        return spec, M, max(2, 8 // n_scale), y, False, theta
    if workload == "fhn-paper":
        spec = W.fhn_paper()
        return spec, M, max(4, 40 // n_scale), oracle.simulate(spec, T, W.SEED_FHN_OBS)[1], False, None
    spec = W.fhn_lattice(J=W.RAGGED["J"])
    counts = W.ragged_counts(W.RAGGED["n_filters"], W.RAGGED["n_lo"], W.RAGGED["n_hi"])
    N = np.maximum(1, counts[:M] // (16 * n_scale))  # the first M filters' counts, scaled down
    y = np.stack([oracle.simulate(spec, T, W.SEED_RAGGED, record=m)[1] for m in range(M)], axis=1)
    if theta is None:
        from paper_1407_8071_gb300 import proposal
        theta = proposal.initial_theta(1)
    return spec, M, N, y, True, theta


def oracle_run(case, T, seed, threads, aux=False):
    import oracle
    spec, M, N, y, per_filter, theta = case
    if aux:
        oracle.apf_run(spec, M, N, T, y[:T], seed=seed, est_idx=[1], obs_per_filter=per_filter, threads=threads)
    elif spec.kind == W.FHN:
        oracle.bf_run_proposal(spec, theta, M, N, T, y[:T], seed=seed, est_idx=[1], obs_per_filter=per_filter,
                               threads=threads)
    else:
        oracle.bf_run(spec, M, N, T, y[:T], seed=seed, est_idx=[1], threads=threads)
    return int(np.sum(np.broadcast_to(N, (M,)))) * T * spec.K


def oracle_sample(workload: str, target_s: float, theta=None):
    """Times the FP64 oracle on a bounded sample of the workload; returns
    (particle-steps/s, threads, sample description)."""
    cores = os.cpu_count() or 1
    M = min(64 if workload.startswith("lorenz-sweep") else (10 if workload == "fhn-paper" else 32), 2 * cores)
    Tmax = 200 if workload.startswith("lorenz-sweep") else (40 if workload == "fhn-paper" else 6)
    case = oracle_case(workload, M, 1, Tmax, theta)
    threads = min(M, cores)
    t0 = time.perf_counter()
    aux = workload in ("fhn-apf", "fhn-paper")
    oracle_run(case, 1, 1, threads, aux)
    dt1 = time.perf_counter() - t0
    T = int(max(1, min(Tmax, round(target_s / max(dt1, 1e-3)))))
    t0 = time.perf_counter()
    ps = oracle_run(case, T, 2, threads, aux)
    dt = time.perf_counter() - t0
    spec, _, N, _, _, th = case
    ntxt = f"{N} particles" if np.ndim(N) == 0 else f"{int(np.sum(N))} particles in all (ragged)"
    desc = (f"{W.KIND_NAMES[spec.kind]}: {M} filters, {ntxt}, {T} observations x K={spec.K} "
            f"(= {ps:.3g} particle-steps) of the {workload} workload, FP64, OpenMP over filters"
            + (", learned proposal" if th is not None else "") + (", auxiliary filters" if aux else ""))
    return ps / dt, threads, desc


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    M = min(32, 2 * cores)
    case = oracle_case(args.workload, M, 4, 2)
    threads = min(M, cores)
    for k in range(args.warmup):
        oracle_run(case, 1, 3 + k, threads, args.workload in ("fhn-apf", "fhn-paper"))
    t0 = time.perf_counter()
    work = 0
    for k in range(args.steps):
        work += oracle_run(case, 1, 100 + k, threads, args.workload in ("fhn-apf", "fhn-paper"))
    dt = time.perf_counter() - t0
    value = work / dt
    spec, _, N, _, _, th = case
    ntxt = f"{N} particles each" if np.ndim(N) == 0 else f"{int(np.sum(N))} particles in all (ragged)"
    sample = (f"each step: one observation interval (K={spec.K}) of {M} filters, {ntxt}, of the "
              f"{args.workload} workload in the FP64 C oracle (prior draw included)"
              + (", learned proposal" if th is not None else ""))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_study(args):
    """MSE of the averaged estimator against a reference posterior: the Lorenz
    2^20 sweep over 64 seeds, and plain vs learned proposal on the lattice at
    equal MSE (wall time to reach the plain filter's MSE at N = 1024)."""
    import torch
    from paper_1407_8071_gb300 import pf, proposal, study
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    pf.lib()
    log = lambda m: print(m, file=sys.stderr, flush=True)  # noqa: E731
    t0 = time.perf_counter()
    if args.study == "time-error":
        # Sec. 3.4's time-error index (wall time x MSE) of every split of the Lorenz 2^20 budget, and of
        # the ragged batch in one context against 256 separate contexts
        lor = study.lorenz_sweep_mse(log=log)
        spec = W.fhn_lattice(J=W.RAGGED["J"])
        train_record = pf.pf_simulate(spec, 20, W.SEED_RAGGED, record=1 << 20)[1]
        theta = proposal.trained_theta(spec, train_record, seed=77)
        rag = study.ragged_time_error(theta, log=log)
        print(json.dumps({"study": "time-error", "data": "synthetic", "lorenz_sweep": lor, "ragged": rag,
                          "wall_s": time.perf_counter() - t0}))
        return 0
    lor = study.lorenz_sweep_mse(log=log)
    spec = W.fhn_lattice()
    train_record = pf.pf_simulate(spec, 20, W.SEED_FHN_OBS, record=1)[1]  # not the scored record
    theta = proposal.trained_theta(spec, train_record, seed=77)
    lat = study.lattice_time_to_mse(theta, log=log)
    paper = study.paper_lattice_mse(log=log)
    line = {"study": "mse", "data": "synthetic", "lorenz_sweep": lor, "lattice": lat, "paper_lattice": paper,
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line))
    return 0


def measure(name, steps, warmup, rank, world, barrier, cpu_seconds):
    """One workload: W untimed steps, K timed steps (device-resident inputs), the
    same K through host buffers, the dominant kernel timed live, the oracle
    timed on a bounded sample (cpu_seconds > 0, rank 0, N = 1).  Returns the
    workload's JSON object."""
    import torch
    import torch.distributed as dist
    wl = Workload(name, seed_base=1000 * rank + 1)
    for _ in range(warmup):
        wl.step_device()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    elapsed = time_region(torch, wl, wl.step_device, steps, barrier)
    clocks = sampler.stop()
    if world > 1:
        t = torch.tensor([elapsed], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    value = world * wl.particle_steps_per_step * steps / elapsed

    # end to end through the public API with host buffers
    for _ in range(2):
        wl.step_host()
    e2e_elapsed = time_region(torch, wl, wl.step_host, steps, barrier)
    if world > 1:
        t = torch.tensor([e2e_elapsed], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_elapsed = float(t.item())
    e2e_value = world * wl.particle_steps_per_step * steps / e2e_elapsed
    nf = len(wl.filters)

    # the dominant kernel, timed live per launch
    t_prop, t_res, _ = phase_times(torch, wl)
    # bootstrap steps, and learned-proposal steps whose proposal acts on the last sub-step only (the
    # bench's), fold the resampling's gather into the next propagation: the resampling then reads the
    # ancestors' values for the means and writes no copy of the state
    folded = not wl.aux
    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if wl.spec.kind == W.LORENZ63:
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12  # T ops/s
        per_launch_ops = (wl.particles / nf) * wl.spec.K * LORENZ_OPS_PER_PARTICLE_STEP
        achieved = per_launch_ops / t_prop / 1e12
        roofline = {"bound": "alu", "kernel": "k_propagate_small<3>", "achieved": achieved, "peak": alu_peak,
                    "unit": "Tops/s", "frac": achieved / alu_peak,
                    "traffic": recorded_traffic("k_propagate_small<3>"),
                    "peak_source": f"152 SMs x 128 FP32/INT32 lanes x {sm_max:.0f} MHz ({peak_src} max clock)",
                    "ops_per_particle_step": LORENZ_OPS_PER_PARTICLE_STEP, "avg_launch_s": t_prop}
    elif wl.spec.kind == W.FHN_PAPER:
        # one Euler step per observation: the step streams the state four times (look-ahead read,
        # second-stage read of the ancestors' rows + write, weighted means read), so HBM bounds it
        hbm = float(peaks["hbm_gbs"])
        per_launch_bytes = (wl.particles / nf) * wl.spec.dx * 4 * FHNP_STATE_PASSES
        achieved = per_launch_bytes / t_prop / 1e9
        roofline = {"bound": "hbm", "kernel": "auxiliary step (look-ahead, resampling, second stage from the ancestors' rows, means)",
                    "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                    "peak_source": f"{peak_src} copy bandwidth", "bytes_per_particle_step": wl.spec.dx * 4 *
                    FHNP_STATE_PASSES, "avg_launch_s": t_prop}
    else:
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
        base_ops = FHN_OPS_PER_NODE_STEP
        ops_node = base_ops + (FHN_LOOKAHEAD_OPS_PER_NODE_STEP if wl.aux else 0)
        per_launch_ops = (wl.particles / nf) * wl.spec.K * wl.spec.J * wl.spec.J * ops_node
        achieved = per_launch_ops / t_prop / 1e12
        # the four- and eight-node builds (template G = 1, 2; either CTAs-per-SM build)
        lattice_kernel = {4: "k_propagate_fhn4<1,*,1>", 8: "k_propagate_fhn4<1,*,2>"}.get(
            wl.choice[2] if wl.choice else 0, "k_propagate_fhn<float>")
        kern = (lattice_kernel if wl.theta is None else "proposal propagate (5 kernels)") if not wl.aux \
            else "auxiliary step (look-ahead + second-stage propagate + resampling)"
        roofline = {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                    "frac": achieved / alu_peak,
                    "traffic": recorded_traffic(lattice_kernel) if wl.theta is None and not wl.aux else None,
                    "peak_source": f"152 SMs x 128 FP32/INT32 lanes x {sm_max:.0f} MHz ({peak_src} max clock)",
                    "ops_per_node_step": FHN_OPS_PER_NODE_STEP, "avg_launch_s": t_prop}

    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": elapsed / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": WORKLOAD_TEXT[name],
            "rows": ([{"M": M, "N": N} for M, N in wl.rows] if wl.N_list is None else
                     [{"M": len(wl.N_list), "N_min": int(wl.N_list.min()), "N_max": int(wl.N_list.max()),
                       "N_total": int(wl.N_list.sum())}]),
            "K": wl.spec.K, "dt": wl.spec.dt,
            "autotuned": None if wl.choice is None else {"particles_per_cta": wl.choice[0],
                                                         "resample_threads": wl.choice[1],
                                                         "nodes_per_thread": wl.choice[2]},
            "precision": "FP32 state and propagation; FP64 normaliser, prefix sum and M-average",
            "l2": ("working set of the seven configurations (~340 MB: state 2 x 88 MB, prefix 59 MB, ...) exceeds "
                   "the 129 MB L2") if name.startswith("lorenz-sweep")
            else f"state {wl.particles * wl.spec.dx * 4 / 1e6:.0f} MB per buffer, larger than L2",
        },
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "particle-steps/s", "h2d_bytes_per_step": wl.obs_bytes(),
                "d2h_bytes_per_step": nf * 8},
        "gpu_launches": steps * wl.launches_per_step(),
        "roofline": roofline,
        "phases_s": {"propagate_weight": t_prop, "resample_chain": t_res, "gather_folded": folded},
        "resample_roofline": resample_roofline(wl, t_res, peaks, peak_src, folded) if t_res > 0 else None,
    }
    theta = wl.theta
    if wl.name == "ragged":
        line["separate_contexts"] = separate_contexts(torch, wl, max(1, steps // 4))
    wl.close()
    if rank == 0 and world == 1 and cpu_seconds > 0:
        v, cores, desc = oracle_sample(name, cpu_seconds, theta)
        line["cpu_baseline"] = {"value": v, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
                                "sample": desc}
    return line


# The other workloads of the default run: (timed steps, oracle seconds).  Each
# is a separate context, measured the way the headline is.
EXTRA_WORKLOADS = {"fhn": (20, 3.0), "fhn-learned": (20, 3.0), "ragged": (12, 3.0), "fhn-paper": (100, 3.0)}


def extra_workloads(rank, world, barrier, args):
    out = {}
    for name, (steps, cpu_s) in EXTRA_WORKLOADS.items():
        out[name] = measure(name, steps, 3, rank, world, barrier, 0.0 if args.no_cpu_baseline else cpu_s)
    return out


def time_to_mse_block():
    """Short seeded studies of the wall time to reach a fixed MSE.

    config4: the 40 x 40 lattice at M = 32: MSE of the averaged v-estimates against
    a large-ensemble reference for the plain, learned-proposal (on the last
    sub-step, and on every sub-step of the interval) and auxiliary ensembles at
    N = 256, 512, 1024, and the wall time each needs to reach the
    plain ensemble's MSE at N = 1024 (log-log interpolation between the runs that
    bracket it).
    config5: the ragged batch of 256 20 x 20 lattices: the learned proposal in one
    batched context (particle counts scaled by 0.5, 1, 2) against the bootstrap
    filters as 256 separate contexts, and the wall time the batched learned form
    needs to reach the separate bootstrap filters' MSE."""
    from paper_1407_8071_gb300 import pf, proposal, study
    t0 = time.perf_counter()
    spec = W.fhn_lattice()
    train_record = pf.pf_simulate(spec, 20, W.SEED_FHN_OBS, record=1)[1]  # not the scored record
    theta = proposal.trained_theta(spec, train_record, seed=77)
    theta_interval = proposal.trained_theta(spec, train_record, seed=78, span=spec.K)
    r = study.lattice_time_to_mse(theta, Ns=(256, 512, 1024), R=4, T=30, M_ref=512, N_ref=1024, ref_seeds=(951,),
                                  skip=5, methods=("plain", "learned", "auxiliary"), theta_interval=theta_interval)
    plain = r["plain_s_at_target"]
    c4 = {
        "workload": "fhn 40x40 lattice, M=32 ensembles of N in {256, 512, 1024}; R=4 ensembles per point, T=30 "
                    "observations (the first 5 not scored), reference: 512 x 1024 bootstrap ensemble",
        "target_mse": r["target_mse"], "plain_s": plain,
        "learned_s": r["learned_s_at_target"], "auxiliary_s": r["auxiliary_s_at_target"],
        "learned_interval_s": r["learned_interval_s_at_target"],
        "learned_vs_plain": (r["learned_s_at_target"] / plain) if r["learned_s_at_target"] else None,
        "auxiliary_vs_plain": (r["auxiliary_s_at_target"] / plain) if r["auxiliary_s_at_target"] else None,
        "rows": {k: [{kk: row[kk] for kk in ("N", "mse", "s_per_run", "mean_ess_frac")} for row in v]
                 for k, v in r["rows"].items()},
    }
    rspec = W.fhn_lattice(J=W.RAGGED["J"])
    rtheta = proposal.trained_theta(rspec, pf.pf_simulate(rspec, 20, W.SEED_RAGGED, record=1 << 20)[1], seed=77)
    rg = study.ragged_time_error(rtheta, T=12, R=1, M_ref=4, N_ref=2048, skip=3)
    c5 = {"workload": rg["workload"] + "; T=12 (the first 3 not scored), R=1, reference 4 x 2048 per record",
          "target_mse": rg["target_mse"], "plain_separate_s": rg["plain_separate_s"],
          "learned_batched_s": rg["learned_batched_s_at_target"],
          "learned_batched_vs_plain_separate": rg["learned_batched_vs_plain_separate"],
          "rows": [{k: row[k] for k in ("form", "proposal", "scale", "N_total", "mse", "s_per_run")}
                   for row in rg["rows"]]}
    return {"config4": c4, "config5": c5, "wall_s": time.perf_counter() - t0}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="lorenz-sweep", choices=list(WORKLOAD_TEXT))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="the headline workload only (no other workloads, no time-to-MSE study)")
    ap.add_argument("--study", choices=["mse", "time-error"], default=None,
                    help="accuracy study instead of the throughput bench (one JSON line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.study:
        return run_study(args)

    import torch
    import torch.distributed as dist
    from paper_1407_8071_gb300 import pf

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    barrier = None
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = dist.barrier
    pf.lib()

    line = measure(args.workload, args.steps, args.warmup, rank, world, barrier,
                   0.0 if args.no_cpu_baseline else args.cpu_seconds)
    if args.workload == "lorenz-sweep" and world == 1 and not args.no_extras:
        line["workloads"] = extra_workloads(rank, world, barrier, args)
        line["time_to_mse"] = time_to_mse_block()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
