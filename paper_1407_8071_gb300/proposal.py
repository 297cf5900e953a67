"""Training the learned proposal from tuples the filter itself generates.

The plain (bootstrap) lattice filter records, at each observation, for its
resampled particles and each observed node, the network input of the
ancestor before the last sub-step and the standardised residual of the
node's new value, r = (x_t - m) / h (pf_record_tuples).  The network is then
fitted to those tuples by minimising the Gaussian negative log-likelihood on
the GPU (pf_mlp_train_step): it learns where, given the local state and the
observation, the resampled (posterior) particles moved in their last
sub-step.  All arithmetic runs in libpf_gb300.so; this module only orders the
calls.
"""
from __future__ import annotations

import numpy as np

from . import pf
from . import workloads as W


def collect_tuples(spec: W.ModelSpec, M: int, N: int, record: np.ndarray, seed: int, capacity: int,
                   stride: int = 1, steps: int | None = None, span: int = 1):
    """Runs the bootstrap filter over the record and returns (X, R) device tensors
    (capacity x 51 and capacity x 2) holding the first `count` tuples, and count.
    The network inputs are taken before the last `span` sub-steps of each
    interval (where a proposal of that span evaluates its network)."""
    import torch
    X = torch.empty((capacity, 51), dtype=torch.float32, device="cuda")
    R = torch.empty((capacity, 2), dtype=torch.float32, device="cuda")
    steps = len(record) if steps is None else steps
    with pf.EnsembleFilter(spec, M, N, seed) as f:
        f.set_proposal_span(span)
        f.record_tuples(X, R, stride=stride)
        for t in range(steps):
            f.step(record[t])
            if f.recorded_tuples() >= capacity:
                break
        n = f.recorded_tuples()
        f.record_tuples(None, None)
    return X[:n], R[:n], n


def epoch_seed(seed: int, epoch: int) -> int:
    """The permutation key of one epoch: the run's seed in the low word, the epoch above it."""
    return (int(seed) & 0xFFFFFFFF) | ((int(epoch) & 0xFFFFFFFF) << 32)


def train(theta0: np.ndarray, X, R, epochs: int = 4, batch: int = 8192, lr: float = 1e-3, seed: int = 0,
          log=None) -> tuple[np.ndarray, list]:
    """Adam on the tuples in shuffled mini-batches; returns the parameters and the loss history.
    Each epoch's order is the library's keyed permutation of the rows (pf_permutation),
    and the library gathers each batch's rows (pf_mlp_train_step_shuffled)."""
    n = X.shape[0]
    batch = min(batch, n)
    tr = pf.MLPTrainer(theta0, max_batch=batch)
    losses = []
    try:
        for ep in range(epochs):
            key = epoch_seed(seed, ep)
            for b0 in range(0, n - batch + 1, batch):
                loss, _ = tr.step_shuffled(X, R, batch, b0, key, lr=lr)
                losses.append(loss)
            if log:
                log(f"epoch {ep}: loss {np.mean(losses[-max(1, n // batch):]):.5f}")
        return tr.theta(), losses
    finally:
        tr.close()


def mean_nll(theta: np.ndarray, X, R) -> float:
    """Held-out loss of a parameter vector (one gradient-free trainer step)."""
    tr = pf.MLPTrainer(theta, max_batch=X.shape[0])
    try:
        loss, _ = tr.step(X, R, lr=0.0)
        return loss
    finally:
        tr.close()


def initial_theta(seed: int) -> np.ndarray:
    """Starting parameters: He-normal hidden layers, zero output layer (the
    zero network makes q equal the transition, so training starts from the
    bootstrap filter).  Layout: W1 (128 x 51), b1, W2 (128 x 128), b2,
    W3 (4 x 128), b3, row-major, PF_MLP_PARAMS values."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / 51), 128 * 51), np.zeros(128),
             rng.normal(0.0, np.sqrt(2.0 / 128), 128 * 128), np.zeros(128),
             np.zeros(4 * 128), np.zeros(4)]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == pf.MLP_PARAMS
    return theta


def trained_theta(spec: W.ModelSpec, record: np.ndarray, seed: int, tuples: int = 300_000, epochs: int = 2,
                  M: int = 16, N: int = 256, stride: int = 4, span: int = 1) -> np.ndarray:
    """Collect tuples with the plain filter on `record`, then train from initial_theta
    (for a proposal acting on the last `span` sub-steps of each interval)."""
    X, R, n = collect_tuples(spec, M, N, record, seed=seed, capacity=tuples, stride=stride, span=span)
    theta, _ = train(initial_theta(seed), X, R, epochs=epochs, batch=8192, lr=1e-3)
    return theta
