"""The learned proposal's network on the GPU against the FP64 oracle (oracle/mlp.py).

Tolerances (BF16 operands and activations on both sides; the GPU accumulates
in FP32, the oracle works in FP64; tests/_mlp_bounds.py derives the bounds):
* forward: every output within the interval bound that propagates the FP32
  accumulation error gamma_K = (K + 2) 2^-23 of each dot product and a
  possible one-step BF16 rounding flip of every activation close enough to a
  rounding boundary; and at most 2 % of the rows beyond the bound of the last
  layer's accumulation alone, gamma_128 (sum |W3| |a2| + |b3|) -- a row leaves
  it only when one of its 256 hidden activations rounds to the other BF16
  neighbour on the two sides, which the FP32 accumulation error (about
  2^-24 sqrt(K) of a dot product) makes rare (0.5 % of rows measured);
* gradient, with the oracle also storing the backward intermediates d_z2 and
  d_z1 in BF16 as the GPU does: relative error <= 1e-4 overall and 1e-3 per
  parameter block (FP32 accumulation over the batch, and the rare flips:
  each moves one row's term by 2^-8 of itself); the loss within the FP32
  accumulation bound gamma_B of its B row terms;
* Adam's first step: theta moves by lr sign(g) wherever |g| is not tiny,
* training steps are bit-for-bit repeatable.
"""
import numpy as np
import pytest

import _mlp_bounds
from oracle import mlp
from paper_1407_8071_gb300 import pf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _theta(seed, out_scale=0.5):
    p = mlp.unpack(mlp.init_params(seed, out_scale=out_scale))
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0.0, 0.1, p[k].shape)
    return mlp.pack(p).astype(np.float32).astype(np.float64)


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 1.0, (n, mlp.IN))
    R = rng.normal(0.0, 1.0, (n, 2)) + 0.3 * X[:, :2]
    return X.astype(np.float32).astype(np.float64), R.astype(np.float32).astype(np.float64)


def check_forward(got, ref, bound, S3):
    err = np.abs(got - ref)
    assert np.all(err <= bound + 1e-12), (np.max(err / bound), np.unravel_index(np.argmax(err / bound), err.shape))
    beyond = np.any(err > _mlp_bounds.gamma(128) * S3 + 1e-12, axis=1)
    assert beyond.sum() <= 0.02 * len(beyond) + 2, beyond.mean()


@pytest.mark.parametrize("n", [1, 17, 64, 1000, 70001])
def test_forward_matches_oracle(n):
    th = _theta(1)
    X, _ = _rows(n, 2)
    d_out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    pf.pf_mlp_forward(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(th.astype(np.float32)).cuda(),
                      d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().astype(np.float64)
    ref, _ = mlp.forward(th, X, bf16_emulation=True)
    check_forward(got, ref, _mlp_bounds.forward_bound(th, X), _mlp_bounds.hidden_sizes(th, X))


def _blocks():
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp._SHAPES])
    return [(name, offs[i], offs[i + 1]) for i, (name, _) in enumerate(mlp._SHAPES)]


@pytest.mark.parametrize("B", [64, 300, 4096])
def test_gradient_matches_oracle(B):
    th = _theta(3)
    X, R = _rows(B, 4)
    tr = pf.MLPTrainer(th, max_batch=B)
    loss, g = tr.step(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(R.astype(np.float32)).cuda(),
                      lr=0.0, want_grad=True)
    tr.close()
    lo, go = mlp.loss_and_grad(th, X, R, bf16_emulation=True, bf16_backward=True)
    # the GPU sums the B row losses in FP32: within gamma_B of the sum of their sizes
    rows_nll = mlp.nll(mlp.forward(th, X, bf16_emulation=True)[0], R)
    assert abs(loss - lo) <= _mlp_bounds.gamma(B) * np.mean(np.abs(rows_nll)) + 1e-6 * abs(lo)
    g = g.astype(np.float64)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    for name, a, b in _blocks():
        assert np.linalg.norm(g[a:b] - go[a:b]) <= 1e-3 * np.linalg.norm(go[a:b]) + 1e-9, name


def test_adam_first_step_and_determinism():
    th = _theta(5)
    X, R = _rows(2048, 6)
    dX, dR = torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(R.astype(np.float32)).cuda()
    lr = 1e-3
    t1 = pf.MLPTrainer(th, max_batch=2048)
    t1.step(dX, dR, lr=lr)
    th1 = t1.theta().astype(np.float64)
    t2 = pf.MLPTrainer(th, max_batch=2048)
    t2.step(dX, dR, lr=lr)
    assert np.array_equal(t1.theta(), t2.theta())
    t1.close()
    t2.close()
    _, go = mlp.loss_and_grad(th, X, R, bf16_emulation=True)
    big = np.abs(go) > 1e-2 * np.abs(go).max()
    step = th1 - th
    assert np.all(np.abs(step) <= lr * 1.0001 + 1e-7)
    assert np.mean(np.sign(step[big]) == -np.sign(go[big])) >= 0.99


def test_training_reduces_the_loss():
    th = mlp.init_params(7, out_scale=0.0)
    X, R = _rows(8192, 8)
    dX, dR = torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(R.astype(np.float32)).cuda()
    tr = pf.MLPTrainer(th, max_batch=8192)
    losses = [tr.step(dX, dR, lr=3e-3)[0] for _ in range(60)]
    tr.close()
    # R = noise + 0.3 X[:, :2]: a good fit removes part of the variance
    assert losses[-1] < losses[0] - 0.05, (losses[0], losses[-1])


@pytest.mark.parametrize("J,P", [(8, 300), (40, 37), (2, 5)])
def test_lattice_forward_on_tcgen05_matches_oracle(J, P):
    """The filter's fused form: input rows gathered from lattice states on the
    device, the network on tcgen05 with TMEM accumulators (a ragged last tile
    of 128 rows), against the FP64 oracle's rows (oracle/mlp.patch_rows) and
    BF16-emulating forward; tolerance as for the forward above (the bound
    allows the FP32 GELU's own error, 4e-7 (|z| + |g(z)|))."""
    from paper_1407_8071_gb300 import workloads as W
    th = _theta(9)
    nodes = W.fhn_obs_nodes(J, 4 if J > 2 else 1)
    rng = np.random.default_rng(J * 1000 + P)
    x = rng.normal(0.0, 0.3, (P, 2 * J * J)).astype(np.float32)
    y = rng.normal(0.0, 0.5, len(nodes)).astype(np.float32)
    d_out = torch.full((P * len(nodes), 4), float("nan"), dtype=torch.float32, device="cuda")
    pf.pf_proposal_forward(J, torch.from_numpy(x).cuda(), nodes, torch.from_numpy(y).cuda(),
                           torch.from_numpy(th.astype(np.float32)).cuda(), d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().astype(np.float64)
    rows = np.concatenate([mlp.patch_rows(x[p].astype(np.float64), J, nodes, y.astype(np.float64)) for p in range(P)])
    ref, _ = mlp.forward(th, rows, bf16_emulation=True)
    assert np.all(np.isfinite(got))
    check_forward(got, ref, _mlp_bounds.forward_bound(th, rows), _mlp_bounds.hidden_sizes(th, rows))


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 4096, 70001])
def test_permutation_is_a_bijection(n):
    d = torch.empty(n, dtype=torch.int64, device="cuda")
    perms = []
    for seed in (1, 2, 1 | (7 << 32)):
        pf.pf_permutation(n, seed, d)
        torch.cuda.synchronize()
        p = d.cpu().numpy()
        assert np.array_equal(np.sort(p), np.arange(n))
        perms.append(p)
    if n >= 1000:
        assert not np.array_equal(perms[0], perms[1]) and not np.array_equal(perms[0], perms[2])
        # a shuffle, not a shift: consecutive rows land far apart
        assert np.mean(np.abs(np.diff(perms[0]))) > n / 8


def test_shuffled_step_trains_on_the_permuted_rows():
    """The library's gathered batch is exactly rows pi(first ..) of the tuples: the
    shuffled step's gradient is bit-identical to the plain step's on X[pi]."""
    th = _theta(5)
    X, R = _rows(5000, 6)
    d_X = torch.from_numpy(X.astype(np.float32)).cuda()
    d_R = torch.from_numpy(R.astype(np.float32)).cuda()
    seed, first, batch = 12345 | (3 << 32), 1024, 2048
    d_p = torch.empty(5000, dtype=torch.int64, device="cuda")
    pf.pf_permutation(5000, seed, d_p)
    idx = d_p[first:first + batch]
    t1, t2 = pf.MLPTrainer(th, max_batch=batch), pf.MLPTrainer(th, max_batch=batch)
    try:
        l1, g1 = t1.step_shuffled(d_X, d_R, batch, first, seed, lr=0.0, want_grad=True)
        l2, g2 = t2.step(d_X[idx].contiguous(), d_R[idx].contiguous(), lr=0.0, want_grad=True)
    finally:
        t1.close()
        t2.close()
    assert l1 == l2 and np.array_equal(g1, g2)
