"""Error bounds between the GPU's BF16 network and the FP64 oracle's BF16 emulation.

Both sides round the same operands to bfloat16 (weights, layer inputs, hidden
activations) and differ only in what happens between the roundings: the GPU
accumulates each dot product in FP32 on the tensor cores (products of BF16
values are exact in FP32) and evaluates the tanh-form GELU in FP32 as
x / (1 + 2^a) with the hardware exp2 and reciprocal; the oracle does both in
FP64.  So, layer by layer:

* a pre-activation differs by at most the FP32 accumulation error
  gamma_K (sum |w a| + |b|), gamma_K = (K + 2) 2^-23 (K terms plus the bias and
  one spare, with truncating adds), plus |W| times the upstream activation
  differences;
* an activation before rounding differs by at most L times that (L = 1.13
  bounds |GELU'|, whose largest value is 1.12899) plus the FP32 GELU's own
  error, 3.6e-7 (|z| + |GELU(z)|) when exp2 and the reciprocal are within
  2^-21 and 2^-22 of their results (the derivation is beside the device
  code), taken here as 4e-7;
* a rounded activation differs only when a BF16 rounding boundary lies
  between the two values -- when the oracle's value is closer to a boundary
  than the difference above -- and then by one BF16 step (at most 2^-7 of
  its size); otherwise it is the same BF16 number on both sides.

Propagating these interval bounds through the three layers gives, per row and
output, a bound that is tight (about 1e-5 of the last dot product's size) for
the rows where no activation sits near a rounding boundary, and wider exactly
for the few rows where one does.  Inputs that themselves differ (states
propagated in FP32 against FP64) enter through `x_tol`, their absolute
uncertainty.
"""
import numpy as np

from oracle import mlp

L_GELU = 1.13
GELU_ERR = 4e-7


def gamma(K):
    return (K + 2) * 2.0 ** -23


def _bf16_neighbours(g):
    """Margin of g to the nearest BF16 rounding boundary and the largest BF16
    step next to its rounded value."""
    r = mlp.bf16(g)
    mag = np.abs(r).astype(np.float32).view(np.uint32).astype(np.int64)
    up = (mag + 0x10000).astype(np.uint32).view(np.float32).astype(np.float64)
    dn = np.where(mag >= 0x10000, (np.maximum(mag - 0x10000, 0)).astype(np.uint32).view(np.float32), 0.0)
    dn = dn.astype(np.float64)
    a = np.abs(g)
    ra = np.abs(r)
    hi = (ra + up) / 2.0 - a
    lo = np.where(mag >= 0x10000, a - (ra + dn) / 2.0, np.inf)  # below zero the rounding is zero either way
    margin = np.maximum(np.minimum(hi, lo), 0.0)
    step = np.maximum(up - ra, ra - dn)
    return margin, step


def _layer(a_prev, da_prev, W, b, K):
    """Rounded activation of one hidden layer and the bound on its difference."""
    z = a_prev @ W.T + b
    dz = gamma(K) * (np.abs(a_prev) @ np.abs(W).T + np.abs(b)) + da_prev @ np.abs(W).T
    g = mlp.gelu(z)
    dg = L_GELU * dz + GELU_ERR * (np.abs(z) + np.abs(g))
    margin, step = _bf16_neighbours(g)
    da = np.where(margin <= dg, step, 0.0)
    return mlp.bf16(g), da


def forward_bound(theta, X, x_tol=0.0):
    """Per row and output, the largest |o_gpu - o_oracle| the arithmetic allows
    (rows x 4), for inputs X (rows x 51) known to within x_tol (scalar or
    array) on the GPU side."""
    p = mlp.unpack(np.asarray(theta, dtype=np.float64))
    W1, W2, W3 = mlp.bf16(p["W1"]), mlp.bf16(p["W2"]), mlp.bf16(p["W3"])
    X = np.asarray(X, dtype=np.float64)
    x0 = mlp.bf16(X)
    margin0, step0 = _bf16_neighbours(X)
    dx0 = np.where(margin0 <= np.broadcast_to(x_tol, X.shape), step0, 0.0)
    a1, da1 = _layer(x0, dx0, W1, p["b1"], 64)
    a2, da2 = _layer(a1, da1, W2, p["b2"], 128)
    return gamma(128) * (np.abs(a2) @ np.abs(W3).T + np.abs(p["b3"])) + da2 @ np.abs(W3).T


def hidden_sizes(theta, X):
    """S3 (rows x 4): the size sum |W3| |a2| + |b3| of each output's last dot product,
    whose FP32 accumulation error alone bounds a row where no activation flips."""
    p = mlp.unpack(np.asarray(theta, dtype=np.float64))
    _, c = mlp.forward(theta, np.asarray(X, dtype=np.float64), bf16_emulation=True)
    return np.abs(c["a2"]) @ np.abs(mlp.bf16(p["W3"])).T + np.abs(p["b3"])


def step_bounds(spec, theta, o, zm, rows, x_prop, y, x_tol_rows=0.0, state_rtol=1e-5):
    """Bounds on the learned-proposal step (the last Euler-Maruyama sub-step at the
    observed nodes and its weight) from a bound on the network outputs.

    o, zm, rows: the oracle's network outputs, (normals, transition means) and
    network inputs per (particle, observed node); x_prop: the oracle's proposed
    states; y: the observation.  With h = sigma sqrt(dt), s = clip(o_s, -3, 3),
    the proposed value is x' = m + h r, r = o_mu + e^s z, and the node's weight
    term is s + z^2/2 - r^2/2.  An output error (d_mu, d_s) moves r by at most
    d_mu + e^s |z| (e^d_s - 1); FP32 forms x' from m and r (relative rounding of
    order 2^-23 of |m|, inside the state tolerance) and the GPU may form r back
    from x' - m, which loses 2^-22 (|m| + |x'|) / h to cancellation.
    Returns (dx rigorous, dx without flips, dl rigorous): dx per (particle,
    node, component), dl per particle."""
    n, dy = o.shape[0], o.shape[1]
    h = spec.sigma_dyn * np.sqrt(spec.dt)
    X = rows.reshape(n * dy, 51)
    B = forward_bound(theta, X, x_tol_rows).reshape(n, dy, 4)
    S3 = hidden_sizes(theta, X).reshape(n, dy, 4)
    nn = spec.J * spec.J
    nodes = np.asarray(spec.obs_idx)
    xo = np.stack([x_prop[:, nodes], x_prop[:, nn + nodes]], axis=2)  # (n, dy, 2)
    rms = np.sqrt(np.mean(xo ** 2, axis=(0, 1)))
    s = np.clip(o[..., 2:], -3.0, 3.0)
    e = np.exp(s)
    z, m = zm[..., :2], zm[..., 2:]
    r = o[..., :2] + e * z
    canc = 2.0 ** -22 * (np.abs(m) + np.abs(xo)) / h

    def moved(d):  # |delta r| and |delta x'| for an output bound d
        dr = d[..., :2] + e * np.abs(z) * np.expm1(d[..., 2:]) + canc
        return dr, state_rtol * np.maximum(np.abs(xo), rms) + h * dr

    dr, dx = moved(B)
    _, dx_nf = moved(S3 * gamma(128))
    ds = B[..., 2:]
    dq = ds + np.abs(r) * dr + dr ** 2 / 2.0
    q = s + z ** 2 / 2.0 - r ** 2 / 2.0
    sig2 = spec.sigma_obs ** 2
    res = np.abs(np.asarray(y, dtype=np.float64)[None, :] - xo[..., 0])
    dg = res / sig2 * dx[..., 0] + dx[..., 0] ** 2 / (2.0 * sig2)
    terms_g = res ** 2 / (2.0 * sig2)
    dl = (dq.sum(axis=(1, 2)) + dg.sum(axis=1) + gamma(dy) * terms_g.sum(axis=1)
          + gamma(2 * dy) * np.abs(q).sum(axis=(1, 2)))
    return dx, dx_nf, dl
