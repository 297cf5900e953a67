"""FP64 oracle of the learned proposal's network (TEST INFRASTRUCTURE).

The growth direction "learned proposal" replaces, at the observed lattice
nodes and only for the last Euler-Maruyama sub-step before an observation,
the transition p(x'|x) = N(m_p(x), (sigma sqrt dt)^2 I) by a Gaussian
q(x'|x, y) = N(m_p + h o_mu, (h exp(o_s))^2 I), h = sigma sqrt(dt), whose
residual mean o_mu and log-scale o_s come from a small network; the
importance weight then carries the full ratio p g / q, so the filter stays
consistent (the paper's analysis admits such tailored importance functions,
Sec. 6 footnote; Remark after Cor. 2 for the auxiliary filter).

Network: 51 inputs (the 5x5 patch of v, the 5x5 patch of w around the node,
row-major with zero-flux mirroring at the lattice edge, and y at the node)
-> 128 -> 128 -> 4 (o_mu_v, o_mu_w, o_s_v, o_s_w), GELU in its tanh form
(Hendrycks & Gimpel 2016) g(x) = x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) / 2
between layers, written here as that definition in FP64.  Parameters are one flat FP32 vector:
W1 (128 x 51), b1 (128), W2 (128 x 128), b2 (128), W3 (4 x 128), b3 (4).

Loss: Gaussian negative log-likelihood of the standardised residual
r = (x'_target - m_p) / h per row and component,
    L = sum_c [ (r_c - o_mu_c)^2 / (2 exp(2 s_c)) + s_c ],  s_c = clip(o_s_c, -3, 3)
(averaged over rows); its gradient is written out by hand below and pinned by
central finite differences in the tests.

BF16 emulation: with bf16=True the weights and each layer's input are
rounded to bfloat16 (round to nearest even) and everything else is FP64,
which brackets the GPU's BF16-operand / FP32-accumulate kernels.
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 51, 128, 4
CLAMP = 3.0

_SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in _SHAPES)


def unpack(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in _SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    assert o == len(theta)
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in _SHAPES])


def init_params(seed: int, out_scale: float = 0.0) -> np.ndarray:
    """He-style init for the hidden layers; the last layer scaled by out_scale
    (0 gives q = p exactly, the safe start)."""
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.normal(0.0, math.sqrt(2.0 / IN), (HID, IN)), "b1": np.zeros(HID),
        "W2": rng.normal(0.0, math.sqrt(2.0 / HID), (HID, HID)), "b2": np.zeros(HID),
        "W3": rng.normal(0.0, math.sqrt(1.0 / HID), (OUT, HID)) * out_scale, "b3": np.zeros(OUT),
    }
    return pack(p).astype(np.float32).astype(np.float64)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest bfloat16 (ties to even), via FP32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    nan = np.isnan(f)
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


GELU_K0 = math.sqrt(2.0 / math.pi)
GELU_K1 = 0.044715


def gelu(x):
    """x (1 + tanh(u)) / 2, u = k0 (x + k1 x^3): the tanh form of x Phi(x)."""
    return 0.5 * x * (1.0 + np.tanh(GELU_K0 * (x + GELU_K1 * x * x * x)))


def gelu_grad(x):
    """d/dx of gelu: (1 + t) / 2 + x (1 - t^2) u' / 2, t = tanh(u), u' = k0 (1 + 3 k1 x^2)."""
    t = np.tanh(GELU_K0 * (x + GELU_K1 * x * x * x))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_K0 * (1.0 + 3.0 * GELU_K1 * x * x)


def forward(theta: np.ndarray, X: np.ndarray, bf16_emulation: bool = False):
    """Outputs (rows x 4) and the activations needed by backward."""
    p = unpack(theta)
    rnd = bf16 if bf16_emulation else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3 = rnd(p["W1"]), rnd(p["W2"]), rnd(p["W3"])
    x0 = rnd(X)
    z1 = x0 @ W1.T + p["b1"]
    a1 = gelu(z1)
    a1r = rnd(a1)
    z2 = a1r @ W2.T + p["b2"]
    a2 = gelu(z2)
    a2r = rnd(a2)
    out = a2r @ W3.T + p["b3"]
    return out, dict(x0=x0, z1=z1, a1=a1r, z2=z2, a2=a2r, W1=W1, W2=W2, W3=W3)


def nll(out: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Per-row Gaussian NLL of standardised residuals R (rows x 2)."""
    mu, s = out[:, :2], np.clip(out[:, 2:], -CLAMP, CLAMP)
    return np.sum((R - mu) ** 2 / (2.0 * np.exp(2.0 * s)) + s, axis=1)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, R: np.ndarray, bf16_emulation: bool = False,
                  bf16_backward: bool = False):
    """Mean NLL over the rows and its gradient with respect to theta (hand-written backprop).
    bf16_backward also rounds the two hidden-layer pre-activation gradients d_z2 and d_z1 to
    bfloat16 where they are formed (the precision in which a BF16 training step stores them
    between its passes)."""
    out, c = forward(theta, X, bf16_emulation)
    rb = bf16 if bf16_backward else (lambda a: a)
    B = len(X)
    loss = float(np.mean(nll(out, R)))
    mu, s_raw = out[:, :2], out[:, 2:]
    s = np.clip(s_raw, -CLAMP, CLAMP)
    inv = np.exp(-2.0 * s)
    d_out = np.zeros_like(out)
    d_out[:, :2] = -(R - mu) * inv / B
    inside = (s_raw > -CLAMP) & (s_raw < CLAMP)
    d_out[:, 2:] = np.where(inside, 1.0 - (R - mu) ** 2 * inv, 0.0) / B
    g = {}
    g["W3"] = d_out.T @ c["a2"]
    g["b3"] = d_out.sum(0)
    d_a2 = d_out @ c["W3"]
    d_z2 = rb(d_a2 * gelu_grad(c["z2"]))
    g["W2"] = d_z2.T @ c["a1"]
    g["b2"] = d_z2.sum(0)
    d_a1 = d_z2 @ c["W2"]
    d_z1 = rb(d_a1 * gelu_grad(c["z1"]))
    g["W1"] = d_z1.T @ c["x0"]
    g["b1"] = d_z1.sum(0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def patch_rows(x: np.ndarray, J: int, nodes, y: np.ndarray) -> np.ndarray:
    """Network inputs for the observed nodes of one lattice state x (2 J^2):
    5x5 patches of v and w (zero-flux mirror at the edges) and y at the node."""
    nn = J * J
    v, w = x[:nn].reshape(J, J), x[nn:].reshape(J, J)

    def refl(k):
        if k < 0:
            return -k - 1
        if k >= J:
            return 2 * J - k - 1
        return k

    rows = np.empty((len(nodes), IN))
    for r, node in enumerate(nodes):
        i, j = divmod(int(node), J)
        idx = [(refl(i + di), refl(j + dj)) for di in range(-2, 3) for dj in range(-2, 3)]
        rows[r, :25] = [v[a, b] for a, b in idx]
        rows[r, 25:50] = [w[a, b] for a, b in idx]
        rows[r, 50] = y[r]
    return rows
