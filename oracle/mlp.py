"""FP64 CPU oracle of the learned rank predictor (test infrastructure only).

A 35 -> 128 -> 128 -> 1 multilayer perceptron with tanh hidden layers, in
plain numpy float64, with the same parameter layout as the GPU kernels:
W1 [128 x 35] row-major, b1 [128], W2 [128 x 128], b2 [128], w3 [128], b3, then
mu [35], sigma [35] (input standardisation) and y_mu, y_sigma (output scale).

Loss on a batch: L = mean_i (yhat_i - (t_i - y_mu) / y_sigma)^2, yhat the
standardised output.  The gradient below is backpropagation written out term
by term; the tests pin it with finite differences.
"""
from __future__ import annotations

import numpy as np

IN, H = 35, 128
SIZES = [("W1", H * IN), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)]
TRAINABLE = sum(s for _, s in SIZES)
TOTAL = TRAINABLE + IN + IN + 2


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, off = {}, 0
    for name, size in SIZES:
        out[name] = p[off:off + size]
        off += size
    out["W1"] = out["W1"].reshape(H, IN)
    out["W2"] = out["W2"].reshape(H, H)
    out["b3"] = out["b3"][0]
    out["mu"] = p[off:off + IN]
    out["sigma"] = p[off + IN:off + 2 * IN]
    out["y_mu"] = p[off + 2 * IN]
    out["y_sigma"] = p[off + 2 * IN + 1]
    return out


def forward(p, x):
    """Predicted log2 rank for each row of x (batch x 35)."""
    q = unpack(p)
    xs = (np.asarray(x, dtype=np.float64) - q["mu"]) / q["sigma"]
    h1 = np.tanh(xs @ q["W1"].T + q["b1"])
    h2 = np.tanh(h1 @ q["W2"].T + q["b2"])
    yhat = h2 @ q["w3"] + q["b3"]
    return yhat * q["y_sigma"] + q["y_mu"]


def loss(p, x, target):
    q = unpack(p)
    yhat = (forward(p, x) - q["y_mu"]) / q["y_sigma"]
    t = (np.asarray(target, dtype=np.float64) - q["y_mu"]) / q["y_sigma"]
    return float(np.mean((yhat - t) ** 2))


def loss_grad(p, x, target):
    """(loss, gradient over the TRAINABLE parameters in layout order)."""
    q = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    xs = (x - q["mu"]) / q["sigma"]
    h1 = np.tanh(xs @ q["W1"].T + q["b1"])
    h2 = np.tanh(h1 @ q["W2"].T + q["b2"])
    yhat = h2 @ q["w3"] + q["b3"]
    t = (np.asarray(target, dtype=np.float64) - q["y_mu"]) / q["y_sigma"]
    r = yhat - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B                      # dL/dyhat
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = (dy[:, None] * q["w3"][None, :]) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ q["W2"]) * (1.0 - h1 * h1)
    gW1 = dz1.T @ xs
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return L, g


def features(pivots, m, n, rel_tol):
    """log10 of the first 32 pivot magnitudes relative to the first, log10 m,
    log10 n, log10 of the relative tolerance."""
    piv = np.asarray(pivots, dtype=np.float64)
    p0 = piv[0] if piv[0] > 0 else 1.0
    f = np.empty(IN)
    for i in range(32):
        v = piv[i] if i < len(piv) else 0.0
        f[i] = np.log10(max(v / p0, 1e-30))
    f[32], f[33], f[34] = np.log10(m), np.log10(n), np.log10(max(rel_tol, 1e-300))
    return f


def adam(p, g, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) on the trainable prefix of p."""
    p = np.array(p, dtype=np.float64)
    m1 = b1 * np.asarray(m1) + (1 - b1) * g
    m2 = b2 * np.asarray(m2) + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    p[:TRAINABLE] -= lr * mh / (np.sqrt(vh) + eps)
    return p, m1, m2
