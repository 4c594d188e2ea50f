"""Test infrastructure: plain FP64 numpy statement of the tile-proposer MLP
(32 -> 64 -> 64 -> 1, ReLU) and of the gradient of its training loss, used
to check the library's forward and backward kernels.  Not part of the
product path: only tests/ may import it.

Parameter vector layout: W1[32][64] (input-major), b1[64], W2[64][64], b2[64],
w3[64], b3.  Loss: L = sum_s w_s * BCE(z_s, y_s), BCE on the logit z:
max(z, 0) - z y + log(1 + exp(-|z|)); dL/dz_s = w_s (sigmoid(z_s) - y_s).
"""
import numpy as np

N_IN, N_H = 32, 64
SIZES = [("W1", N_IN * N_H), ("b1", N_H), ("W2", N_H * N_H), ("b2", N_H), ("w3", N_H), ("b3", 1)]
N_PARAM = sum(n for _, n in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, k = {}, 0
    for name, n in SIZES:
        out[name] = p[k:k + n]
        k += n
    out["W1"] = out["W1"].reshape(N_IN, N_H)
    out["W2"] = out["W2"].reshape(N_H, N_H)
    out["b3"] = float(out["b3"][0])
    return out


def forward(p, X):
    q = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ q["W1"] + q["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ q["W2"] + q["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ q["w3"] + q["b3"]
    return z, (X, a1, h1, a2, h2)


def loss(p, X, y, w):
    z, _ = forward(p, X)
    y = np.asarray(y, np.float64)
    w = np.asarray(w, np.float64)
    return float(np.sum(w * (np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z))))))


def grad(p, X, y, w):
    """Analytic gradient by the chain rule through the three layers."""
    q = unpack(p)
    z, (X, a1, h1, a2, h2) = forward(p, X)
    y = np.asarray(y, np.float64)
    w = np.asarray(w, np.float64)
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y)
    g_w3 = h2.T @ dz
    g_b3 = dz.sum()
    d2 = np.outer(dz, q["w3"]) * (a2 > 0)
    g_W2 = h1.T @ d2
    g_b2 = d2.sum(0)
    d1 = (d2 @ q["W2"].T) * (a1 > 0)
    g_W1 = X.T @ d1
    g_b1 = d1.sum(0)
    return np.concatenate([g_W1.reshape(-1), g_b1, g_W2.reshape(-1), g_b2, g_w3, [g_b3]])
