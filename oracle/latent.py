"""Latent decoder reference (plain FP64 numpy).  TEST INFRASTRUCTURE ONLY.

decode(): the MLP 32 -> 64 -> 64 -> n1 + 27 n2 with ReLU after the first two
layers, giving each leaf's Fourier coefficients (the learned stand-in for the
stored coefficients of Sec. 4.1).  table(): sigma = max(0, Eq. 7) and the 27
z of Eq. 9 at time t, i.e. what the renderer's per-frame table holds.
"""

import numpy as np

import oracle


def decode(latents, w1, b1, w2, b2, w3, b3):
    x = np.asarray(latents, np.float64)
    h1 = np.maximum(x @ np.asarray(w1, np.float64).T + b1, 0.0)
    h2 = np.maximum(h1 @ np.asarray(w2, np.float64).T + b2, 0.0)
    return h2 @ np.asarray(w3, np.float64).T + b3


def table(coeffs, t, period=60.0, n1=31, n2=5):
    c = np.asarray(coeffs, np.float64)
    b = oracle.basis(max(n1, n2), t, period)
    out = np.zeros((c.shape[0], 32))
    out[:, 0] = np.maximum(c[:, :n1] @ b[:n1], 0.0)
    out[:, 1:28] = c[:, n1:].reshape(-1, 27, n2) @ b[:n2]
    return out


def loss_grad(latents, w1, b1, w2, b2, w3, b3, targets, coef_weight):
    """L = sum_rows sum_j coef_weight_j (y_j - target_j)^2 and its gradients
    (hand-written back-propagation in FP64).  Returns (L, dlatents, dict of
    weight gradients)."""
    x = np.asarray(latents, np.float64)
    W1, W2, W3 = (np.asarray(w, np.float64) for w in (w1, w2, w3))
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    r = y - targets
    cw = np.asarray(coef_weight, np.float64)
    L = float(np.sum(cw * r * r))
    dy = 2.0 * cw * r
    g = {"w3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ W3) * (z2 > 0)
    g["w2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g["w1"], g["b1"] = dz1.T @ x, dz1.sum(0)
    return L, dz1 @ W1, g
