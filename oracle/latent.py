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
