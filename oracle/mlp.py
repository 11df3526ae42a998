"""FP64 CPU oracle of the proposal network -- TEST INFRASTRUCTURE ONLY.

The proposal MLP 6 -> 128 -> 128 -> 1024 (ReLU) with a soft cross-entropy
loss against cluster masses q, written from its definition with numpy:
  h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), z = h2 W3^T + b3,
  loss = -(1/B) sum_n sum_g q_ng log softmax(z_n)_g,
and its gradient by backpropagation (dz = (softmax(z) - q) / B, ...).
Parameters are one flat vector [W1 | b1 | W2 | b2 | W3 | b3] (row-major
weights, out x in).  Pinned in tests/test_oracle_pins.py by central finite
differences, so the backward pass is checked against the forward pass, not
against itself.  Also the k-means assignment rule (nearest centroid, ties
to the lower index) and the top-4 rule (largest logits, ties to the lower
index) against which the GPU's integer decisions are checked.
"""
from __future__ import annotations

import numpy as np

SHAPES = [(128, 6), (128,), (128, 128), (128,), (1024, 128), (1024,)]


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, off = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[off:off + n].reshape(s))
        off += n
    return out


def forward(theta, x):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    z = h2 @ W3.T + b3
    return h1, h2, z


def log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - m - np.log(np.exp(z - m).sum(axis=1, keepdims=True))


def loss(theta, x, q):
    _, _, z = forward(theta, x)
    return float(-(np.asarray(q, dtype=np.float64) * log_softmax(z)).sum() / x.shape[0])


def grad(theta, x, q):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    h1, h2, z = forward(theta, x)
    B = x.shape[0]
    dz = (np.exp(log_softmax(z)) - q) / B
    gW3, gb3 = dz.T @ h2, dz.sum(0)
    dh2 = (dz @ W3) * (h2 > 0)
    gW2, gb2 = dh2.T @ h1, dh2.sum(0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    gW1, gb1 = dh1.T @ x, dh1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def top4(z):
    """Indices of the 4 largest entries per row, ties to the lower index."""
    idx = np.argsort(-np.asarray(z), axis=1, kind="stable")
    return idx[:, :4]


def nearest_centroid(points, centroids):
    """Nearest centroid per point (squared distance), ties to the lower index."""
    d2 = ((np.asarray(points)[:, None, :] - np.asarray(centroids)[None, :, :]) ** 2).sum(-1)
    return np.argmin(d2, axis=1), d2
