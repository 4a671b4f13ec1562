"""Oracle: the proposal network's MLP in FP64 (forward, MSE loss, backward, Adam).

TEST INFRASTRUCTURE (see oracle/network.py).

x (F) -> h1 = relu(W1 x + b1) (H) -> h2 = relu(W2 h1 + b2) (H) -> y = w3 . h2 + b3,
loss = mean over the batch of (y - t)^2. Parameters in one flat array:
W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3. Adam: Kingma and Ba, "Adam: a method
for stochastic optimization", ICLR 2015 (beta1 0.9, beta2 0.999, eps 1e-8).
"""

from __future__ import annotations

import numpy as np


def n_params(nf, hidden):
    return hidden * nf + hidden + hidden * hidden + hidden + hidden + 1


def unpack(p, nf, hidden):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + hidden * nf].reshape(hidden, nf); i += hidden * nf
    b1 = p[i:i + hidden]; i += hidden
    W2 = p[i:i + hidden * hidden].reshape(hidden, hidden); i += hidden * hidden
    b2 = p[i:i + hidden]; i += hidden
    w3 = p[i:i + hidden]; i += hidden
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def forward(p, x, nf, hidden):
    W1, b1, W2, b2, w3, b3 = unpack(p, nf, hidden)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (x, a1, h1, a2, h2)


def loss(p, x, t, nf, hidden):
    y, _ = forward(p, x, nf, hidden)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(p, x, t, nf, hidden):
    """dL/dp by the chain rule, layer by layer (the flat layout of p)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, nf, hidden)
    y, (x, a1, h1, a2, h2) = forward(p, x, nf, hidden)
    B = x.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    d2 = np.outer(dy, w3) * (a2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ x
    gb1 = d1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t = step number, starting at 1); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
