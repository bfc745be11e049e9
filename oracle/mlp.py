"""Plain FP64 CPU oracle of the learned preconditioner correction.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may use this module; the library never does.

The paper preconditions the out-of-subspace gradient with the TPA kinetic
preconditioner K (Eqs. 16-18).  The learned part multiplies K, per plane wave
G and band n, by m = exp(clip(s, -3, 3)), where s is the output of a small
per-coefficient network (two hidden layers of 64, tanh):

  features u (3):  u0 = log(1 + x),  x = (|G|^2 / 2) / T_n,
                   T_n = sum_G (|G|^2/2) |g_nG|^2 / sum_G |g_nG|^2
                   u1 = log(1 + |g_nG| / rms_n),  rms_n = (sum_G |g_nG|^2 / N_pw)^{1/2}
                   u2 = eps_n  (band energy <n|F^n|n> / w_n, Ha)
  h1 = tanh(W1 u + b1), h2 = tanh(W2 h1 + b2), s = w3 . h2 + b3

Training minimises the weighted mean square L = sum_i w_i (s_i - t_i)^2 /
sum_i w_i with Adam (Kingma & Ba 2015).  Parameters are one flat vector in
the order W1 (64 x 3, row major), b1 (64), W2 (64 x 64, row major), b2 (64),
w3 (64), b3 (1): 4481 values.

Pins (tests/test_oracle_mlp.py): the gradient against central differences of
the loss; the network's closed forms (zero weights give s = b3; a single
active path reduces to nested tanh); Adam's first step against its closed
form; the features against their definitions on a hand-made residual.
"""
from __future__ import annotations

import numpy as np

H = 64
NPARAM = H * 3 + H + H * H + H + H + 1


def unpack(p: np.ndarray):
    """Views (W1, b1, W2, b2, w3, b3) of the flat parameter vector."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + 3 * H].reshape(H, 3); o += 3 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def features(g: np.ndarray, g2half: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """Features of every coefficient of a residual block g (npw x nb, complex):
    returns (npw * nb) x 3 in column-major order (band by band)."""
    npw, nb = g.shape
    a2 = np.abs(g) ** 2
    s0 = a2.sum(axis=0)
    s1 = (g2half[:, None] * a2).sum(axis=0)
    T = s1 / np.maximum(s0, 1e-300)
    rms = np.sqrt(s0 / npw)
    x = g2half[:, None] / np.maximum(T, 1e-300)[None, :]
    r = np.abs(g) / np.maximum(rms, 1e-300)[None, :]
    u = np.empty((npw, nb, 3))
    u[:, :, 0] = np.log1p(x)
    u[:, :, 1] = np.log1p(r)
    u[:, :, 2] = eps[None, :]
    return u.transpose(1, 0, 2).reshape(-1, 3)


def forward(p: np.ndarray, U: np.ndarray):
    """Network outputs s (n) and the hidden activations."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    h1 = np.tanh(U @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    s = h2 @ w3 + b3
    return s, h1, h2


def multiplier(p: np.ndarray, U: np.ndarray) -> np.ndarray:
    """m = exp(clip(s, -3, 3)): the factor applied to the TPA step."""
    s, _, _ = forward(p, U)
    return np.exp(np.clip(s, -3.0, 3.0))


def loss_and_grad(p: np.ndarray, U: np.ndarray, t: np.ndarray, w: np.ndarray):
    """L = sum w (s - t)^2 / sum w and dL/dp by back-propagation."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    s, h1, h2 = forward(p, U)
    sw = float(np.sum(w))
    r = s - t
    L = float(np.sum(w * r * r) / sw)
    ds = 2.0 * w * r / sw                      # dL/ds
    gw3 = h2.T @ ds
    gb3 = np.sum(ds)
    dz2 = np.outer(ds, w3) * (1.0 - h2 * h2)   # through tanh
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ U
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return L, g


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
