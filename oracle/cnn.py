"""FP64 reference of the learned post-equaliser (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may use this
module; the CUDA path never does.

The paper has no learned stage; its learned counterpart here is a small 1-D
CNN applied to the chain's phase-recovered symbols (paper-silent; the
readings are stated once here):

  features  x[n, :] = (Re z_X[n], Im z_X[n], Re z_Y[n], Im z_Y[n]), n = 0..K-1
  layer l   a_l[n, co] = b_l[co] + sum_k sum_ci W_l[k, ci, co] h_{l-1}[n + k - c, ci]
            ("same" zero padding, c = (ksize - 1) / 2, h_0 = x),
            h_l = max(a_l, 0) for the hidden layers, h_L = a_L for the last;
  output    y = x + h_L (residual), 4 -> C -> ... -> C -> 4 channels;
  loss      J = sum_{n, f} (y[n, f] - t[n, f])^2 / (4 K), t = the transmitted
            symbols in the same feature layout;
  Adam      m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
            p <- p - lr (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps)
            at step s = 1, 2, ... (Kingma & Ba, ICLR 2015), defaults lr 1e-3,
            b1 0.9, b2 0.999, eps 1e-8.

Parameters are a list of (W, b) per layer with W of shape (ksize, ci, co).
"""
from __future__ import annotations

import numpy as np


def features(z: np.ndarray) -> np.ndarray:
    """(2, K) complex symbols -> (K, 4) real features."""
    return np.stack([z[0].real, z[0].imag, z[1].real, z[1].imag], axis=1).astype(np.float64)


def symbols(x: np.ndarray) -> np.ndarray:
    """(K, 4) real features -> (2, K) complex symbols."""
    return np.stack([x[:, 0] + 1j * x[:, 1], x[:, 2] + 1j * x[:, 3]])


def shift_rows(h: np.ndarray, s: int) -> np.ndarray:
    """out[n] = h[n + s] inside [0, K), zero outside."""
    K = h.shape[0]
    out = np.zeros_like(h)
    lo, hi = max(0, -s), min(K, K - s)
    if hi > lo:
        out[lo:hi] = h[lo + s:hi + s]
    return out


def conv1d(h: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """a[n, co] = b[co] + sum_k h[n + k - c, :] @ W[k] (zero padding)."""
    ks = W.shape[0]
    c = (ks - 1) // 2
    a = np.broadcast_to(b, (h.shape[0], W.shape[2])).copy()
    for k in range(ks):
        a += shift_rows(h, k - c) @ W[k]
    return a


def conv1d_backward(h: np.ndarray, W: np.ndarray, da: np.ndarray):
    """Gradients of a = conv1d(h, W, b) given da = dJ/da: (dh, dW, db)."""
    ks = W.shape[0]
    c = (ks - 1) // 2
    dW = np.stack([shift_rows(h, k - c).T @ da for k in range(ks)])
    db = da.sum(axis=0)
    dh = np.zeros_like(h)
    for k in range(ks):
        # a[n] uses h[n + k - c] W[k]  =>  dh[m] += da[m - (k - c)] W[k]^T
        dh += shift_rows(da, -(k - c)) @ W[k].T
    return dh, dW, db


def forward(params, x: np.ndarray, x_conv: np.ndarray | None = None):
    """Returns (y, cache) with cache = [h_0, a_1, h_1, ..., a_L].

    x_conv (default x) feeds the first convolution; the residual always adds
    x.  A caller whose network stores its input features at lower precision
    passes them rounded here (a statement about the input, not the method).
    """
    h = x if x_conv is None else x_conv
    cache = [h]
    L = len(params)
    for l, (W, b) in enumerate(params):
        a = conv1d(h, W, b)
        cache.append(a)
        h = np.maximum(a, 0.0) if l < L - 1 else a
        if l < L - 1:
            cache.append(h)
    return x + h, cache


def loss_and_grads(params, x: np.ndarray, t: np.ndarray, x_conv: np.ndarray | None = None):
    """J and its gradients [(dW, db)] per layer (x_conv as in forward)."""
    y, cache = forward(params, x, x_conv)
    K = x.shape[0]
    diff = y - t
    J = float(np.sum(diff * diff) / (4.0 * K))
    dy = 2.0 * diff / (4.0 * K)
    L = len(params)
    grads = [None] * L
    da = dy                                   # the residual skip does not change dJ/dh_L
    for l in range(L - 1, -1, -1):
        h_in = cache[2 * l] if l > 0 else cache[0]
        dh, dW, db = conv1d_backward(h_in, params[l][0], da)
        grads[l] = (dW, db)
        if l > 0:
            a_prev = cache[2 * l - 1]
            da = dh * (a_prev > 0)
    return J, grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.s = 0

    def step(self, params, grads):
        """New parameters after one Adam step on grads."""
        self.s += 1
        c1 = 1.0 - self.b1 ** self.s
        c2 = 1.0 - self.b2 ** self.s
        out = []
        for i in range(len(params)):
            new = []
            for j in range(2):
                p, g = params[i][j], grads[i][j]
                self.m[i][j] = self.b1 * self.m[i][j] + (1.0 - self.b1) * g
                self.v[i][j] = self.b2 * self.v[i][j] + (1.0 - self.b2) * g * g
                new.append(p - self.lr * (self.m[i][j] / c1) / (np.sqrt(self.v[i][j] / c2) + self.eps))
            out.append((new[0], new[1]))
        return out


# Seeded initial weights are inputs of the method: they come from the shared
# generator module (linksim), like every other random draw.
from linksim import cnn_init_params as init_params  # noqa: E402,F401
