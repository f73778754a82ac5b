"""FP64 CPU reference of the learned initialiser's layers.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline, never by the library.  It shares no code with the
CUDA kernels in paper_2404_07780_b300/csrc/gm_cnn.cuh and is written from the
definitions of each operation:

  convolution, 3x3, stride 2, zero padding 1 (NHWC; weights [co][3][3][ci]):
      y[b, i, j, o] = bias[o] + sum_{ky, kx, c} xp[b, 2i + ky, 2j + kx, c] w[o, ky, kx, c]
      with xp = x padded by one zero on every side;
  its adjoint in x (the input gradient) and its gradient in w and bias;
  dense layer y[n, o] = bias[o] + sum_i x[n, i] w[o, i] and its gradients;
  ReLU; the mean squared error over the first dv of d output columns;
  Adam (Kingma & Ba 2015) with bias correction;
  the network input: 2x2 block mean of the stamp, then asinh(scale * mean).

The paper motivates the network (manual starting values are a limitation it
names; CNNs that estimate galaxy parameters, Sec. 1 and Sec. 6) but prints no
architecture: the layer shapes are this project's.  Pinned in
tests/test_oracle_cnn.py against brute-force loops, scipy's 2-D correlation,
central finite differences and a hand-computed Adam step.
"""
from __future__ import annotations

import numpy as np


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))


def conv_out(h: int) -> int:
    return (h + 1) // 2


def conv_fwd(x, w, b=None, relu=False):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    n, h, wd, ci = x.shape
    ho, wo = conv_out(h), conv_out(wd)
    xp = _pad(x)
    y = np.zeros((n, ho, wo, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :]  # xp[b, 2i + ky, 2j + kx, c]
            y += patch @ w[:, ky, kx, :].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def conv_bwd_data(dy, w, h: int, wd: int, mask=None):
    """d/dx of sum(dy * conv_fwd(x, w)) for an h x wd input."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    n, ho, wo, co = dy.shape
    dxp = np.zeros((n, h + 2, wd + 2, w.shape[3]))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :] += dy @ w[:, ky, kx, :]
    dx = dxp[:, 1:h + 1, 1:wd + 1, :]
    if mask is not None:
        dx = dx * (np.asarray(mask, np.float64) > 0)
    return dx


def conv_bwd_weight(x, dy):
    """(d/dw, d/dbias) of sum(dy * conv_fwd(x, w, bias))."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    n, ho, wo, co = dy.shape
    xp = _pad(x)
    dw = np.zeros((co, 3, 3, x.shape[3]))
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + 2 * ho:2, kx:kx + 2 * wo:2, :]
            dw[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dy, patch)
    return dw, dy.sum((0, 1, 2))


def dense_fwd(x, w, b=None, relu=False):
    y = np.asarray(x, np.float64) @ np.asarray(w, np.float64).T
    if b is not None:
        y += np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def dense_bwd_data(dy, w, mask=None):
    dx = np.asarray(dy, np.float64) @ np.asarray(w, np.float64)
    if mask is not None:
        dx = dx * (np.asarray(mask, np.float64) > 0)
    return dx


def dense_bwd_weight(x, dy):
    dy = np.asarray(dy, np.float64)
    return dy.T @ np.asarray(x, np.float64), dy.sum(0)


def mse(pred, target, dv: int):
    """(loss, dpred): loss = mean over rows and the first dv columns of (pred - target)^2;
    dpred = d loss / d pred = 2 (pred - target) / (n dv) in those columns, 0 in the others."""
    pred = np.asarray(pred, np.float64)
    n, d = pred.shape
    e = np.zeros_like(pred)
    e[:, :dv] = pred[:, :dv] - np.asarray(target, np.float64)[:, :dv]
    return float((e * e).sum()) / (n * dv), 2.0 * e / (n * dv)


def adam(p, g, m, v, lr, beta1, beta2, eps, step):
    """One Adam step; returns (p, m, v) updated."""
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * np.asarray(g, np.float64)
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * np.asarray(g, np.float64) ** 2
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return np.asarray(p, np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def prep(image, scale):
    """asinh(scale * 2x2 block mean) of [G][h][w] stamps -> [G][h/2][w/2]."""
    im = np.asarray(image, np.float64)
    G, h, w = im.shape
    mean = im.reshape(G, h // 2, 2, w // 2, 2).mean((2, 4))
    return np.arcsinh(scale * mean)
