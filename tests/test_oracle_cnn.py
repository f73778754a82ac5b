"""Pins of the FP64 CNN reference (oracle/cnn.py) against what fixes each layer:
brute-force loops written from the definition, scipy's 2-D correlation,
central finite differences of scalar losses, and hand-computed values."""
import math

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def _brute_conv(x, w, b):
    n, h, wd, ci = x.shape
    co = w.shape[0]
    ho, wo = (h + 1) // 2, (wd + 1) // 2
    y = np.zeros((n, ho, wo, co))
    for bb in range(n):
        for i in range(ho):
            for j in range(wo):
                for o in range(co):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            r, c = 2 * i + ky - 1, 2 * j + kx - 1
                            if 0 <= r < h and 0 <= c < wd:
                                s += float(np.dot(x[bb, r, c, :], w[o, ky, kx, :]))
                    y[bb, i, j, o] = s
    return y


@pytest.mark.parametrize("shape", [(2, 6, 6, 3, 4), (1, 5, 7, 2, 3), (1, 1, 1, 1, 2), (3, 8, 4, 1, 8)])
def test_conv_fwd_is_the_definition(shape):
    n, h, w, ci, co = shape
    rng = np.random.default_rng(1)
    x, W, b = rng.normal(size=(n, h, w, ci)), rng.normal(size=(co, 3, 3, ci)), rng.normal(size=co)
    np.testing.assert_allclose(cnn.conv_fwd(x, W, b), _brute_conv(x, W, b), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(cnn.conv_fwd(x, W, b, relu=True), np.maximum(_brute_conv(x, W, b), 0), atol=1e-12)


def test_conv_fwd_single_channel_is_strided_correlate2d():
    rng = np.random.default_rng(2)
    x, W = rng.normal(size=(9, 10)), rng.normal(size=(3, 3))
    ref = correlate2d(np.pad(x, 1), W, mode="valid")[::2, ::2]
    got = cnn.conv_fwd(x[None, :, :, None], W[None, :, :, None])[0, :, :, 0]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def _fd(f, a, h=1e-6):
    g = np.zeros_like(a)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        ap, am = a.copy(), a.copy()
        ap[idx] += h
        am[idx] -= h
        g[idx] = (f(ap) - f(am)) / (2 * h)
    return g


def test_conv_gradients_are_finite_differences():
    rng = np.random.default_rng(3)
    n, h, w, ci, co = 2, 5, 6, 3, 4
    x, W, b = rng.normal(size=(n, h, w, ci)), rng.normal(size=(co, 3, 3, ci)), rng.normal(size=co)
    r = rng.normal(size=(n, 3, 3, co))  # upstream gradient dL/dy
    loss = lambda x_, W_, b_: float((r * cnn.conv_fwd(x_, W_, b_)).sum())
    np.testing.assert_allclose(cnn.conv_bwd_data(r, W, h, w), _fd(lambda a: loss(a, W, b), x), rtol=1e-6, atol=1e-8)
    dW, db = cnn.conv_bwd_weight(x, r)
    np.testing.assert_allclose(dW, _fd(lambda a: loss(x, a, b), W), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(db, _fd(lambda a: loss(x, W, a), b), rtol=1e-6, atol=1e-8)


def test_relu_network_gradient_through_masks():
    # two convolutions with ReLU, then a dense layer: the chain of layer gradients with the
    # ReLU masks equals the finite-difference gradient of the whole network
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 8, 8, 1))
    W1, b1 = rng.normal(size=(4, 3, 3, 1)), rng.normal(size=4) * 0.1
    W2, b2 = rng.normal(size=(8, 3, 3, 4)), rng.normal(size=8) * 0.1
    D, bd = rng.normal(size=(3, 2 * 2 * 8)), rng.normal(size=3)
    t = rng.normal(size=(2, 3))

    def net(W1_):
        a1 = cnn.conv_fwd(x, W1_, b1, relu=True)
        a2 = cnn.conv_fwd(a1, W2, b2, relu=True)
        return a1, a2, cnn.dense_fwd(a2.reshape(2, -1), D, bd)

    a1, a2, y = net(W1)
    loss, dy = cnn.mse(y, t, 3)
    d2 = cnn.dense_bwd_data(dy, D, mask=a2.reshape(2, -1)).reshape(a2.shape)
    d1 = cnn.conv_bwd_data(d2, W2, 4, 4, mask=a1)
    dW1, _ = cnn.conv_bwd_weight(x, d1)
    fd = _fd(lambda a: cnn.mse(net(a)[2], t, 3)[0], W1, h=1e-7)
    np.testing.assert_allclose(dW1, fd, rtol=1e-5, atol=1e-8)


def test_dense_gradients_are_finite_differences():
    rng = np.random.default_rng(5)
    x, W, b = rng.normal(size=(4, 6)), rng.normal(size=(5, 6)), rng.normal(size=5)
    r = rng.normal(size=(4, 5))
    loss = lambda x_, W_, b_: float((r * cnn.dense_fwd(x_, W_, b_)).sum())
    np.testing.assert_allclose(cnn.dense_bwd_data(r, W), _fd(lambda a: loss(a, W, b), x), rtol=1e-6, atol=1e-8)
    dW, db = cnn.dense_bwd_weight(x, r)
    np.testing.assert_allclose(dW, _fd(lambda a: loss(x, a, b), W), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(db, _fd(lambda a: loss(x, W, a), b), rtol=1e-6, atol=1e-8)


def test_mse_by_hand():
    pred = np.array([[1.0, 2.0, 9.0], [0.0, -1.0, 9.0]])
    target = np.array([[0.5, 2.0], [1.0, 1.0]])
    loss, d = cnn.mse(pred, target, 2)
    assert loss == pytest.approx((0.25 + 0 + 1 + 4) / 4)
    np.testing.assert_allclose(d, [[0.25, 0.0, 0.0], [-0.5, -1.0, 0.0]])  # 2 e / (2 rows * 2 columns)


def test_adam_first_step_is_a_signed_step_of_lr():
    # step 1 from zero moments: mhat = g, vhat = g^2, so p moves by lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = cnn.adam(np.ones(3), g, np.zeros(3), np.zeros(3), 0.01, 0.9, 0.999, 1e-12, 1)
    np.testing.assert_allclose(p, 1.0 - 0.01 * np.sign(g), rtol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g ** 2)
    # a second step with the same gradient: mhat = g, vhat = g^2 again
    p2, _, _ = cnn.adam(p, g, m, v, 0.01, 0.9, 0.999, 1e-12, 2)
    np.testing.assert_allclose(p2, 1.0 - 0.02 * np.sign(g), rtol=1e-9)


def test_prep_by_hand():
    im = np.arange(16, dtype=np.float64).reshape(1, 4, 4)
    got = cnn.prep(im, 0.5)
    means = np.array([[2.5, 4.5], [10.5, 12.5]])
    np.testing.assert_allclose(got[0], np.arcsinh(0.5 * means))
    assert math.isclose(float(np.arcsinh(0.5 * -3.0)), -float(np.arcsinh(1.5)))
