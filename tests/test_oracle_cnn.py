"""Pins of the FP64 reference network (oracle/cnn.py): the convolution equals a
brute-force loop, the analytic gradient of the weighted BCE equals central
finite differences, and the output, loss and bias gradient take their closed
forms for weights with a known response (zero filters; one pixel passed
through centre-tap filters and the max pool)."""
import numpy as np

import synthetic
from oracle import cnn


def test_conv_matches_brute_force_loop():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 7))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    for stride in (1, 2):
        out = cnn.conv(x, W, b, stride)
        To = (7 - 1) // stride + 1
        ref = np.zeros((3, To, To))
        for o in range(3):
            for i in range(To):
                for j in range(To):
                    s = b[o]
                    for c in range(2):
                        for di in range(3):
                            for dj in range(3):
                                ii, jj = stride * i + di - 1, stride * j + dj - 1
                                if 0 <= ii < 7 and 0 <= jj < 7:
                                    s += W[o, c, di, dj] * x[c, ii, jj]
                    ref[o, i, j] = s
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12)


def test_gradient_matches_central_differences():
    theta = synthetic.cnn_init_params(cnn.SHAPES, seed=3)
    assert theta.size == cnn.NPARAM
    rng = np.random.default_rng(1)
    T = 9
    xs = [rng.standard_normal((2, T, T)) for _ in range(3)]
    ys = [1.0, 0.0, 1.0]
    theta = theta + 0.05 * rng.standard_normal(theta.size)  # nonzero biases
    L, g = cnn.loss_and_grad(theta, xs, ys, w_pos=4.0)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (cnn.loss_and_grad(tp, xs, ys, 4.0)[0] - cnn.loss_and_grad(tm, xs, ys, 4.0)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_output_and_loss_closed_forms():
    # all weights zero but the output bias b: p = 1 / (1 + e^-b) for any input,
    # and the batch loss is the mean of -(w_pos y log p + (1 - y) log(1 - p))
    theta = np.zeros(cnn.NPARAM)
    b = 0.7
    theta[-1] = b
    rng = np.random.default_rng(2)
    xs = [rng.standard_normal((2, 9, 9)) for _ in range(4)]
    ys = [1.0, 0.0, 0.0, 1.0]
    p = 1.0 / (1.0 + np.exp(-b))
    for x in xs:
        assert cnn.forward(theta, x)[0] == p
    L, g = cnn.loss_and_grad(theta, xs, ys, w_pos=3.0)
    assert abs(L - np.mean([-(3.0 * y * np.log(p) + (1 - y) * np.log(1 - p)) for y in ys])) < 1e-15
    # d L / d b = mean(w_pos y (p - 1) + (1 - y) p); every other gradient is zero
    assert abs(g[-1] - np.mean([3.0 * y * (p - 1) + (1 - y) * p for y in ys])) < 1e-15
    assert np.all(g[:-1] == 0.0)
    # one positive channel-0 pixel through identity-like filters reaches the max pool
    W1, b1, W2, b2, W3, b3, wl, bl = cnn.unpack(np.zeros(cnn.NPARAM))
    W1[0, 0, 1, 1] = W2[0, 0, 1, 1] = W3[0, 0, 1, 1] = 1.0
    wl[0] = 1.0
    x = np.zeros((2, 9, 9))
    x[0, 4, 4] = 2.5  # even index: survives both stride-2 layers (4 -> 2 -> 1)
    assert abs(cnn.forward(cnn.pack([W1, b1, W2, b2, W3, b3, wl, bl]), x)[0] - 1.0 / (1.0 + np.exp(-2.5))) < 1e-15
