"""Pins of the FP64 reference network (oracle/cnn.py): the convolution equals a
brute-force loop, and the analytic gradient of the weighted BCE equals central
finite differences."""
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
