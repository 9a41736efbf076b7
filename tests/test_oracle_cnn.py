"""Pins of the oracle's U-Net: gradients against central finite differences in
float64, the parameter count, and the pooling / upsampling adjoints."""
import numpy as np

from oracle import cnn

C_SMALL = (2, 3, 4, 5)


def test_param_count_default():
    # the solver's default net: about 2e5 parameters
    n = cnn.num_params(3, 8)
    assert 150_000 < n < 250_000


def test_pool_up_adjoints():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 8, 6))
    y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(cnn.pool(x) * y), np.sum(x * cnn.pool_backward(y)))
    z = rng.standard_normal((2, 3, 16, 12))
    assert np.isclose(np.sum(cnn.up(x) * z), np.sum(x * cnn.up_backward(z)))


def test_conv_matches_direct_loops():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 5, 4))
    W = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    y = cnn.conv(x, W, b)
    ref = np.zeros_like(y)
    for o in range(3):
        for i in range(5):
            for j in range(4):
                s = b[o]
                for c in range(2):
                    for dy in range(3):
                        for dx in range(3):
                            ii, jj = i + dy - 1, j + dx - 1
                            if 0 <= ii < 5 and 0 <= jj < 4:
                                s += W[o, c, dy, dx] * x[0, c, ii, jj]
                ref[0, o, i, j] = s
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_gradient_central_differences():
    rng = np.random.default_rng(2)
    n = cnn.num_params(3, 2, C_SMALL)
    theta = rng.standard_normal(n) * 0.3
    x = rng.standard_normal((2, 3, 16, 8))
    t = rng.standard_normal((2, 2, 16, 8))
    loss, g = cnn.loss_and_grad(theta, x, t, C_SMALL)
    h = 1e-6
    idx = rng.choice(n, 40, replace=False)
    for k in idx:
        e = np.zeros(n)
        e[k] = h
        lp, _ = cnn.loss_and_grad(theta + e, x, t, C_SMALL)
        lm, _ = cnn.loss_and_grad(theta - e, x, t, C_SMALL)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-4), (k, fd, g[k])


def test_adam_decreases_loss():
    rng = np.random.default_rng(3)
    n = cnn.num_params(3, 2, C_SMALL)
    theta = rng.standard_normal(n) * 0.3
    x = rng.standard_normal((2, 3, 16, 8))
    t = np.tanh(x[:, :2])
    m = np.zeros(n)
    v = np.zeros(n)
    l0 = None
    for it in range(1, 60):
        loss, g = cnn.loss_and_grad(theta, x, t, C_SMALL)
        l0 = loss if l0 is None else l0
        theta, m, v = cnn.adam_step(theta, g, m, v, it, lr=1e-2)
    assert loss < 0.5 * l0
