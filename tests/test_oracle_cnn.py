"""Pins of the oracle's convolutions and preconditioner network."""
import numpy as np
import pytest

from oracle import cnn


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3d_equals_direct_loops():
    r = rng(1)
    x = r.standard_normal((3, 4, 3, 5))
    w = r.standard_normal((2, 3, 3, 3, 3))
    b = r.standard_normal(2)
    y = cnn.conv3d(x, w, b)
    C, Z, Y, X = x.shape
    for o in range(2):
        for z in range(Z):
            for yy in range(Y):
                for xx in range(X):
                    s = b[o]
                    for i in range(C):
                        for dz in range(3):
                            for dy in range(3):
                                for dx in range(3):
                                    zz, y2, x2 = z + dz - 1, yy + dy - 1, xx + dx - 1
                                    if 0 <= zz < Z and 0 <= y2 < Y and 0 <= x2 < X:
                                        s += w[o, i, dz, dy, dx] * x[i, zz, y2, x2]
                    assert y[o, z, yy, xx] == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_identity_and_shift_kernels():
    x = rng(2).standard_normal((3, 5, 4, 6))
    w = np.zeros((3, 3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1, 1] = 1.0
    assert np.array_equal(cnn.conv3d(x, w), x)
    w = np.zeros((3, 3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1, 2] = 1.0          # reads x + 1: shift left, zero at the end
    y = cnn.conv3d(x, w)
    assert np.array_equal(y[..., :-1], x[..., 1:]) and np.all(y[..., -1] == 0)


def test_pool_and_upsample_adjoints():
    r = rng(3)
    a = r.standard_normal((2, 4, 6, 8))
    b = r.standard_normal((2, 2, 3, 4))
    assert np.sum(cnn.avgpool2(a) * b) == pytest.approx(np.sum(a * cnn.avgpool2_backward(b)))
    assert np.sum(cnn.up2(b) * a) == pytest.approx(np.sum(b * cnn.up2_backward(a)))
    assert np.allclose(cnn.avgpool2(cnn.up2(b)), b)


def test_conv3d_backward_finite_differences():
    r = rng(4)
    x = r.standard_normal((2, 3, 4, 3))
    w = r.standard_normal((3, 2, 3, 3, 3))
    b = r.standard_normal(3)
    gy = r.standard_normal((3, 3, 4, 3))
    f = lambda x_, w_, b_: float(np.sum(cnn.conv3d(x_, w_, b_) * gy))
    gx, gw, gb = cnn.conv3d_backward(x, w, gy)
    h = 1e-6
    for idx in [(0, 1, 2, 1), (1, 0, 0, 2), (1, 2, 3, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert (f(xp, w, b) - f(xm, w, b)) / (2 * h) == pytest.approx(gx[idx], rel=1e-6)
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 2, 0), (1, 1, 2, 2, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert (f(x, wp, b) - f(x, wm, b)) / (2 * h) == pytest.approx(gw[idx], rel=1e-6)
    assert gb == pytest.approx(gy.sum(axis=(1, 2, 3)))


def test_network_gradient_finite_differences():
    ch = (2, 3, 3, 2)
    params = cnn.init_params(5, ch=ch)
    r = rng(6)
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.1 * r.standard_normal(params[k].shape)
    x = r.standard_normal((cnn.IN_CH, 8, 8, 8))
    target = r.standard_normal((cnn.OUT_CH, 8, 8, 8))

    def loss(p):
        out, _ = cnn.forward(p, x)
        return cnn.relative_loss(out, target)[0]

    out, cache = cnn.forward(params, x)
    L, gout = cnn.relative_loss(out, target)
    grads, _ = cnn.backward(params, cache, gout)
    h = 1e-6
    for key, idx in [("e0a.w", (1, 2, 0, 1, 2)), ("e2b.w", (0, 1, 1, 1, 1)),
                     ("e3a.w", (1, 0, 2, 0, 1)), ("d2a.w", (2, 4, 1, 2, 0)),
                     ("d0a.w", (0, 3, 1, 1, 1)), ("out.w", (2, 1, 0, 0, 0)),
                     ("d1b.b", (1,)), ("out.b", (0,))]:
        pp = {k: v.copy() for k, v in params.items()}
        pm = {k: v.copy() for k, v in params.items()}
        pp[key][idx] += h
        pm[key][idx] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert fd == pytest.approx(grads[key][idx], rel=1e-5, abs=1e-9), key
