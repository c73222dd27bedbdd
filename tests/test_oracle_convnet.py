"""Pins for oracle.convnet: central finite differences of a scalar loss in
every parameter tensor and in the input (sampled entries), pooling and
upsampling against hand-written cases."""
import numpy as np
import pytest

from oracle import convnet as cn


def _small_params(seed=0, width=4):
    # same structure, fewer channels, so the check stays fast
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in cn.LAYERS:
        ci = 8 if name == "enc0" else width
        co = 6 if name == "out" else width
        p[name + ".w"] = rng.standard_normal((co, ci, 3, 3, 3)) * 0.3
        p[name + ".b"] = rng.standard_normal(co) * 0.1
    return p


def test_pool_and_up_definitions():
    x = np.arange(2 * 1 * 3 * 5, dtype=float).reshape(2, 1, 3, 5)
    y = cn.pool(x)
    assert y.shape == (2, 1, 2, 3)
    assert y[0, 0, 0, 0] == np.mean(x[0, 0, 0:2, 0:2])
    assert y[0, 0, 1, 2] == x[0, 0, 2, 4]                 # corner cell: one input
    assert y[1, 0, 0, 2] == np.mean(x[1, 0, 0:2, 4])      # edge cell: two inputs
    u = cn.up(y, 3, 5)
    assert u.shape == x.shape and u[0, 0, 2, 3] == y[0, 0, 1, 1]


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    y = cn.conv3d(x, w, b)
    o, z, yy, xx = 1, 0, 4, 2      # a boundary voxel
    s = b[o]
    for c in range(3):
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    zz, y2, x2 = z + dz - 1, yy + dy - 1, xx + dx - 1
                    if 0 <= zz < 4 and 0 <= y2 < 5 and 0 <= x2 < 6:
                        s += w[o, c, dz, dy, dx] * x[c, zz, y2, x2]
    assert abs(y[o, z, yy, xx] - s) < 1e-12


@pytest.mark.parametrize("shape", [(3, 7, 9), (2, 5, 6)])
def test_gradients_by_finite_differences(shape):
    rng = np.random.default_rng(2)
    p = _small_params()
    nz, ny, nx = shape
    x = rng.standard_normal((8, nz, ny, nx))
    e = rng.standard_normal((6, nz, ny, nx))

    def loss(params, xin):
        y = cn.forward(params, xin)
        return cn.relative_mse(y, e)[0]

    y, cache = cn.forward(p, x, keep=True)
    _, dy = cn.relative_mse(y, e)
    g, dx = cn.backward(p, cache, dy)
    h = 1e-6
    for name in p:
        flat = p[name].ravel()
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = loss(p, x)
            flat[idx] = old - h
            lm = loss(p, x)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)
    xf = x.ravel()
    for idx in rng.choice(xf.size, size=6, replace=False):
        old = xf[idx]
        xf[idx] = old + h
        lp = loss(p, x)
        xf[idx] = old - h
        lm = loss(p, x)
        xf[idx] = old
        assert abs((lp - lm) / (2 * h) - dx.ravel()[idx]) <= 1e-6 * max(1.0, abs(dx.ravel()[idx]))
