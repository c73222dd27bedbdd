"""FP64 reference of the learned right preconditioner (oracle).

Test infrastructure only (see ``oracle/__init__``).

The paper preconditions GMRES with a block-circulant approximation (Sec. 5.4);
the learned preconditioner is this project's addition: a small 3-D
convolutional network z = Net(v, chi) used as the right preconditioner of
flexible GMRES.  The network (our reading of "4 levels, 32 channels, 3x3x3"):

* input 8 channels: re/im of the three current components of v, re/im of chi;
  output 6 channels: re/im of the three components of z;
* encoder level l = 0..3: h_l = relu(conv(a_l)), a_0 = input,
  a_l = pool(h_{l-1}) (average over 2 x 2 in x and y, ceil sizes, z kept);
* decoder l = 2..0: u_l = relu(conv(up(u_{l+1}) + h_l)), u_3 = h_3,
  up = nearest-neighbour repetition cropped to the finer size;
* output z = conv(u_0) (no activation);
* every conv is 3x3x3 with zero padding and a bias; 32 channels inside.

Tensors are (C, nz, ny, nx).  Weights W[o, c, dz, dy, dx], biases b[o].
Everything here is a plain definition: convolution by an explicit loop over
the 27 taps, pooling and nearest upsampling by reshaping, backward passes by
the chain rule written out.  Pins (tests/test_oracle_convnet.py): central
finite differences of the loss in every weight tensor and in the input.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # (name, c_in, c_out)
    ("enc0", 8, 32), ("enc1", 32, 32), ("enc2", 32, 32), ("enc3", 32, 32),
    ("dec2", 32, 32), ("dec1", 32, 32), ("dec0", 32, 32), ("out", 32, 6),
]


def init_params(seed: int, scale: float = 1.0) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for name, ci, co in LAYERS:
        std = scale * np.sqrt(2.0 / (27 * ci))
        p[name + ".w"] = rng.standard_normal((co, ci, 3, 3, 3)) * std
        p[name + ".b"] = rng.standard_normal(co) * 0.01
    return p


def conv3d(x, w, b):
    """y[o] = b[o] + sum_c sum_taps w[o, c, t] x[c, shifted by t - 1] (zero padding)."""
    ci, nz, ny, nx = x.shape
    xp = np.zeros((ci, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], nz, ny, nx)) + b[:, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                y += np.einsum("oc,czyx->ozyx", w[:, :, dz, dy, dx],
                               xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx])
    return y


def conv3d_backward(x, w, dy):
    """Gradients (dx, dw, db) of conv3d for the output gradient dy."""
    ci, nz, ny, nx = x.shape
    xp = np.zeros((ci, nz + 2, ny + 2, nx + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dz in range(3):
        for dy_ in range(3):
            for dx_ in range(3):
                sl = (slice(None), slice(dz, dz + nz), slice(dy_, dy_ + ny), slice(dx_, dx_ + nx))
                dw[:, :, dz, dy_, dx_] = np.einsum("ozyx,czyx->oc", dy, xp[sl])
                dxp[sl] += np.einsum("oc,ozyx->czyx", w[:, :, dz, dy_, dx_], dy)
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, dy.sum(axis=(1, 2, 3))


def pool(x):
    """Average over 2 x 2 blocks in (y, x); a trailing odd row/column averages
    the entries that exist."""
    c, nz, ny, nx = x.shape
    my, mx = (ny + 1) // 2, (nx + 1) // 2
    out = np.zeros((c, nz, my, mx))
    cnt = np.zeros((my, mx))
    for oy in range(2):
        for ox in range(2):
            sub = x[:, :, oy::2, ox::2]
            out[:, :, :sub.shape[2], :sub.shape[3]] += sub
            cnt[:sub.shape[2], :sub.shape[3]] += 1
    return out / cnt


def pool_backward(dout, shape):
    c, nz, ny, nx = shape
    my, mx = dout.shape[2], dout.shape[3]
    cnt = np.zeros((my, mx))
    for oy in range(2):
        for ox in range(2):
            cnt[:len(range(oy, ny, 2)), :len(range(ox, nx, 2))] += 1
    g = dout / cnt
    dx = np.zeros(shape)
    for oy in range(2):
        for ox in range(2):
            sy, sx = len(range(oy, ny, 2)), len(range(ox, nx, 2))
            dx[:, :, oy::2, ox::2] = g[:, :, :sy, :sx]
    return dx


def up(x, ny, nx):
    """Nearest-neighbour: out[..., y, x] = x[..., y // 2, x // 2]."""
    return x[:, :, np.arange(ny) // 2][:, :, :, np.arange(nx) // 2]


def up_backward(dout, coarse_shape):
    c, nz, my, mx = coarse_shape
    d = np.zeros(coarse_shape)
    ny, nx = dout.shape[2], dout.shape[3]
    for y in range(ny):
        for x in range(nx):
            d[:, :, y // 2, x // 2] += dout[:, :, y, x]
    return d


def relu(x):
    return np.maximum(x, 0.0)


def forward(p, x, keep=False):
    """Net(x) in FP64; with keep=True also returns the intermediate tensors."""
    cache = {"x": x}
    a = x
    hs = []
    for lvl in range(4):
        if lvl > 0:
            a = pool(hs[-1])
            cache[f"a{lvl}"] = a
        z = conv3d(a, p[f"enc{lvl}.w"], p[f"enc{lvl}.b"])
        h = relu(z)
        cache[f"encz{lvl}"] = z
        hs.append(h)
    u = hs[3]
    for lvl in (2, 1, 0):
        s = up(u, hs[lvl].shape[2], hs[lvl].shape[3]) + hs[lvl]
        z = conv3d(s, p[f"dec{lvl}.w"], p[f"dec{lvl}.b"])
        cache[f"decin{lvl}"] = s
        cache[f"decz{lvl}"] = z
        u = relu(z)
        cache[f"u{lvl}"] = u
    y = conv3d(u, p["out.w"], p["out.b"])
    cache["hs"] = hs
    return (y, cache) if keep else y


def backward(p, cache, dy):
    """Gradients of sum(dy * Net(x)) in every parameter and in x."""
    g = {}
    hs = cache["hs"]
    du, g["out.w"], g["out.b"] = conv3d_backward(cache["u0"], p["out.w"], dy)
    dh = [np.zeros_like(h) for h in hs]
    for lvl in (0, 1, 2):
        dz = du * (cache[f"decz{lvl}"] > 0)
        ds, g[f"dec{lvl}.w"], g[f"dec{lvl}.b"] = conv3d_backward(cache[f"decin{lvl}"], p[f"dec{lvl}.w"], dz)
        dh[lvl] += ds
        coarse = hs[3].shape if lvl == 2 else cache[f"u{lvl + 1}"].shape
        du = up_backward(ds, coarse)
    dh[3] += du
    dx = None
    for lvl in (3, 2, 1, 0):
        dz = dh[lvl] * (cache[f"encz{lvl}"] > 0)
        a = cache["x"] if lvl == 0 else cache[f"a{lvl}"]
        da, g[f"enc{lvl}.w"], g[f"enc{lvl}.b"] = conv3d_backward(a, p[f"enc{lvl}.w"], dz)
        if lvl > 0:
            dh[lvl - 1] += pool_backward(da, hs[lvl - 1].shape)
        else:
            dx = da
    return g, dx


def relative_mse(y, e):
    """Loss sum |y - e|^2 / sum |e|^2 and its gradient in y."""
    den = np.sum(e * e)
    r = y - e
    return float(np.sum(r * r) / den), 2.0 * r / den


def pack_input(v, chi):
    """(3, nz, ny, nx) complex current and (nz, ny, nx) complex chi -> 8 channels."""
    return np.concatenate([v.real, v.imag, chi.real[None], chi.imag[None]], axis=0)


def unpack_output(y):
    """6 channels -> (3, nz, ny, nx) complex."""
    return y[:3] + 1j * y[3:6]
