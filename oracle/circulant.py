"""Block-circulant preconditioner of the discrete J-VIE (oracle; FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper (arXiv:1803.06237), Sec. 5.4: a block-circulant matrix W closest to
A = I - M_eps N in the Frobenius norm (after Chan and Olkin), inverted with
FFTs, preconditions GMRES.  The paper leaves the details to a later article;
the reading used here:

* the circulant approximation is taken on the x level only (the long axis
  of a waveguide): view A as an nx x nx array of blocks A[i][j] of size
  (3 ny nz)^2, A[i][j][(p,z,y),(q,z',y')] = delta - M(z,y,i) T_pq(i - j, y - y', z - z');
* W = circ(c_0, ..., c_{nx-1}) with the Frobenius-optimal blocks
  c_k = (1/nx) sum_i A[i][(i - k) mod nx]  (the average of the k-th wrapped
  block diagonal); for a contrast that does not depend on x this is T.
  Chan's optimal circulant c_k = ((nx - k) t_k + k t_{k - nx}) / nx;
* W is block-diagonalised by the DFT along x:
  W_hat(w) = sum_k c_k exp(-2 pi i w k / nx), and W^{-1} v is a DFT along x,
  one dense (3 ny nz) solve per frequency, and the inverse DFT;
* it is applied as a right preconditioner of (flexible) GMRES, A W^{-1} u = b,
  x = W^{-1} u (the paper writes the left form W^{-1} A; the two
  preconditioned matrices are similar).

Within a block, unknowns are ordered (p, z, y) with y fastest.  Vectors are
(3, nz, ny, nx) complex128 as elsewhere in the oracle.

Pins (tests/test_oracle_circulant.py): the blocks against a brute-force
average of the wrapped block diagonals of the dense A (``operator.dense_A``);
the first-order optimality condition (A - W is orthogonal to every
block-circulant matrix); T. Chan's closed form for a contrast constant in x;
nx = 1 gives W = A; W^{-1} (W v) = v with W assembled densely.
"""
from __future__ import annotations

import numpy as np

from . import greens


def _offsets_table(n, kappa: float):
    """T_pq(dx, dy, dz) for dx in (-nx, nx), dy in (-ny, ny), dz in (-nz, nz):
    array (6, 2nz-1, 2ny-1, 2nx-1), index d + n - 1 on each axis."""
    nx, ny, nz = (int(v) for v in n)
    zz, yy, xx = np.meshgrid(np.arange(-nz + 1, nz), np.arange(-ny + 1, ny), np.arange(-nx + 1, nx), indexing="ij")
    offs = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    vals = greens.toeplitz_entries(kappa, offs)
    return vals.T.reshape(6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1)


def x_block(Tfull: np.ndarray, n, dx: int) -> np.ndarray:
    """The (3 ny nz)^2 block T(dx): rows (p, z, y), columns (q, z', y'),
    entry T_pq(dx, y - y', z - z')."""
    nx, ny, nz = (int(v) for v in n)
    B = ny * nz
    z = np.repeat(np.arange(nz), ny)
    y = np.tile(np.arange(ny), nz)
    iz = (z[:, None] - z[None, :]) + nz - 1
    iy = (y[:, None] - y[None, :]) + ny - 1
    out = np.zeros((3 * B, 3 * B), dtype=np.complex128)
    for p in range(3):
        for q in range(3):
            c = greens.comp_index(p, q)
            out[p * B:(p + 1) * B, q * B:(q + 1) * B] = Tfull[c, iz, iy, dx + nx - 1]
    return out


def circulant_blocks(n, kappa: float, Mvox: np.ndarray, Tfull: np.ndarray | None = None) -> np.ndarray:
    """c_k, k = 0 .. nx-1, shape (nx, 3B, 3B): the averages of the wrapped
    block diagonals of A = I - diag(M) T (B = ny nz).  For k > 0 the
    diagonal holds A[i][i-k] = -M_i T(k) for i >= k and A[i][i-k+nx] =
    -M_i T(k-nx) for i < k; so c_k = delta_k0 I - S_k^+ T(k) - S_k^- T(k-nx)
    with the row scalings S_k^+ = (1/nx) sum_{i>=k} M_i, S_k^- = (1/nx) sum_{i<k} M_i."""
    nx, ny, nz = (int(v) for v in n)
    B = ny * nz
    if Tfull is None:
        Tfull = _offsets_table(n, kappa)
    M = np.asarray(Mvox, dtype=np.complex128).reshape(nz, ny, nx)
    Mx = M.reshape(B, nx)                      # rows (z, y), columns x
    c = np.zeros((nx, 3 * B, 3 * B), dtype=np.complex128)
    for k in range(nx):
        s_plus = np.tile(Mx[:, k:].sum(axis=1), 3) / nx
        s_minus = np.tile(Mx[:, :k].sum(axis=1), 3) / nx
        blk = -s_plus[:, None] * x_block(Tfull, n, k)
        if k > 0:
            blk -= s_minus[:, None] * x_block(Tfull, n, k - nx)
        else:
            blk += np.eye(3 * B)
        c[k] = blk
    return c


def blocks_hat(c: np.ndarray) -> np.ndarray:
    """W_hat(w) = sum_k c_k exp(-2 pi i w k / nx), shape (nx, 3B, 3B)."""
    return np.fft.fft(c, axis=0)


def to_blocks(v: np.ndarray) -> np.ndarray:
    """(3, nz, ny, nx) -> (nx, 3B) with the in-block order (p, z, y)."""
    nx = v.shape[3]
    return v.reshape(-1, nx).T.copy()


def from_blocks(u: np.ndarray, n) -> np.ndarray:
    nx, ny, nz = (int(v) for v in n)
    return u.T.reshape(3, nz, ny, nx)


def apply_inverse(What: np.ndarray, v: np.ndarray) -> np.ndarray:
    """z = W^{-1} v: DFT along x, one dense solve per frequency, inverse DFT."""
    n = (v.shape[3], v.shape[2], v.shape[1])
    vh = np.fft.fft(to_blocks(v), axis=0)
    zh = np.linalg.solve(What, vh[:, :, None])[:, :, 0]
    return from_blocks(np.fft.ifft(zh, axis=0), n)


def apply_W(c: np.ndarray, v: np.ndarray) -> np.ndarray:
    """W v = sum_j c_{(i-j) mod nx} v_j (block circular convolution), directly."""
    n = (v.shape[3], v.shape[2], v.shape[1])
    nx = n[0]
    vb = to_blocks(v)
    out = np.zeros_like(vb)
    for i in range(nx):
        for j in range(nx):
            out[i] += c[(i - j) % nx] @ vb[j]
    return from_blocks(out, n)
