"""Shared helpers for the GPU parity tests (oracle side computed on the CPU)."""
import numpy as np

from oracle import greens
from oracle import operator as op


def oracle_matvec(grid, kappa, M, x, mode="operator"):
    Gh = op.green_spectrum(greens.octant_table(kappa, grid), grid, tuple(2 * v for v in grid))
    if mode == "operator":
        return op.matvec(Gh, grid, M, x)
    return op.rhs_from_source(Gh, grid, M, x)


def oracle_sparse_apply(kappa, grid, M, x, out_idx):
    """y[out_idx] of y = x - M (T x) for a sparse x, each output summed
    directly over the non-zeros of x (no FFT)."""
    nx, ny, nz = grid
    N = nx * ny * nz
    xf = np.asarray(x).ravel()
    nzj = np.flatnonzero(xf)
    qj, vj = nzj // N, nzj % N
    zj, yj, xj = vj // (nx * ny), (vj // nx) % ny, vj % nx
    pi, vi = out_idx // N, out_idx % N
    zi, yi, xi = vi // (nx * ny), (vi // nx) % ny, vi % nx
    D = np.stack([xi[:, None] - xj[None, :], yi[:, None] - yj[None, :], zi[:, None] - zj[None, :]], -1)
    uniq, inv = np.unique(D.reshape(-1, 3), axis=0, return_inverse=True)
    T = greens.toeplitz_entries(kappa, uniq)[inv.ravel()].reshape(len(out_idx), len(nzj), 6)
    comp = np.array([[greens.comp_index(p, q) for q in range(3)] for p in range(3)])
    c = comp[pi[:, None], qj[None, :]]
    Tsel = np.take_along_axis(T, c[..., None], axis=2)[..., 0]
    u = Tsel @ xf[nzj]
    return xf[out_idx] - np.asarray(M).ravel()[vi] * u


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
