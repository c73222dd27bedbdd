"""Field on the centre axis and reflection coefficient R (oracle; FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper (arXiv:1803.06237):
* Sec. 3, equivalent currents: J = c_e (eps_r - 1) E, so inside the scatterer
  E = J / (c_e chi) with chi = eps_r - 1 (relative to the background).  With the
  Galerkin weights w_i = <J, P_i> and J constant per voxel, E_i is
  w_i / (c_e chi_i h^{3/2}); the common factor c_e h^{3/2} cancels in R and is
  dropped.
* Sec. 5.1: R = ||E_inf - E_L||^2 / ||E_inf||^2, the L2 norm taken along the
  centre axis over 0 <= x <= X (the waveguide before the absorber).  On the
  voxel grid the integral over x is the sum over axis voxels with centre
  x_c < X (the voxel length is common to both norms and cancels).

Reading: the axis is the voxel row at (ny // 2, nz // 2); all three field
components enter the norm.

The transmission through a plane (Sec. 5.2), T = sum |E|^2 over the plane's
voxels inside the structure (chi != 0), with the same E.

Pins (tests/test_oracle_metrics.py): R = 0 for identical fields, R = 1 for a
zero field, R = |r|^2 for a mode plus a reflected wave r exp(+j beta x) over
whole half-periods, R = |1 - a exp(j phi)|^2 for a scaled and phase-shifted
field; the GPU solves' R is compared with R from oracle solves
(tests/test_gpu_reflection.py).
"""
from __future__ import annotations

import numpy as np


def axis_field(w: np.ndarray, chi: np.ndarray, n_x_keep: int) -> np.ndarray:
    """E (up to c_e h^{3/2}) on the centre axis for ix < n_x_keep, shape (3, n_x_keep)."""
    nz, ny, nx = chi.shape
    w = np.asarray(w).reshape(3, nz, ny, nx)
    yc, zc = ny // 2, nz // 2
    return w[:, zc, yc, :n_x_keep] / chi[zc, yc, :n_x_keep][None, :]


def reflection_coefficient(E_ref: np.ndarray, E_L: np.ndarray) -> float:
    """R = sum |E_ref - E_L|^2 / sum |E_ref|^2 (Sec. 5.1)."""
    E_ref = np.asarray(E_ref)
    E_L = np.asarray(E_L)
    return float(np.sum(np.abs(E_ref - E_L) ** 2) / np.sum(np.abs(E_ref) ** 2))


def slice_power(w: np.ndarray, chi: np.ndarray, ix: int) -> float:
    """Transmission through the voxel plane ix (Sec. 5.2): sum of |E|^2 over
    the plane's voxels with chi != 0, E = w / chi (up to c_e h^{3/2})."""
    nz, ny, nx = chi.shape
    w = np.asarray(w).reshape(3, nz, ny, nx)[:, :, :, ix]
    c = chi[:, :, ix]
    inside = c != 0
    return float(np.sum(np.abs(w[:, inside] / c[inside][None]) ** 2))
