"""Discrete J-VIE operator, contrast, absorber and right-hand side (oracle; FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper (arXiv:1803.06237):
* Sec. 3, boxed J-VIE: (I - M_eps N) J = c_e M_eps E_inc with
  M_eps = (eps_r - 1) / eps_r; discrete form Sec. 3.1:
  (I - M_eps N) w_e = c_e M_eps e_inc.
* Sec. 3.1: material constant per voxel (value at the voxel centre), pulled out
  of the inner products, so A = I - diag(M) T with the Toeplitz T of
  ``oracle.greens``.
* Sec. 5.4: the block-Toeplitz N is applied with FFTs (circulant embedding).
* Sec. 2: a background eps_bg is scaled out (eps -> eps / eps_bg, k0 -> k0 sqrt(eps_bg)).
* Sec. 4.1: sigma(x) = sigma_0 s(x / L), s(u) = u^d for 0 <= u <= 1, d = 0..3.
* Sec. 4.2: eps_r = eps' - j eps'' inside the absorber.  Reading: eps'' = sigma / (w eps_0)
  (the only reading consistent with the round-trip formula of Sec. 4.3); the
  absorber is applied to core voxels (eps' != eps_bg) only.
* Sec. 4.3: sigma_0 from a target round-trip reflection R_rt.

Layout: a current vector is w[c][z][y][x] (x fastest), shape (3, nz, ny, nx),
complex128.  Grids are given as n = (nx, ny, nz).

Pins (tests/test_oracle_operator.py): dense per-pair assembly vs FFT matvec on
1x1x1, 2x3x5 and 4^3 grids (brute force, no parity used by the dense side),
chi = 0 gives A = I exactly, complex symmetry of the dense matrix
(reciprocity), -Im(T) positive semidefinite (radiated power), the absorber
profile against hand-evaluated monomials and the round-trip closed form.
tests/test_oracle_physics.py: the right-hand side b = M((T - I) w_src)
against a direct quadrature of the closed-form dyadic Green function away
from the source and against the static depolarisation (-1/3) of a uniformly
polarised cube in the source voxel; -Im(T) against the far-field
(plane-wave) expansion of the radiated power; a voxelised sphere at k0 a = 1
against the Mie series (lossy and lossless, error shrinking with h); energy
balance (extinction = radiated power) in the lossless case.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

from . import greens


# ----------------------------------------------------------------------------
# contrast (step a1)
# ----------------------------------------------------------------------------
def absorber_eps2(nx: int, x0: float, length: float, degree: int, eps2_max: float,
                  direction: int = +1) -> np.ndarray:
    """eps''(x) at voxel centres x_c = ix + 1/2 (units of h): eps2_max * u^d
    with u = (x_c - x0) / L (direction +1) or (x0 - x_c) / L (direction -1),
    zero where u < 0 or u > 1 (Sec. 4.1 profile)."""
    xc = np.arange(nx) + 0.5
    u = (xc - x0) / length if direction > 0 else (x0 - xc) / length
    prof = np.zeros(nx)
    inside = (u >= 0.0) & (u <= 1.0)
    prof[inside] = eps2_max * u[inside] ** degree
    return prof


def chi_from_permittivity(eps: np.ndarray, eps_bg: float, absorbers=()) -> np.ndarray:
    """chi = eps / eps_bg - 1 per voxel; each absorber (dict with keys x0,
    length, degree, eps2_max, direction) subtracts j eps'' on voxels whose
    eps differs from eps_bg.  ``eps`` has shape (nz, ny, nx)."""
    eps = np.asarray(eps, dtype=np.complex128).copy()
    nx = eps.shape[-1]
    core = np.abs(eps - eps_bg) > 0
    for ab in absorbers:
        e2 = absorber_eps2(nx, ab["x0"], ab["length"], ab["degree"], ab["eps2_max"],
                           ab.get("direction", +1))
        eps = eps - 1j * core * e2[None, None, :]
    return eps / eps_bg - 1.0


def contrast_M(chi: np.ndarray) -> np.ndarray:
    """M = chi / (1 + chi) = (eps_r - 1) / eps_r (Sec. 3, M_eps)."""
    chi = np.asarray(chi, dtype=np.complex128)
    return chi / (1.0 + chi)


def eps2_max_from_rrt(r_rt: float, degree: int, length_um: float, k0_per_um: float,
                      eps_r: float, D: float = 2.0, eta: float = 1.0) -> float:
    """eps''_max = sigma_0 / (w eps_0) for a target round-trip reflection
    (Sec. 4.3 closed form with p = d):
    sigma_0 = -(d+1) ln(R_rt) / (D L eta) sqrt(eps_0 eps_r / mu_0), and
    k0 = w sqrt(eps_0 mu_0) give eps''_max = -(d+1) ln(R_rt) sqrt(eps_r) / (D L eta k0)."""
    return -(degree + 1) * math.log(r_rt) * math.sqrt(eps_r) / (D * length_um * eta * k0_per_um)


# ----------------------------------------------------------------------------
# dense assembly (tiny grids; brute force)
# ----------------------------------------------------------------------------
def voxel_coords(n) -> np.ndarray:
    """Integer voxel coordinates (x, y, z) in the flat order z-slowest, x-fastest."""
    nx, ny, nz = (int(v) for v in n)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def dense_T(n, kappa: float) -> np.ndarray:
    """(3N x 3N) matrix T[(p,i),(q,j)] = T_pq(r_i - r_j), every pair offset
    evaluated directly (negative offsets included, no parity used)."""
    X = voxel_coords(n)
    N = X.shape[0]
    diffs = (X[:, None, :] - X[None, :, :]).reshape(-1, 3)
    uniq, inv = np.unique(diffs, axis=0, return_inverse=True)
    vals = greens.toeplitz_entries(kappa, uniq)[inv.ravel()].reshape(N, N, 6)
    T = np.zeros((3 * N, 3 * N), dtype=np.complex128)
    for p in range(3):
        for q in range(3):
            T[p * N:(p + 1) * N, q * N:(q + 1) * N] = vals[:, :, greens.comp_index(p, q)]
    return T


def dense_A(n, kappa: float, Mvox: np.ndarray) -> np.ndarray:
    """A = I - diag(M) T (Sec. 3.1 discrete J-VIE), M repeated for 3 components."""
    T = dense_T(n, kappa)
    m = np.tile(np.asarray(Mvox, dtype=np.complex128).ravel(), 3)
    return np.eye(T.shape[0], dtype=np.complex128) - m[:, None] * T


# ----------------------------------------------------------------------------
# FFT matvec via circulant embedding (steps a3-a6)
# ----------------------------------------------------------------------------
def embed_octant(T_oct: np.ndarray, n, Msize) -> np.ndarray:
    """Circulant embedding of the octant table (6, n2, n1, n0) into
    (6, M2, M1, M0): along each axis index m holds Delta = m for m < n and
    Delta = m - M for m > M - n (octant value times the parity sign), and the
    gap n <= m <= M - n is zero."""
    n0, n1, n2 = (int(v) for v in n)
    M0, M1, M2 = (int(v) for v in Msize)
    assert M0 >= 2 * n0 - 1 and M1 >= 2 * n1 - 1 and M2 >= 2 * n2 - 1
    C = np.zeros((6, M2, M1, M0), dtype=np.complex128)
    for c in range(6):
        d0, s0 = _axis_map(n0, M0, c, 0)
        d1, s1 = _axis_map(n1, M1, c, 1)
        d2, s2 = _axis_map(n2, M2, c, 2)
        C[c] = (T_oct[c][np.ix_(d2, d1, d0)]
                * s2[:, None, None] * s1[None, :, None] * s0[None, None, :])
    return C


def _axis_map(n, M, c, axis):
    m = np.arange(M)
    pos = m < n
    neg = m > M - n
    d = np.where(pos, m, np.where(neg, M - m, 0))
    s = np.where(pos, 1.0, np.where(neg, greens.parity_sign(c, axis), 0.0))
    return d, s


def green_spectrum(T_oct: np.ndarray, n, Msize) -> np.ndarray:
    """Forward 3-D DFT of each embedded component: (6, M2, M1, M0)."""
    return sfft.fftn(embed_octant(T_oct, n, Msize), axes=(1, 2, 3), workers=-1)


def apply_T(Ghat: np.ndarray, n, w: np.ndarray) -> np.ndarray:
    """u_p = sum_q T_pq * w_q (aperiodic Toeplitz convolution) via the
    circulant embedding: pad, FFT, 3x3 symmetric multiply, inverse FFT, crop."""
    n0, n1, n2 = (int(v) for v in n)
    M2, M1, M0 = Ghat.shape[1:]
    W = np.zeros((3, M2, M1, M0), dtype=np.complex128)
    W[:, :n2, :n1, :n0] = np.asarray(w).reshape(3, n2, n1, n0)
    What = sfft.fftn(W, axes=(1, 2, 3), workers=-1)
    U = np.zeros_like(What)
    for p in range(3):
        for q in range(3):
            U[p] += Ghat[greens.comp_index(p, q)] * What[q]
    u = sfft.ifftn(U, axes=(1, 2, 3), workers=-1)
    return u[:, :n2, :n1, :n0]


def matvec(Ghat: np.ndarray, n, Mvox: np.ndarray, w: np.ndarray) -> np.ndarray:
    """y = w - M (T w) (Sec. 5.4 MVP of I - M_eps N)."""
    w = np.asarray(w, dtype=np.complex128).reshape(3, *np.asarray(Mvox).shape)
    return w - np.asarray(Mvox)[None] * apply_T(Ghat, n, w)


# ----------------------------------------------------------------------------
# right-hand sides (Sec. 3 boxed J-VIE right side c_e M_eps E_inc)
# ----------------------------------------------------------------------------
def rhs_from_source(Ghat: np.ndarray, n, Mvox: np.ndarray, w_src: np.ndarray) -> np.ndarray:
    """b = c_e M e_inc for the field of an impressed current w_src radiating in
    the background: by the integral representation (Sec. 3)
    e_inc = (1/c_e)(N - I) w_src, hence b = M ((T - I) w_src)."""
    w_src = np.asarray(w_src, dtype=np.complex128).reshape(3, *np.asarray(Mvox).shape)
    return np.asarray(Mvox)[None] * (apply_T(Ghat, n, w_src) - w_src)


def rhs_plane_wave_x(n, kappa: float, Mvox: np.ndarray) -> np.ndarray:
    """b = M e_inc for E_inc = x_hat exp(-j k z) (common factors c_e h^{3/2}
    dropped): the voxel average of exp(-j kappa z) over [iz, iz + 1] is
    exp(-j kappa (iz + 1/2)) sin(kappa/2) / (kappa/2)."""
    n0, n1, n2 = (int(v) for v in n)
    zc = np.arange(n2) + 0.5
    avg = np.exp(-1j * kappa * zc) * (np.sinc(kappa / (2 * np.pi)) if kappa else 1.0)
    b = np.zeros((3, n2, n1, n0), dtype=np.complex128)
    b[0] = np.asarray(Mvox) * avg[:, None, None]
    return b
