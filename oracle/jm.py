"""JM-VIE: electric and magnetic currents with impedance-matched loss (oracle; FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper (arXiv:1803.06237):
* Sec. 3, the JM-VIE: (I - M T)(J, M) = C M (E_inc, H_inc) with
  T = [[N, -c_e K], [c_m K, N]], K f = curl S f, M = diag(M_eps, M_mu),
  M_mu = (mu_r - 1)/mu_r, c_e = j w eps_0, c_m = j w mu_0; discrete form in
  Sec. 3.1 with the same piecewise-constant basis for both currents.
* Sec. 4.2: impedance matching in the absorber, mu_r = 1 - j mu'' with
  mu'' = eps''/eps'.

Scaling (our reading; the paper keeps c_e and c_m explicit).  With
u_e = J / c_e and u_m = eta M / c_m (both in units of the electric field;
eta the background impedance) and h as the unit of length (kappa = k h), the
rows of the system become

    u_e - M_eps (T u_e) + j kappa M_eps (C x u_m) = M_eps e_inc
    u_m - M_mu  (T u_m) - j kappa M_mu  (C x u_e) = M_mu  h_inc

with T the J-VIE Toeplitz table of ``greens`` and (C x f)_p = eps_paq C_a * f_q
the curl Toeplitz operator (``greens.curl_entries``; K = h C), and h_inc =
eta H_inc.  The total fields are E = e_inc + (T - I) u_e - j kappa C x u_m and
eta H = h_inc + (T - I) u_m + j kappa C x u_e, so u_e = chi_e E and
u_m = chi_m eta H.  A plane wave E = x exp(-j k z) has eta H = y exp(-j k z).

Layout: a JM vector is u[c][z][y][x] with c = 0..2 the electric and c = 3..5
the magnetic components, shape (6, nz, ny, nx).

Pins (tests/test_oracle_jm.py): C_a odd in Delta_a and even in the other
offsets, C_a(0) = 0, axis permutation; for |Delta|_inf >= 2 C_a equals the
tent-weighted integral of the closed-form d_a g; the far field
C_a -> (1 - kappa^2/12) d_a g; Im C_a against its plane-wave expansion;
dense per-pair assembly vs the FFT matvec; the dense curl matrix is complex
symmetric (reciprocity); zero contrast gives the identity; a cube with
eps_r = mu_r scatters nothing backwards (zero-backscatter theorem for
dual-symmetric scatterers with four-fold rotation symmetry about the
incidence axis); energy balance in a lossless case.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import greens
from . import operator as op

# (p, q) -> (a, sign) with K_pq = sign * C_a (sign = eps_paq)
_CURL = {(0, 1): (2, -1.0), (1, 0): (2, +1.0), (0, 2): (1, +1.0), (2, 0): (1, -1.0),
         (1, 2): (0, -1.0), (2, 1): (0, +1.0)}


def mu_contrast(mu: np.ndarray) -> np.ndarray:
    """M_mu = (mu_r - 1)/mu_r (Sec. 3) per voxel."""
    mu = np.asarray(mu, dtype=np.complex128)
    return (mu - 1.0) / mu


def matched_permeability(chi: np.ndarray) -> np.ndarray:
    """mu_r = 1 - j mu'' with mu'' = eps''/eps' (Sec. 4.2) from the contrast
    chi = eps_r/eps_bg - 1 (eps' - j eps'' = eps_bg (1 + chi); the ratio does
    not depend on eps_bg): non-zero where the permittivity is lossy, i.e. in
    the absorbers."""
    chi = np.asarray(chi, dtype=np.complex128)
    return 1.0 - 1j * (-chi.imag) / (1.0 + chi.real)


# ----------------------------------------------------------------------------
# dense assembly (tiny grids)
# ----------------------------------------------------------------------------
def dense_K(n, kappa: float) -> np.ndarray:
    """(3N x 3N) curl matrix in units of h: K[(p,i),(q,j)] = eps_paq C_a(r_i - r_j),
    every pair offset evaluated directly (no parity used)."""
    X = op.voxel_coords(n)
    N = X.shape[0]
    diffs = (X[:, None, :] - X[None, :, :]).reshape(-1, 3)
    uniq, inv = np.unique(diffs, axis=0, return_inverse=True)
    vals = greens.curl_entries(kappa, uniq)[inv.ravel()].reshape(N, N, 3)
    K = np.zeros((3 * N, 3 * N), dtype=np.complex128)
    for (p, q), (a, sg) in _CURL.items():
        K[p * N:(p + 1) * N, q * N:(q + 1) * N] = sg * vals[:, :, a]
    return K


def dense_A(n, kappa: float, Me: np.ndarray, Mm: np.ndarray) -> np.ndarray:
    """The (6N x 6N) JM-VIE matrix in the scaled unknowns (u_e, u_m)."""
    T = op.dense_T(n, kappa)
    K = dense_K(n, kappa)
    me = np.tile(np.asarray(Me, dtype=np.complex128).ravel(), 3)
    mm = np.tile(np.asarray(Mm, dtype=np.complex128).ravel(), 3)
    I3 = np.eye(T.shape[0], dtype=np.complex128)
    top = np.hstack([I3 - me[:, None] * T, 1j * kappa * me[:, None] * K])
    bot = np.hstack([-1j * kappa * mm[:, None] * K, I3 - mm[:, None] * T])
    return np.vstack([top, bot])


# ----------------------------------------------------------------------------
# FFT matvec
# ----------------------------------------------------------------------------
def curl_spectrum(C_oct: np.ndarray, n, Msize) -> np.ndarray:
    """Circulant embedding of the octant table (3, n2, n1, n0) of C_a (odd in
    axis a, even in the others; the gap zero) and its 3-D DFT: (3, M2, M1, M0)."""
    n0, n1, n2 = (int(v) for v in n)
    M0, M1, M2 = (int(v) for v in Msize)
    assert M0 >= 2 * n0 - 1 and M1 >= 2 * n1 - 1 and M2 >= 2 * n2 - 1
    C = np.zeros((3, M2, M1, M0), dtype=np.complex128)
    for a in range(3):
        maps = []
        for axis, (nn, MM) in enumerate(((n0, M0), (n1, M1), (n2, M2))):
            m = np.arange(MM)
            pos, neg = m < nn, m > MM - nn
            d = np.where(pos, m, np.where(neg, MM - m, 0))
            sg = np.where(pos, 1.0, np.where(neg, -1.0 if axis == a else 1.0, 0.0))
            maps.append((d, sg))
        (d0, s0), (d1, s1), (d2, s2) = maps
        C[a] = C_oct[a][np.ix_(d2, d1, d0)] * s2[:, None, None] * s1[None, :, None] * s0[None, None, :]
    return sfft.fftn(C, axes=(1, 2, 3), workers=-1)


def apply_curl(Ch: np.ndarray, n, f: np.ndarray) -> np.ndarray:
    """(C x f)_p = eps_paq C_a * f_q (aperiodic convolution) via the embedding."""
    n0, n1, n2 = (int(v) for v in n)
    M2, M1, M0 = Ch.shape[1:]
    F = np.zeros((3, M2, M1, M0), dtype=np.complex128)
    F[:, :n2, :n1, :n0] = np.asarray(f).reshape(3, n2, n1, n0)
    Fh = sfft.fftn(F, axes=(1, 2, 3), workers=-1)
    U = np.zeros_like(Fh)
    for (p, q), (a, sg) in _CURL.items():
        U[p] += sg * Ch[a] * Fh[q]
    u = sfft.ifftn(U, axes=(1, 2, 3), workers=-1)
    return u[:, :n2, :n1, :n0]


def matvec(Gh: np.ndarray, Ch: np.ndarray, n, Me: np.ndarray, Mm: np.ndarray, u: np.ndarray, kappa: float):
    """y = (I - M T) u for the scaled JM unknowns u (6, nz, ny, nx)."""
    n0, n1, n2 = (int(v) for v in n)
    u = np.asarray(u, dtype=np.complex128).reshape(6, n2, n1, n0)
    ue, um = u[:3], u[3:]
    Me = np.asarray(Me)[None]
    Mm = np.asarray(Mm)[None]
    ye = ue - Me * (op.apply_T(Gh, n, ue) - 1j * kappa * apply_curl(Ch, n, um))
    ym = um - Mm * (op.apply_T(Gh, n, um) + 1j * kappa * apply_curl(Ch, n, ue))
    return np.concatenate([ye, ym])


def rhs_plane_wave_x(n, kappa: float, Me: np.ndarray, Mm: np.ndarray) -> np.ndarray:
    """b = (M_eps e_inc, M_mu h_inc) for E = x exp(-j k z), eta H = y exp(-j k z)
    (voxel averages, common factors dropped as in ``operator.rhs_plane_wave_x``)."""
    be = op.rhs_plane_wave_x(n, kappa, Me)
    avg = op.rhs_plane_wave_x(n, kappa, np.ones_like(np.asarray(Me)))[0]
    bm = np.zeros_like(be)
    bm[1] = np.asarray(Mm) * avg
    return np.concatenate([be, bm])


def rhs_from_source(Gh: np.ndarray, Ch: np.ndarray, n, Me: np.ndarray, Mm: np.ndarray, w_src: np.ndarray,
                    kappa: float) -> np.ndarray:
    """b for an impressed electric current w_src (scaled like u_e) radiating in
    the background: e_inc = (T - I) w_src and eta H_inc = j kappa C x w_src
    (Sec. 3 integral representation), b = (M_eps e_inc, M_mu h_inc)."""
    n0, n1, n2 = (int(v) for v in n)
    w_src = np.asarray(w_src, dtype=np.complex128).reshape(3, n2, n1, n0)
    e = op.apply_T(Gh, n, w_src) - w_src
    h = 1j * kappa * apply_curl(Ch, n, w_src)
    return np.concatenate([np.asarray(Me)[None] * e, np.asarray(Mm)[None] * h])


def fields(Gh: np.ndarray, Ch: np.ndarray, n, u: np.ndarray, e_inc: np.ndarray, h_inc: np.ndarray, kappa: float):
    """Total E and eta H in the voxels from the solution u and the incident fields."""
    n0, n1, n2 = (int(v) for v in n)
    u = np.asarray(u).reshape(6, n2, n1, n0)
    ue, um = u[:3], u[3:]
    E = e_inc + op.apply_T(Gh, n, ue) - ue - 1j * kappa * apply_curl(Ch, n, um)
    H = h_inc + op.apply_T(Gh, n, um) - um + 1j * kappa * apply_curl(Ch, n, ue)
    return E, H
