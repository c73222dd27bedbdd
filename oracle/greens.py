"""Galerkin entries T_pq(Delta) of the discrete operator N (oracle; FP64).

Test infrastructure only (see ``oracle/__init__``).

What the paper fixes (arXiv:1803.06237)
---------------------------------------
* Sec. 3: N f = curl curl S f, S f = int G f, G(r) = exp(-j k0 |r|) / (4 pi |r|),
  time convention exp(+j w t); the scattered field is (1/c_e)(N - I) J, so N
  contains the identity.
* Sec. 3.1 (Discretization): piecewise-constant basis P_i = (Delta V)^(-1/2) on
  voxel V_i, <P_i, P_j> = delta_ij, and N_ij = <N P_j, P_i> per Cartesian
  component pair (p, q).  On a uniform grid N is block-Toeplitz (Sec. 3.1 end)
  with six unique tensor components (Sec. 5.4).
* Sec. 2 (setup): an exterior medium eps_bg is handled by scaling, so the
  wavenumber inside the operator is k = k0 sqrt(eps_bg).

Reading (the paper gives no formula for N_ij; this derivation is ours)
---------------------------------------------------------------------
Because (lap + k^2) G = -delta,  N f = k^2 S f + grad div S f + f.  With the
voxel size h as the length unit (v = r / h, kappa = k h) the Galerkin entry
depends only on kappa and the integer offset Delta = i - j:

  T_pq(Delta) = delta_pq delta_{Delta,0} + kappa^2 delta_pq V(Delta) + D_pq(Delta)

  V(Delta)   = int g(v) L(v_x - D_x) L(v_y - D_y) L(v_z - D_z) dv
  g(v)       = exp(-j kappa |v|) / (4 pi |v|)
  L(t)       = max(0, 1 - |t|)       (overlap length of two unit boxes)

The grad-div part is reduced by the divergence theorem on V_i and on V_j to
integrals over the faces normal to p of V_i and normal to q of V_j.  After the
box-box convolution along each axis these become

  D_pp(Delta) = F_p(D_p + 1) - 2 F_p(D_p) + F_p(D_p - 1)
  F_p(t)      = int int g(t e_p + v_a e_a + v_b e_b) L(v_a - D_a) L(v_b - D_b)
  D_pq(Delta) = int g(v) s(v_p - D_p) s(v_q - D_q) L(v_r - D_r) dv   (p != q)

with s(t) = sign(t) on |t| < 1 (zero outside) and r the remaining axis.

Quadrature
----------
Every integration region is a union of unit cells whose corners are integer
points, so the singular point v = 0 is either outside a closed cell (distance
>= 1) or one of its corners.  Corner-singular cells use the Duffy split (three
pyramids in 3-D, two triangles in 2-D, apex at the origin), whose Jacobian
cancels the 1/|v| singularity; all other cells use tensor Gauss-Legendre.
Orders are chosen by the offset's Chebyshev distance and are verified by the
convergence tests.

Pins (tests/test_oracle_greens.py): closed-form static self terms (the
mean reciprocal distance of a unit cube and of a unit square), T_pp(0) = 2/3
at kappa = 0, the trace identity sum_p T_pp = 2 delta + 2 kappa^2 V (from
lap G = -k^2 G - delta), the imaginary part through the smooth kernel
-sin(kappa r)/(4 pi r) with the derivatives moved onto the kernel, the far
field (kappa^2 delta_pq + d_p d_q) g, symmetry under axis permutation and
reflection, and quadrature-order convergence.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

# Component order used everywhere in this package (symmetric tensor, six
# unique components, Sec. 5.4): xx, yy, zz, xy, xz, yz.
COMPONENTS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def comp_index(p: int, q: int) -> int:
    """Index into COMPONENTS of the (p, q) pair (symmetric)."""
    a, b = min(p, q), max(p, q)
    return COMPONENTS.index((a, b))


@functools.lru_cache(maxsize=None)
def _gl01(q: int):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def _g(r: np.ndarray, kappa: float) -> np.ndarray:
    """Scalar Green function in units of h: exp(-j kappa r) / (4 pi r)."""
    return np.exp(-1j * kappa * r) / (4.0 * np.pi * r)


def _tent(t: np.ndarray) -> np.ndarray:
    return np.maximum(0.0, 1.0 - np.abs(t))


def _sgn(t: np.ndarray) -> np.ndarray:
    return np.where(np.abs(t) < 1.0, np.sign(t), 0.0)


# ----------------------------------------------------------------------------
# quadrature rules on unit cells
# ----------------------------------------------------------------------------
@functools.lru_cache(maxsize=None)
def _duffy_cube(q: int):
    """Rule for int_{[0,1]^3} f(v) dv with an integrable 1/|v| singularity at
    the corner v = 0: three pyramids v = t (e_a + s1 e_b + s2 e_c), Jacobian t^2."""
    x, w = _gl01(q)
    T, S1, S2 = np.meshgrid(x, x, x, indexing="ij")
    W = np.einsum("i,j,k->ijk", w, w, w) * T**2
    pts, wts = [], []
    for a in range(3):
        b, c = [i for i in range(3) if i != a]
        P = np.zeros(T.shape + (3,))
        P[..., a] = T
        P[..., b] = T * S1
        P[..., c] = T * S2
        pts.append(P.reshape(-1, 3))
        wts.append(W.reshape(-1))
    return np.concatenate(pts), np.concatenate(wts)


@functools.lru_cache(maxsize=None)
def _duffy_square(q: int):
    """Rule for int_{[0,1]^2} f(v) dv with a 1/|v| singularity at v = 0:
    two triangles v = t (e_a + s e_b), Jacobian t."""
    x, w = _gl01(q)
    T, S = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w) * T
    pts, wts = [], []
    for a in range(2):
        P = np.zeros(T.shape + (2,))
        P[..., a] = T
        P[..., 1 - a] = T * S
        pts.append(P.reshape(-1, 2))
        wts.append(W.reshape(-1))
    return np.concatenate(pts), np.concatenate(wts)


@functools.lru_cache(maxsize=None)
def _gl_cube(q: int):
    x, w = _gl01(q)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return (np.stack([X, Y, Z], -1).reshape(-1, 3),
            np.einsum("i,j,k->ijk", w, w, w).reshape(-1))


@functools.lru_cache(maxsize=None)
def _gl_square(q: int):
    x, w = _gl01(q)
    X, Y = np.meshgrid(x, x, indexing="ij")
    return np.stack([X, Y], -1).reshape(-1, 2), np.outer(w, w).reshape(-1)


def _cell_rule_3d(corner, q: int, q_duffy: int):
    """Absolute points and weights for the unit cube [corner, corner + 1]."""
    corner = np.asarray(corner)
    if np.all((corner == 0) | (corner == -1)):
        # origin is a corner: reflect the Duffy rule of [0,1]^3 onto the cell
        P, W = _duffy_cube(q_duffy)
        sign = np.where(corner == -1, -1.0, 1.0)
        return P * sign, W
    P, W = _gl_cube(q)
    return P + corner, W


def _cell_rule_2d(corner2, plane_t: int, q: int, q_duffy: int):
    """Points (in-plane coordinates) and weights for a unit square in the
    plane v_p = plane_t."""
    corner2 = np.asarray(corner2)
    if plane_t == 0 and np.all((corner2 == 0) | (corner2 == -1)):
        P, W = _duffy_square(q_duffy)
        sign = np.where(corner2 == -1, -1.0, 1.0)
        return P * sign, W
    P, W = _gl_square(q)
    return P + corner2, W


def gl_order(cheb_dist: int) -> int:
    """Tensor Gauss-Legendre order per unit cell for an offset at Chebyshev
    distance ``cheb_dist`` (every non-singular cell is then at Euclidean
    distance >= max(1, cheb_dist - 1) from the singular point)."""
    d = int(cheb_dist)
    if d <= 2:
        return 16
    if d == 3:
        return 12
    if d <= 5:
        return 10
    if d <= 9:
        return 8
    if d <= 19:
        return 7
    return 6


Q_DUFFY = 16


# ----------------------------------------------------------------------------
# the entries
# ----------------------------------------------------------------------------
def face_integral(kappa: float, t: int, Da: int, Db: int, q: int = 16,
                  q_duffy: int = Q_DUFFY) -> complex:
    """F(t) = int int g(t, v_a, v_b) L(v_a - Da) L(v_b - Db) dv_a dv_b over the
    four unit squares of [Da - 1, Da + 1] x [Db - 1, Db + 1] in the plane
    v_p = t (the box-box convolution of two parallel voxel faces)."""
    acc = 0.0 + 0.0j
    for m in itertools.product((-1, 0), repeat=2):
        corner2 = np.array([Da + m[0], Db + m[1]])
        Q, Wq = _cell_rule_2d(corner2, t, q, q_duffy)
        r = np.sqrt(t * t + Q[:, 0] ** 2 + Q[:, 1] ** 2)
        acc += np.sum(_g(r, kappa) * Wq * _tent(Q[:, 0] - Da) * _tent(Q[:, 1] - Db))
    return acc


def _entries_one_rule(kappa, offsets, q, q_duffy):
    """All six T_pq for a batch of offsets that share quadrature orders."""
    offsets = np.asarray(offsets, dtype=np.int64).reshape(-1, 3)
    out = np.zeros((offsets.shape[0], 6), dtype=np.complex128)
    for n, D in enumerate(offsets):
        # ---- volume cells: the 8 unit cubes covering [D - 1, D + 1]^3
        pts, wts = [], []
        for m in itertools.product((-1, 0), repeat=3):
            P, W = _cell_rule_3d(D + np.array(m), q, q_duffy)
            pts.append(P)
            wts.append(W)
        P = np.concatenate(pts)
        W = np.concatenate(wts)
        rel = P - D
        gw = _g(np.linalg.norm(P, axis=1), kappa) * W
        Lx, Ly, Lz = _tent(rel[:, 0]), _tent(rel[:, 1]), _tent(rel[:, 2])
        Sx, Sy, Sz = _sgn(rel[:, 0]), _sgn(rel[:, 1]), _sgn(rel[:, 2])
        V = np.sum(gw * Lx * Ly * Lz)
        out[n, 3] = np.sum(gw * Sx * Sy * Lz)          # xy
        out[n, 4] = np.sum(gw * Sx * Sz * Ly)          # xz
        out[n, 5] = np.sum(gw * Sy * Sz * Lx)          # yz
        # ---- face terms: three planes per diagonal component
        self_term = 1.0 if not np.any(D) else 0.0
        for p in range(3):
            a, b = [i for i in range(3) if i != p]
            F = {dt: face_integral(kappa, int(D[p] + dt), int(D[a]), int(D[b]), q, q_duffy)
                 for dt in (-1, 0, 1)}
            out[n, p] = self_term + kappa**2 * V + (F[1] - 2.0 * F[0] + F[-1])
    return out


def toeplitz_entries(kappa: float, offsets, q_override: int | None = None,
                     q_duffy: int = Q_DUFFY) -> np.ndarray:
    """T_pq(Delta) for integer offsets (any signs), shape (K, 6), complex128.

    ``kappa`` = k h with k = k0 sqrt(eps_bg).  Component order: COMPONENTS.
    """
    offsets = np.asarray(offsets, dtype=np.int64).reshape(-1, 3)
    out = np.zeros((offsets.shape[0], 6), dtype=np.complex128)
    cheb = np.abs(offsets).max(axis=1)
    orders = np.array([q_override or gl_order(c) for c in cheb])
    for q in np.unique(orders):
        sel = np.nonzero(orders == q)[0]
        out[sel] = _entries_one_rule(kappa, offsets[sel], int(q), q_duffy)
    return out


def curl_entries(kappa: float, offsets, q_override: int | None = None,
                 q_duffy: int = Q_DUFFY) -> np.ndarray:
    """Galerkin entries of the scalar derivatives of S, in units of h:
    C_a(Delta) = <P_i, d_a S P_j> / h = int (d_a g)(u) L_Delta(u) du, shape (K, 3)
    for a = x, y, z.  By parts on the tent (no boundary terms: L_Delta vanishes
    on the edge of its support, d_a g ~ 1/|u|^2 is integrable)

        C_a(Delta) = int g(u) s(u_a - Delta_a) L(u_b - Delta_b) L(u_c - Delta_c) du,

    s(t) = sign(t) on |t| < 1, integrated with the same unit-cell rules as the
    entries of T.  The curl operator K = curl S (Sec. 3) has the entries
    K_pq(Delta) = h eps_paq C_a(Delta) (eps the Levi-Civita symbol), i.e.
    (K f) = C * f as a cross product C x f."""
    offsets = np.asarray(offsets, dtype=np.int64).reshape(-1, 3)
    out = np.zeros((offsets.shape[0], 3), dtype=np.complex128)
    cheb = np.abs(offsets).max(axis=1)
    for n, D in enumerate(offsets):
        q = q_override or gl_order(int(cheb[n]))
        pts, wts = [], []
        for m in itertools.product((-1, 0), repeat=3):
            P, W = _cell_rule_3d(D + np.array(m), q, q_duffy)
            pts.append(P)
            wts.append(W)
        P = np.concatenate(pts)
        W = np.concatenate(wts)
        rel = P - D
        gw = _g(np.linalg.norm(P, axis=1), kappa) * W
        L = [_tent(rel[:, a]) for a in range(3)]
        S = [_sgn(rel[:, a]) for a in range(3)]
        out[n, 0] = np.sum(gw * S[0] * L[1] * L[2])
        out[n, 1] = np.sum(gw * L[0] * S[1] * L[2])
        out[n, 2] = np.sum(gw * L[0] * L[1] * S[2])
    return out


def curl_octant_table(kappa: float, n) -> np.ndarray:
    """C_a for Delta in [0, n0) x [0, n1) x [0, n2); shape (3, n2, n1, n0).
    C_a is odd in Delta_a and even in the other two components."""
    n0, n1, n2 = (int(v) for v in n)
    zz, yy, xx = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    offs = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    return curl_entries(kappa, offs).T.reshape(3, n2, n1, n0)


def volume_integral(kappa: float, offset, q: int = 16, q_duffy: int = Q_DUFFY):
    """V(Delta) alone (used by the trace-identity and closed-form pins)."""
    D = np.asarray(offset, dtype=np.int64)
    acc = 0.0 + 0.0j
    for m in itertools.product((-1, 0), repeat=3):
        P, W = _cell_rule_3d(D + np.array(m), q, q_duffy)
        rel = P - D
        acc += np.sum(_g(np.linalg.norm(P, axis=1), kappa) * W
                      * _tent(rel[:, 0]) * _tent(rel[:, 1]) * _tent(rel[:, 2]))
    return acc


def octant_table(kappa: float, n) -> np.ndarray:
    """T for Delta in [0, n0) x [0, n1) x [0, n2); shape (6, n2, n1, n0)
    (z slowest, x fastest, matching the voxel layout)."""
    n0, n1, n2 = (int(v) for v in n)
    zz, yy, xx = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    offs = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    vals = toeplitz_entries(kappa, offs)
    return vals.T.reshape(6, n2, n1, n0)


def parity_sign(c: int, axis: int) -> float:
    """Sign of T_c under Delta_axis -> -Delta_axis: -1 for an off-diagonal
    component that involves ``axis`` (it is odd in D_p and D_q), else +1."""
    p, q = COMPONENTS[c]
    return -1.0 if (p != q and axis in (p, q)) else 1.0
