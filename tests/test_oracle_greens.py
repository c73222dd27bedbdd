"""Pins for oracle.greens (Galerkin entries of N, Sec. 3 and Sec. 3.1).

Each test checks the oracle against something other than itself: closed forms,
an identity of the Green function, an independent route through a smooth
kernel, the far-field asymptote, symmetry, and quadrature convergence.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import greens

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "static_self_terms.txt")
KAPPAS = (0.1351, 0.1169, 0.5)


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_golden_constants_match_closed_forms():
    g = _golden()
    s2, s3 = math.sqrt(2), math.sqrt(3)
    cube = 0.4 * (1 + s2 - 2 * s3) - 2 * math.pi / 3 + 2 * math.log((1 + s2) * (2 + s3))
    square = 4 * math.log(1 + s2) - 4.0 / 3.0 * (s2 - 1)
    assert abs(g["mean_inv_dist_unit_cube"] - cube) < 1e-15
    assert abs(g["mean_inv_dist_unit_square"] - square) < 1e-15


def test_static_volume_self_term_closed_form():
    g = _golden()
    V0 = greens.volume_integral(0.0, (0, 0, 0))
    assert abs(V0 - g["mean_inv_dist_unit_cube"] / (4 * math.pi)) < 1e-14


def test_static_face_self_term_closed_form():
    g = _golden()
    F0 = greens.face_integral(0.0, 0, 0, 0)
    assert abs(F0 - g["mean_inv_dist_unit_square"] / (4 * math.pi)) < 1e-14


def test_static_self_entry_is_two_thirds():
    g = _golden()
    T = greens.toeplitz_entries(0.0, [(0, 0, 0)])[0]
    np.testing.assert_allclose(T[:3], g["T_pp_self_static"], atol=1e-14)
    np.testing.assert_allclose(T[3:], 0.0, atol=1e-15)


def _offsets(seed=0, count=40, lo=-9, hi=9):
    rng = np.random.default_rng(seed)
    near = list(itertools.product((-1, 0, 1), repeat=3)) + [(2, 1, 0), (0, -2, 1), (2, 2, 2)]
    far = rng.integers(lo, hi + 1, size=(count, 3))
    return np.array(near + [tuple(v) for v in far])


@pytest.mark.parametrize("kappa", KAPPAS)
def test_trace_identity(kappa):
    """sum_p T_pp(D) = 2 delta_D0 + 2 kappa^2 V(D): from lap G = -k^2 G - delta the
    face (grad-div) terms are tied to the independently integrated volume term."""
    offs = _offsets(1, 20)
    T = greens.toeplitz_entries(kappa, offs)
    for D, t in zip(offs, T):
        V = greens.volume_integral(kappa, D, q=greens.gl_order(np.abs(D).max()))
        expect = 2.0 * (not np.any(D)) + 2.0 * kappa**2 * V
        assert abs(t[0] + t[1] + t[2] - expect) < 2e-15, (D, t, expect)


def _smooth_im_kernel_hessian(v, kappa):
    """(kappa^2 delta_pq + d_p d_q) applied to f(v) = -sin(kappa r)/(4 pi r) through the
    everywhere-convergent series f = -(kappa / 4 pi) S(s), s = kappa^2 r^2,
    S(s) = sum_n (-s)^n / (2n+1)!.  Returns (6, npts) in the COMPONENTS order."""
    s = kappa**2 * np.sum(v * v, axis=1)
    S1 = np.zeros_like(s)
    S2 = np.zeros_like(s)
    S0 = np.zeros_like(s)
    for n in range(0, 40):
        c = (-1.0) ** n / math.factorial(2 * n + 1)
        S0 += c * s**n
        if n >= 1:
            S1 += c * n * s ** (n - 1)
        if n >= 2:
            S2 += c * n * (n - 1) * s ** (n - 2)
    pre = -kappa / (4 * math.pi)
    out = []
    for p, q in greens.COMPONENTS:
        d2 = pre * (2 * kappa**2 * S1 * (p == q) + 4 * kappa**4 * S2 * v[:, p] * v[:, q])
        out.append(d2 + (kappa**2 * pre * S0 if p == q else 0.0))
    return np.array(out)


@pytest.mark.parametrize("kappa", KAPPAS)
def test_imaginary_part_through_smooth_kernel(kappa):
    """Im G = -sin(kr)/(4 pi r) is smooth, so Im T_pq = int L_D (k^2 d_pq + d_p d_q) Im g
    with the derivatives on the kernel and plain Gauss-Legendre: an independent route
    to the imaginary part of every entry, the self term included."""
    x, w = np.polynomial.legendre.leggauss(12)
    x01, w01 = 0.5 * (x + 1), 0.5 * w
    cells = []
    for m in itertools.product((-1, 0), repeat=3):
        X, Y, Z = np.meshgrid(x01 + m[0], x01 + m[1], x01 + m[2], indexing="ij")
        W = np.einsum("i,j,k->ijk", w01, w01, w01)
        cells.append((np.stack([X, Y, Z], -1).reshape(-1, 3), W.ravel()))
    rel = np.concatenate([c[0] for c in cells])
    W = np.concatenate([c[1] for c in cells])
    tent = np.prod(np.maximum(0, 1 - np.abs(rel)), axis=1)
    offs = _offsets(2, 12)
    T = greens.toeplitz_entries(kappa, offs)
    for D, t in zip(offs, T):
        H = _smooth_im_kernel_hessian(rel + D, kappa)
        im = H @ (W * tent)
        np.testing.assert_allclose(t.imag, im, rtol=0, atol=2e-15 * max(1.0, kappa**3 * 50))


def _dyadic(v, kappa):
    """(kappa^2 delta_pq + d_p d_q) g at points v (npts, 3), closed form of the
    dyadic Green function: e^{-jkr}/(4 pi r^3) [(k^2 r^2 - 1 - jkr) d_pq + (3 + 3jkr - k^2 r^2) vp vq / r^2]."""
    r = np.linalg.norm(v, axis=1)
    e = np.exp(-1j * kappa * r) / (4 * np.pi * r**3)
    a = kappa**2 * r**2 - 1 - 1j * kappa * r
    b = 3 + 3j * kappa * r - kappa**2 * r**2
    return np.array([e * (a * (p == q) + b * v[:, p] * v[:, q] / r**2) for p, q in greens.COMPONENTS])


@pytest.mark.parametrize("kappa", KAPPAS)
def test_integration_by_parts_route_away_from_origin(kappa):
    """For |D|_inf >= 2 the support of L_D misses the singularity, so the
    derivatives may be moved onto g: T_pq = int L_D (k^2 d_pq + d_p d_q) g.  This
    checks the face-integral (divergence theorem) formulation, signs included."""
    x, w = np.polynomial.legendre.leggauss(16)
    x01, w01 = 0.5 * (x + 1), 0.5 * w
    pts, wts = [], []
    for m in itertools.product((-1, 0), repeat=3):
        X, Y, Z = np.meshgrid(x01 + m[0], x01 + m[1], x01 + m[2], indexing="ij")
        pts.append(np.stack([X, Y, Z], -1).reshape(-1, 3))
        wts.append(np.einsum("i,j,k->ijk", w01, w01, w01).ravel())
    rel = np.concatenate(pts)
    W = np.concatenate(wts) * np.prod(np.maximum(0, 1 - np.abs(rel)), axis=1)
    offs = np.array([(2, 0, 0), (0, 2, 1), (2, 2, -1), (-3, 1, 2), (5, -4, 3), (-7, 0, 6), (11, 3, -2)])
    T = greens.toeplitz_entries(kappa, offs)
    for D, t in zip(offs, T):
        ref = _dyadic(rel + D, kappa) @ W
        np.testing.assert_allclose(t, ref, rtol=0, atol=1e-14 * np.abs(ref).max() + 1e-17)


def test_far_field_asymptote():
    """T(D) -> (1 - k^2/12)(k^2 d_pq + d_p d_q) g(D) with a residual that falls like
    |D|^-4 relative (second tent moment 1/6 per axis, lap g = -k^2 g)."""
    kappa = 0.01
    errs = []
    for R in (4, 8, 16):
        D = np.array([R, R // 2, R // 4])
        t = greens.toeplitz_entries(kappa, [D])[0]
        ref = (1 - kappa**2 / 12) * _dyadic(D[None].astype(float), kappa)[:, 0]
        errs.append(np.abs(t - ref).max() / np.abs(ref).max())
    assert errs[0] < 2e-2
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


def test_symmetries():
    """Reciprocity T(-D) = T(D); reflection parity (odd in D_p, D_q for p != q);
    axis permutation: T_xx(a,b,c) = T_yy(b,a,c), T_xz(a,b,c) = T_yz(b,a,c)."""
    kappa = 0.1351
    rng = np.random.default_rng(3)
    for D in list(rng.integers(-4, 5, size=(6, 3))) + [np.array([1, 0, 0]), np.array([1, 1, 0])]:
        t = greens.toeplitz_entries(kappa, [D])[0]
        np.testing.assert_allclose(greens.toeplitz_entries(kappa, [-D])[0], t, atol=1e-16, rtol=1e-13)
        for ax in range(3):
            Dr = D.copy()
            Dr[ax] = -Dr[ax]
            tr = greens.toeplitz_entries(kappa, [Dr])[0]
            sgn = np.array([greens.parity_sign(c, ax) for c in range(6)])
            np.testing.assert_allclose(tr, sgn * t, atol=1e-16, rtol=1e-13)
        Dp = np.array([D[1], D[0], D[2]])
        tp = greens.toeplitz_entries(kappa, [Dp])[0]
        np.testing.assert_allclose(tp[1], t[0], atol=1e-16, rtol=1e-13)
        np.testing.assert_allclose(tp[3], t[3], atol=1e-16, rtol=1e-13)
        np.testing.assert_allclose(tp[5], t[4], atol=1e-16, rtol=1e-13)


def test_quadrature_convergence():
    kappa = 0.1351
    for D in ([0, 0, 0], [1, 1, 0], [2, 1, 0], [3, 0, 2], [6, 5, 1], [12, 3, 3], [25, 9, 4]):
        q = greens.gl_order(max(abs(v) for v in D))
        a = greens.toeplitz_entries(kappa, [D])[0]
        b = greens.toeplitz_entries(kappa, [D], q_override=q + 6, q_duffy=22)[0]
        assert np.abs(a - b).max() < 5e-16, (D, np.abs(a - b).max())
