"""Pins for the JM-VIE oracle (oracle/jm.py, greens.curl_entries): curl
entries by symmetry, by a second integration route and the far field, the
imaginary part by the plane-wave expansion, dense vs FFT matvec,
reciprocity, the identity at zero contrast, the zero-backscatter theorem for
a cube with eps_r = mu_r, and energy balance in a lossless case."""
import itertools

import numpy as np
import pytest

from oracle import greens
from oracle import jm
from oracle import operator as op
from paper_1803_06237_gb300 import workloads

KAPPAS = (0.05, 0.4, 1.3)


def _dgrad(v, kappa):
    """d_a g at points v (npts, 3): g' (r) v_a / r = -g (1 + j kappa r) v_a / r^2."""
    r = np.linalg.norm(v, axis=1)
    g = np.exp(-1j * kappa * r) / (4 * np.pi * r)
    f = -g * (1 + 1j * kappa * r) / r**2
    return np.array([f * v[:, a] for a in range(3)])


def _sphere_rule(ntheta=40, nphi=80):
    ct, wt = np.polynomial.legendre.leggauss(ntheta)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - ct**2)
    S = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)), np.outer(ct, np.ones(nphi))], -1).reshape(-1, 3)
    return S, np.outer(wt, np.full(nphi, 2 * np.pi / nphi)).ravel()


def test_curl_entry_symmetries():
    kappa = 0.37
    rng = np.random.default_rng(4)
    offs = [np.array(d) for d in rng.integers(-4, 5, size=(6, 3))] + [np.array([1, 0, 0]), np.array([1, 1, 0])]
    assert np.allclose(greens.curl_entries(kappa, [[0, 0, 0]]), 0, atol=1e-15)
    for D in offs:
        c = greens.curl_entries(kappa, [D])[0]
        np.testing.assert_allclose(greens.curl_entries(kappa, [-D])[0], -c, atol=1e-16, rtol=1e-13)
        for ax in range(3):
            Dr = D.copy()
            Dr[ax] = -Dr[ax]
            cr = greens.curl_entries(kappa, [Dr])[0]
            sgn = np.array([-1.0 if a == ax else 1.0 for a in range(3)])
            np.testing.assert_allclose(cr, sgn * c, atol=1e-16, rtol=1e-13)
        Dp = np.array([D[1], D[0], D[2]])
        cp = greens.curl_entries(kappa, [Dp])[0]
        np.testing.assert_allclose(cp[1], c[0], atol=1e-16, rtol=1e-13)
        np.testing.assert_allclose(cp[0], c[1], atol=1e-16, rtol=1e-13)


@pytest.mark.parametrize("kappa", KAPPAS)
def test_curl_entries_by_the_derivative_route(kappa):
    """For |D|_inf >= 2 the support of the tent misses the singularity, so the
    derivative may stay on g: C_a = int (d_a g)(u) L_D(u) du (closed-form
    gradient) must equal the by-parts form with sign(u_a - D_a)."""
    x, w = np.polynomial.legendre.leggauss(16)
    x01, w01 = 0.5 * (x + 1), 0.5 * w
    pts, wts = [], []
    for m in itertools.product((-1, 0), repeat=3):
        X, Y, Z = np.meshgrid(x01 + m[0], x01 + m[1], x01 + m[2], indexing="ij")
        P = np.stack([X, Y, Z], -1).reshape(-1, 3)
        pts.append(P)
        wts.append(np.einsum("i,j,k->ijk", w01, w01, w01).ravel() * np.prod(1 - np.abs(P), axis=1))
    rel = np.concatenate(pts)
    W = np.concatenate(wts)
    for D in ([2, 0, 0], [2, 1, 0], [0, 3, 1], [2, 2, 2], [-3, 1, 2]):
        c = greens.curl_entries(kappa, [D])[0]
        ref = _dgrad(rel + np.array(D, float), kappa) @ W
        np.testing.assert_allclose(c, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_curl_far_field_asymptote():
    """C_a(D) -> (1 - kappa^2/12) d_a g(D), the residual falling like |D|^-4
    relative (tent second moment 1/6 per axis, lap d_a g = -kappa^2 d_a g)."""
    kappa = 0.01
    errs = []
    for R in (4, 8, 16):
        D = np.array([R, R // 2, R // 4])
        c = greens.curl_entries(kappa, [D])[0]
        ref = (1 - kappa**2 / 12) * _dgrad(D[None].astype(float), kappa)[:, 0]
        errs.append(np.abs(c - ref).max() / np.abs(ref).max())
    assert errs[0] < 2e-2
    assert errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs


@pytest.mark.parametrize("kappa", (0.4, 1.1))
def test_curl_imaginary_part_by_plane_waves(kappa):
    """Im g = -(kappa/16 pi^2) int exp(j kappa s.u) dOmega gives
    Im C_a(D) = -(kappa/16 pi^2) int j kappa s_a exp(j kappa s.D)
    prod_b sinc^2(kappa s_b / 2) dOmega (exact up to the angular rule)."""
    S, wq = _sphere_rule()
    form = np.prod(np.sinc(kappa * S / (2 * np.pi)) ** 2, axis=1)
    for D in ([1, 0, 0], [1, 1, 0], [0, 2, 1], [3, -1, 2], [0, 0, 0]):
        c = greens.curl_entries(kappa, [D])[0]
        ph = np.exp(1j * kappa * S @ np.array(D, float))
        ref = np.array([-(kappa / (16 * np.pi**2)) * np.sum(wq * 1j * kappa * S[:, a] * ph * form) for a in range(3)])
        assert np.abs(ref.imag).max() < 1e-14
        np.testing.assert_allclose(c.imag, ref.real, rtol=0, atol=1e-12 * max(1e-3, np.abs(ref).max()))


@pytest.mark.parametrize("grid", [(2, 3, 2), (3, 2, 2), (1, 1, 1)])
def test_jm_fft_matvec_matches_dense(grid):
    kappa = 0.45
    Me = op.contrast_M(op.chi_from_permittivity(workloads.random_permittivity(grid, seed=31), 1.0))
    Mm = jm.mu_contrast(workloads.random_permittivity(grid, seed=32) * 0.3 + 1.0)
    u = np.concatenate([workloads.random_currents(grid, seed=33), workloads.random_currents(grid, seed=34)])
    A = jm.dense_A(grid, kappa, Me, Mm)
    y_dense = A @ u.ravel()
    Gh = op.green_spectrum(greens.octant_table(kappa, grid), grid, tuple(2 * v for v in grid))
    Ch = jm.curl_spectrum(greens.curl_octant_table(kappa, grid), grid, tuple(2 * v for v in grid))
    y = jm.matvec(Gh, Ch, grid, Me, Mm, u, kappa).ravel()
    np.testing.assert_allclose(y, y_dense, rtol=0, atol=1e-13 * np.abs(y_dense).max())
    Ch2 = jm.curl_spectrum(greens.curl_octant_table(kappa, grid), grid, tuple(2 * v + 1 for v in grid))
    Gh2 = op.green_spectrum(greens.octant_table(kappa, grid), grid, tuple(2 * v + 1 for v in grid))
    np.testing.assert_allclose(jm.matvec(Gh2, Ch2, grid, Me, Mm, u, kappa).ravel(), y_dense, rtol=0,
                               atol=1e-13 * np.abs(y_dense).max())


def test_curl_matrix_reciprocity_and_identity():
    K = jm.dense_K((3, 2, 2), 0.6)
    np.testing.assert_allclose(K, K.T, rtol=1e-13, atol=1e-16)
    grid = (2, 2, 2)
    A = jm.dense_A(grid, 0.6, np.zeros((2, 2, 2)), np.zeros((2, 2, 2)))
    assert np.array_equal(A, np.eye(A.shape[0]))


def _far(u, grid, kappa, S):
    """Far-field pattern (I - s s) W_e - s x W_m with W(s) = sum_j u_j exp(+j kappa s.c_j)
    (the voxel form factor is common to both and dropped)."""
    nx, ny, nz = grid
    C = op.voxel_coords(grid) + 0.5
    ph = np.exp(1j * kappa * (S @ C.T))
    We = ph @ u[:3].reshape(3, -1).T
    Wm = ph @ u[3:].reshape(3, -1).T
    return We - S * np.sum(S * We, axis=1)[:, None] - np.cross(S, Wm)


def test_zero_backscatter_for_eps_equal_mu_cube():
    """A scatterer with eps_r = mu_r (here a 4^3 voxel cube, invariant under a
    quarter turn about the incidence axis) sends nothing back towards the
    source; the same cube with mu_r = 1 does."""
    grid = (4, 4, 4)
    kappa = 0.5
    S = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]])
    for mu, back_small in ((3.0 - 0.5j, True), (1.0, False)):
        Me = np.full((4, 4, 4), op.contrast_M(2.0 - 0.5j))
        Mm = np.full((4, 4, 4), jm.mu_contrast(mu))
        A = jm.dense_A(grid, kappa, Me, Mm)
        b = jm.rhs_plane_wave_x(grid, kappa, Me, Mm).ravel()
        u = np.linalg.solve(A, b).reshape(6, 4, 4, 4)
        F = _far(u, grid, kappa, S)
        ratio = np.linalg.norm(F[0]) / np.linalg.norm(F[1])
        if back_small:
            assert ratio < 1e-12, ratio
        else:
            assert ratio > 1e-2, ratio


def test_energy_balance_lossless_and_far_field():
    """Real eps and mu: extinction Im(u_e^H e_inc + u_m^H h_inc) equals the power
    radiated by both currents, (kappa^3/16 pi^2) int |(I - s s) W_e - s x W_m|^2
    dOmega (voxel form factor included), to the solver's precision."""
    grid = (3, 3, 2)
    kappa = 0.7
    Me = np.full((2, 3, 3), op.contrast_M(3.0))
    Mm = np.full((2, 3, 3), jm.mu_contrast(1.8))
    A = jm.dense_A(grid, kappa, Me, Mm)
    b = jm.rhs_plane_wave_x(grid, kappa, Me, Mm)
    u = np.linalg.solve(A, b.ravel()).reshape(6, 2, 3, 3)
    einc = jm.rhs_plane_wave_x(grid, kappa, np.ones((2, 3, 3)), np.ones((2, 3, 3)))
    ext = np.imag(np.vdot(u.ravel(), einc.ravel()))
    S, wq = _sphere_rule(48, 96)
    form = np.prod(np.sinc(kappa * S / (2 * np.pi)), axis=1)
    F = _far(u, grid, kappa, S) * form[:, None]
    rad = kappa**3 / (16 * np.pi**2) * np.sum(wq * np.sum(np.abs(F) ** 2, axis=1))
    assert rad > 0
    assert abs(ext - rad) <= 1e-10 * rad, (ext, rad)


def test_matched_permeability():
    eps = np.full((2, 2, 10), 12.11 + 0j)
    eps[:, 0, :] = 2.085
    ab = [dict(x0=5.0, length=5.0, degree=1, eps2_max=2.0)]
    chi = op.chi_from_permittivity(eps, 2.085, ab)
    mu = jm.matched_permeability(chi)
    e2 = op.absorber_eps2(10, 5.0, 5.0, 1, 2.0)
    np.testing.assert_allclose(mu[:, 1, :], np.broadcast_to(1 - 1j * e2 / 12.11, (2, 10)), rtol=1e-15)
    assert np.all(mu[:, 0, :] == 1)
    assert np.all(mu[:, 1, :5] == 1)
