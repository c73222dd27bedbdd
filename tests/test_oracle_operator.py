"""Pins for oracle.operator: FFT matvec vs brute-force dense assembly, the
identity at zero contrast, reciprocity, passivity of -Im N, the absorber
profile and the round-trip closed form, and a physics check (voxelised sphere
in the quasi-static limit)."""
import math

import numpy as np
import pytest

from oracle import greens, gmres
from oracle import operator as op
from paper_1803_06237_gb300 import workloads


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 3, 5), (4, 4, 4), (5, 2, 3)])
def test_fft_matvec_matches_dense(grid):
    kappa = 0.3
    eps = workloads.random_permittivity(grid, seed=11)
    M = op.contrast_M(op.chi_from_permittivity(eps, 1.0))
    w = workloads.random_currents(grid, seed=12)
    A = op.dense_A(grid, kappa, M)
    y_dense = A @ w.ravel()
    T = greens.octant_table(kappa, grid)
    for Msize in ((2 * grid[0], 2 * grid[1], 2 * grid[2]),
                  (2 * grid[0] - 1, 2 * grid[1] + 3, 2 * grid[2] + 1)):
        Gh = op.green_spectrum(T, grid, Msize)
        y_fft = op.matvec(Gh, grid, M, w).ravel()
        np.testing.assert_allclose(y_fft, y_dense, rtol=0,
                                   atol=1e-13 * np.abs(y_dense).max())


def test_zero_contrast_is_identity():
    grid = (3, 2, 4)
    M = np.zeros((4, 2, 3), dtype=complex)
    A = op.dense_A(grid, 0.2, M)
    assert np.array_equal(A, np.eye(A.shape[0]))
    T = greens.octant_table(0.2, grid)
    Gh = op.green_spectrum(T, grid, (6, 4, 8))
    w = workloads.random_currents(grid, seed=1)
    assert np.array_equal(op.matvec(Gh, grid, M, w), w)


def test_dense_T_complex_symmetric():
    T = op.dense_T((3, 3, 2), 0.4)
    np.testing.assert_allclose(T, T.T, rtol=1e-13, atol=1e-16)


def test_minus_im_T_positive_semidefinite():
    """-Im(T) is the radiated-power form (Im G = -sin(kr)/(4 pi r) has a
    non-negative spectrum on |xi| = k): all its eigenvalues are >= 0."""
    T = op.dense_T((4, 3, 3), 0.5)
    ev = np.linalg.eigvalsh(-T.imag)
    assert ev.min() > -1e-14 * ev.max(), ev.min()
    assert ev.max() > 0


def test_absorber_profile_monomials():
    nx = 40
    for d in range(4):
        prof = op.absorber_eps2(nx, x0=20.0, length=10.0, degree=d, eps2_max=3.0)
        xc = np.arange(nx) + 0.5
        u = (xc - 20.0) / 10.0
        expect = np.where((u >= 0) & (u <= 1), 3.0 * np.clip(u, 0, 1) ** d, 0.0)
        np.testing.assert_allclose(prof, expect, rtol=0, atol=1e-15)
    left = op.absorber_eps2(nx, x0=10.0, length=10.0, degree=1, eps2_max=1.0, direction=-1)
    np.testing.assert_allclose(left[:10], (10.0 - (np.arange(10) + 0.5)) / 10.0)
    assert not np.any(left[10:])


def test_round_trip_closed_form():
    """Inverting Sec. 4.3: with eps''_max from the closed form, the round-trip
    decay exp(-D eta k0 int eps''/sqrt(eps') dx) evaluated by quadrature
    returns the requested R_rt."""
    k0 = 2 * math.pi / 1.55
    for d in range(4):
        for L in (1.0, 4.0):
            e2 = op.eps2_max_from_rrt(1e-10, d, L, k0, 12.11)
            x, w = np.polynomial.legendre.leggauss(20)
            xs, ws = 0.5 * L * (x + 1), 0.5 * L * w
            integral = np.sum(ws * e2 * (xs / L) ** d / math.sqrt(12.11))
            assert abs(math.exp(-2 * k0 * integral) - 1e-10) < 1e-22


def test_contrast_definition():
    eps = workloads.random_permittivity((3, 2, 2), seed=4)
    chi = op.chi_from_permittivity(eps, 2.085)
    np.testing.assert_allclose(chi, eps / 2.085 - 1)
    er = eps / 2.085
    np.testing.assert_allclose(op.contrast_M(chi), (er - 1) / er, rtol=1e-15)


def test_absorber_only_on_core_voxels():
    eps = np.full((2, 3, 10), 12.11 + 0j)
    eps[:, 0, :] = 2.085     # a cladding row
    chi = op.chi_from_permittivity(eps, 2.085, [dict(x0=5.0, length=5.0, degree=0, eps2_max=1.0)])
    assert np.all(chi[:, 0, :] == 0)
    assert np.all(chi[:, 1:, 5:].imag < 0) and np.all(chi[:, 1:, :5].imag == 0)


def test_plane_wave_rhs_voxel_average():
    grid = (2, 2, 3)
    M = np.ones((3, 2, 2), dtype=complex)
    kappa = 0.7
    b = op.rhs_plane_wave_x(grid, kappa, M)
    x, w = np.polynomial.legendre.leggauss(20)
    for iz in range(3):
        z = iz + 0.5 * (x + 1)
        avg = np.sum(0.5 * w * np.exp(-1j * kappa * z))
        np.testing.assert_allclose(b[0, iz], avg, rtol=1e-14)
    assert not np.any(b[1:])


@pytest.mark.slow
def test_sphere_quasi_static_internal_field():
    """Physics: a voxelised dielectric sphere (eps = 4) at k a << 1 has internal
    field -> 3/(eps+2) E0 (Rayleigh).  Staircasing gives an O(h) error that must
    be a few percent and shrink as the sphere is refined."""
    errs = []
    for R in (2.5, 4.5):
        n = int(2 * math.ceil(R))
        grid = (n, n, n)
        X = op.voxel_coords(grid) + 0.5 - n / 2
        inside = np.linalg.norm(X, axis=1) <= R
        eps = 4.0
        kappa = 0.01
        chi = np.where(inside, eps - 1, 0.0).reshape(n, n, n).astype(complex)
        M = op.contrast_M(chi)
        Gh = op.green_spectrum(greens.octant_table(kappa, grid), grid, (2 * n,) * 3)
        b = op.rhs_plane_wave_x(grid, kappa, M)
        x, info = gmres.gmres(lambda v: op.matvec(Gh, grid, M, v).ravel(), b.ravel(), tol=1e-10, restart=60)
        assert info["converged"]
        w = x.reshape(3, n, n, n)
        E = (w[0][chi != 0] / chi[chi != 0]).mean() * np.exp(1j * kappa * n / 2)
        errs.append(abs(E - 3 / (eps + 2)) / (3 / (eps + 2)))
    assert errs[0] < 0.05 and errs[1] < 0.03 and errs[1] < errs[0], errs
