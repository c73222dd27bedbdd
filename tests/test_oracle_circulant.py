"""Pins of the oracle's block-circulant preconditioner (oracle/circulant.py).

The blocks are checked against the definition (averages of the wrapped block
diagonals of the dense A, assembled voxel pair by voxel pair), against the
optimality condition of a Frobenius-nearest block-circulant matrix, against
T. Chan's closed form for a Toeplitz matrix, and the inverse against the
direct block circular convolution."""
import math

import numpy as np
import pytest

from oracle import circulant as circ
from oracle import operator as op
from paper_1803_06237_gb300 import workloads

KAPPA = 0.02 * 2 * math.pi / 1.55 * math.sqrt(2.085)


def _dense_blocks(A, n):
    """A as an nx x nx array of (3B x 3B) blocks with the in-block order (p, z, y)."""
    nx, ny, nz = n
    N = nx * ny * nz
    B = ny * nz
    rows = np.zeros((nx, 3 * B), dtype=np.int64)
    for p in range(3):
        for z in range(nz):
            for y in range(ny):
                r = p * B + z * ny + y
                rows[:, r] = p * N + (z * ny + y) * nx + np.arange(nx)
    return np.array([[A[np.ix_(rows[i], rows[j])] for j in range(nx)] for i in range(nx)])


def _random_M(n, seed):
    return op.contrast_M(op.chi_from_permittivity(workloads.random_permittivity(n, seed=seed), 2.085))


@pytest.mark.parametrize("n", [(5, 3, 2), (4, 2, 3)])
def test_blocks_are_wrapped_diagonal_averages_of_dense_A(n):
    M = _random_M(n, 1)
    A = op.dense_A(n, KAPPA, M)
    Ab = _dense_blocks(A, n)
    nx = n[0]
    c = circ.circulant_blocks(n, KAPPA, M)
    for k in range(nx):
        ref = sum(Ab[i, (i - k) % nx] for i in range(nx)) / nx
        assert np.abs(c[k] - ref).max() <= 1e-13 * np.abs(ref).max() + 1e-15


def test_frobenius_optimality():
    """A - W is orthogonal to every block-circulant matrix, so W + e B is
    farther from A than W for any block-circulant B and any e != 0."""
    n = (5, 2, 2)
    M = _random_M(n, 2)
    A = op.dense_A(n, KAPPA, M)
    Ab = _dense_blocks(A, n)
    nx = n[0]
    c = circ.circulant_blocks(n, KAPPA, M)
    W = np.array([[c[(i - j) % nx] for j in range(nx)] for i in range(nx)])
    rng = np.random.default_rng(3)
    base = np.linalg.norm(Ab - W)
    for _ in range(4):
        d = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
        D = np.array([[d[(i - j) % nx] for j in range(nx)] for i in range(nx)])
        # first-order condition: <A - W, D> = 0
        assert abs(np.vdot(D, Ab - W)) <= 1e-10 * np.linalg.norm(D) * base
        for e in (1e-3, -1e-3):
            assert np.linalg.norm(Ab - W - e * D) > base


def test_chan_closed_form_for_constant_contrast():
    """Contrast independent of x: A is block Toeplitz in x and the optimal
    circulant is T. Chan's c_k = ((nx - k) a_k + k a_{k - nx}) / nx with
    a_d = delta_d0 I - m T(d) (m the contrast of each row)."""
    n = (6, 2, 2)
    nx, ny, nz = n
    m_yz = _random_M((1, ny, nz), 4).reshape(nz, ny, 1)
    M = np.repeat(m_yz, nx, axis=2)
    c = circ.circulant_blocks(n, KAPPA, M)
    Tfull = circ._offsets_table(n, KAPPA)
    rowm = np.tile(m_yz.ravel(), 3)
    eye = np.eye(3 * ny * nz)
    a = lambda d: (eye if d == 0 else 0.0) - rowm[:, None] * circ.x_block(Tfull, n, d)
    for k in range(nx):
        ref = ((nx - k) * a(k) + (k * a(k - nx) if k else 0.0)) / nx
        assert np.abs(c[k] - ref).max() <= 1e-13


def test_single_slice_is_exact():
    n = (1, 3, 2)
    M = _random_M(n, 5)
    A = op.dense_A(n, KAPPA, M)
    c = circ.circulant_blocks(n, KAPPA, M)
    Ab = _dense_blocks(A, n)
    assert np.abs(c[0] - Ab[0, 0]).max() <= 1e-14


def test_inverse_undoes_block_circular_convolution():
    n = (7, 3, 2)
    M = _random_M(n, 6)
    c = circ.circulant_blocks(n, KAPPA, M)
    What = circ.blocks_hat(c)
    v = workloads.random_currents(n, seed=7)
    z = circ.apply_inverse(What, v)
    assert np.linalg.norm(circ.apply_W(c, z) - v) <= 1e-11 * np.linalg.norm(v)


def test_preconditioned_gmres_needs_far_fewer_steps():
    """Sec. 5.4: on a strip guide with an absorber the circulant preconditioner
    cuts the GMRES step count several-fold (here 60 x 6 x 3 voxels of 80 nm)."""
    from oracle import gmres as gm
    from oracle import greens
    wl = workloads.waveguide(nx=60, ny=6, nz=3, h_um=0.08, absorber_len_um=1.6, src_x_um=1.2, waist_um=0.2)
    ab = wl.absorbers[0]
    e2 = op.eps2_max_from_rrt(ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
    chi = op.chi_from_permittivity(wl.eps, wl.eps_bg, [dict(x0=ab.x0, length=ab.length, degree=ab.degree,
                                                           eps2_max=e2)])
    M = op.contrast_M(chi)
    n = wl.grid
    Gh = op.green_spectrum(greens.octant_table(wl.kappa, n), n, (2 * n[0], 2 * n[1], 2 * n[2]))
    b = op.rhs_from_source(Gh, n, M, wl.src).ravel()
    A = lambda x: op.matvec(Gh, n, M, x.reshape(3, n[2], n[1], n[0])).ravel()
    What = circ.blocks_hat(circ.circulant_blocks(n, wl.kappa, M))
    P = lambda v: circ.apply_inverse(What, v.reshape(3, n[2], n[1], n[0])).ravel()
    x0, i0 = gm.gmres(A, b, tol=1e-6, restart=30, maxiter=3000)
    x1, i1 = gm.fgmres(A, b, P, tol=1e-6, restart=30, maxiter=3000)
    assert np.linalg.norm(b - A(x1)) <= 1e-6 * np.linalg.norm(b)
    assert i1["iterations"] * 4 <= i0["iterations"]
    assert np.linalg.norm(x1 - x0) <= 1e-4 * np.linalg.norm(x0)
