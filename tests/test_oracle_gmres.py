"""Pins for oracle.gmres: LU agreement, Arnoldi relation, residual estimate,
finite termination, flexible variant with a nonlinear preconditioner."""
import numpy as np

from oracle import gmres, greens
from oracle import operator as op
from paper_1803_06237_gb300 import workloads


def _system(grid=(3, 3, 2), seed=5, kappa=0.4):
    eps = workloads.random_permittivity(grid, seed=seed)
    M = op.contrast_M(op.chi_from_permittivity(eps, 1.0))
    A = op.dense_A(grid, kappa, M)
    b = workloads.random_currents(grid, seed=seed + 1).ravel()
    return A, b


def test_gmres_matches_lu():
    A, b = _system()
    x_lu = np.linalg.solve(A, b)
    for restart in (5, 20, 200):
        x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-12, restart=restart, maxiter=2000)
        assert info["converged"]
        kappa_est = np.linalg.cond(A)
        assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 10 * 1e-12 * kappa_est


def test_full_gmres_terminates_in_n_steps():
    rng = np.random.default_rng(0)
    n = 12
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 5 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-13, restart=n, maxiter=n)
    assert info["iterations"] <= n and info["final_residual"] < 1e-12


def test_arnoldi_relation_and_residual_estimate():
    A, b = _system(seed=8)
    m = 15
    x, info = gmres.fgmres(lambda v: A @ v, b, tol=1e-30, restart=m, maxiter=m, record_arnoldi=True)
    V, Z = info["last_cycle"]["V"], info["last_cycle"]["Z"]
    H = np.zeros((m + 1, m), dtype=complex)
    for j, col in enumerate(info["H_raw"]):
        H[: col.size, j] = col
    lhs = np.array([A @ z for z in Z]).T
    rhs = V.T @ H
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()
    # MGS keeps orthogonality to O(eps * cond(A)), not to eps
    np.testing.assert_allclose(V.conj() @ V.T, np.eye(m + 1), atol=1e-8)
    true_res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(true_res - info["residuals"][-1]) < 1e-10


def test_flexible_with_nonlinear_preconditioner():
    A, b = _system(seed=9)
    D = np.diag(A).copy()
    P = lambda v: v / D + 1e-3 * np.tanh(v.real)      # nonlinear right preconditioner
    x, info = gmres.fgmres(lambda v: A @ v, b, precond=P, tol=1e-11, restart=30)
    assert info["converged"]
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-11
