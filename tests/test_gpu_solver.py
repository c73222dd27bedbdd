"""GPU Krylov solves against the FP64 oracle (dense LU on small grids,
oracle GMRES on the cube and a guide section), through the C ABI.

Tolerances: a solve to relative residual tol has forward error at most
cond(A) * tol; the tests use the measured condition number (small grids) or
a factor-of-100 allowance (cube, guide) on the stated tolerance."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle import gmres, greens
from oracle import operator as op
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu
K0 = 2 * math.pi / 1.55


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.complex128).ravel())).cuda()


@pytest.mark.parametrize("mode", [vie.VIE_SOLVE_FP64, vie.VIE_SOLVE_MIXED])
def test_small_solve_matches_lu(mode):
    grid = (5, 4, 3)
    plan = vie.vie_plan_create(grid, 0.05, K0, 2.085)
    eps = workloads.random_permittivity(grid, seed=61)
    vie.vie_set_permittivity(plan, eps)
    kappa = plan.info()["kappa"]
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    A = op.dense_A(grid, kappa, M)
    b = workloads.random_currents(grid, seed=62).ravel()
    x_lu = np.linalg.solve(A, b)
    bd, xd = _dev(b), torch.zeros(b.size, dtype=torch.complex128, device="cuda")
    tol = 1e-10
    info = vie.vie_solve(plan, bd, xd, tol, mode=mode, restart=30)
    assert info["converged"] and info["residual"] <= tol
    x = xd.cpu().numpy()
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= 2 * tol
    assert rel_l2(x, x_lu) <= np.linalg.cond(A) * tol
    if mode == vie.VIE_SOLVE_MIXED:
        assert info["matvecs32"] > 0 and info["outer"] >= 2


def test_cube_plane_wave_fp64_gmres50():
    """Cube 12^3, eps = 12.25, x-polarised plane wave, complex128, GMRES(50) to 1e-10."""
    wl = workloads.cube(12)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps)
    M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg))
    b = op.rhs_plane_wave_x(wl.grid, wl.kappa, M)
    bd, xd = _dev(b), torch.zeros(b.size, dtype=torch.complex128, device="cuda")
    info = vie.vie_solve(plan, bd, xd, 1e-10, mode=vie.VIE_SOLVE_FP64, restart=50)
    assert info["converged"]
    Gh = op.green_spectrum(greens.octant_table(wl.kappa, wl.grid), wl.grid, (24, 24, 24))
    x_ref, rinfo = gmres.gmres(lambda v: op.matvec(Gh, wl.grid, M, v).ravel(), b.ravel(), tol=1e-12, restart=50)
    assert rinfo["converged"]
    assert rel_l2(xd.cpu().numpy(), x_ref) <= 1e-9


def test_guide_section_mixed_and_fp64_agree_with_oracle():
    nx = 80
    wl = workloads.waveguide(nx=nx, absorber_len_um=0.6, src_x_um=0.3)
    ab = wl.absorbers[0]
    e2 = op.eps2_max_from_rrt(1e-10, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
    absorbers = [dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2)]
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    src = _dev(wl.src)
    bd = torch.empty_like(src)
    vie.vie_rhs_from_source(plan, src, bd)
    M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg, absorbers))
    Gh = op.green_spectrum(greens.octant_table(wl.kappa, wl.grid), wl.grid, tuple(2 * v for v in wl.grid))
    b_ref = op.rhs_from_source(Gh, wl.grid, M, wl.src).ravel()
    assert rel_l2(bd.cpu().numpy(), b_ref) <= 1e-12
    x_ref, rinfo = gmres.gmres(lambda v: op.matvec(Gh, wl.grid, M, v).ravel(), b_ref, tol=1e-11, restart=200)
    assert rinfo["converged"]
    for mode, tol in ((vie.VIE_SOLVE_FP64, 1e-8), (vie.VIE_SOLVE_MIXED, 1e-6), (vie.VIE_SOLVE_MIXED, 1e-9)):
        xd = torch.zeros_like(bd)
        info = vie.vie_solve(plan, bd, xd, tol, mode=mode, restart=100)
        assert info["converged"] and info["residual"] <= tol, info
        assert rel_l2(xd.cpu().numpy(), x_ref) <= 100 * tol, (mode, tol, info)


def test_warm_start_and_zero_rhs():
    grid = (6, 5, 4)
    plan = vie.vie_plan_create(grid, 0.03, K0, 1.0)
    vie.vie_set_permittivity(plan, workloads.random_permittivity(grid, seed=71))
    b = _dev(workloads.random_currents(grid, seed=72))
    x = torch.zeros_like(b)
    i1 = vie.vie_solve(plan, b, x, 1e-9, mode=vie.VIE_SOLVE_FP64)
    i2 = vie.vie_solve(plan, b, x, 1e-9, mode=vie.VIE_SOLVE_FP64, x0_given=True)
    assert i2["converged"] and i2["iterations"] == 0 and i1["iterations"] > 0
    z = torch.zeros_like(b)
    i3 = vie.vie_solve(plan, z, x, 1e-9)
    assert i3["converged"] and torch.count_nonzero(x).item() == 0


def test_iteration_cap_reports_not_converged():
    grid = (8, 6, 5)
    plan = vie.vie_plan_create(grid, 0.03, K0, 1.0)
    vie.vie_set_permittivity(plan, workloads.random_permittivity(grid, seed=81))
    b = _dev(workloads.random_currents(grid, seed=82))
    x = torch.zeros_like(b)
    info = vie.vie_solve(plan, b, x, 1e-12, mode=vie.VIE_SOLVE_FP64, restart=5, max_iters=7,
                         raise_on_not_converged=False)
    assert info["status"] == 4 and not info["converged"] and info["iterations"] <= 7
    assert np.isfinite(x.cpu().numpy()).all()
