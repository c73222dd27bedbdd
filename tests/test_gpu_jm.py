"""GPU JM-VIE (Sec. 3: electric and magnetic currents; Sec. 4.2 impedance
matching) against the FP64 oracle (oracle/jm.py): operator and right-hand
side on grids that span several blocks with ragged edges, solves against
dense LU, the zero-backscatter theorem on a GPU solution, and the
reflection of a matched absorber against an electric-only one."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle import greens, jm
from oracle import operator as op
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu
K0 = 2 * math.pi / 1.55
TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def _oracle_spectra(grid, kappa):
    M = tuple(2 * v for v in grid)
    Gh = op.green_spectrum(greens.octant_table(kappa, grid), grid, M)
    Ch = jm.curl_spectrum(greens.curl_octant_table(kappa, grid), grid, M)
    return Gh, Ch


def _plan(grid, seed, h=0.03, eps_bg=2.085):
    plan = vie.vie_plan_create(grid, h, K0, eps_bg)
    eps = workloads.random_permittivity(grid, seed=seed)
    vie.vie_set_permittivity(plan, eps)
    mu = 1.0 + 0.3 * (workloads.random_permittivity(grid, seed=seed + 1) - 1.0) / 12.0
    vie.vie_set_permeability(plan, mu)
    Me = op.contrast_M(op.chi_from_permittivity(eps, eps_bg))
    Mm = jm.mu_contrast(mu)
    return plan, Me, Mm


# (6, 23, 11): the strip cross-section, circulant 45 x 24, whose complex64
# pass B runs the register kernel with the cross-section compiled in
@pytest.mark.parametrize("grid", [(5, 4, 3), (17, 6, 5), (33, 9, 4), (6, 23, 11)])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_jm_operator_and_rhs_match_oracle(grid, dtype):
    plan, Me, Mm = _plan(grid, 41)
    kappa = plan.info()["kappa"]
    Gh, Ch = _oracle_spectra(grid, kappa)
    u = np.concatenate([workloads.random_currents(grid, seed=42), workloads.random_currents(grid, seed=43)])
    x = torch.from_numpy(u.ravel()).to(dtype).cuda()
    y = torch.empty_like(x)
    vie.vie_jm_matvec(plan, x, y)
    b = torch.empty_like(x)
    vie.vie_jm_rhs_from_source(plan, x, b)
    torch.cuda.synchronize()
    y_ref = jm.matvec(Gh, Ch, grid, Me, Mm, u, kappa).ravel()
    assert rel_l2(y.cpu().numpy().astype(np.complex128), y_ref) <= TOL[dtype]
    nx, ny, nz = grid
    # right-hand side of impressed currents (w_e, w_m) = u
    ue, um = u[:3], u[3:]
    e_inc = op.apply_T(Gh, grid, ue) - ue - 1j * kappa * jm.apply_curl(Ch, grid, um)
    h_inc = op.apply_T(Gh, grid, um) - um + 1j * kappa * jm.apply_curl(Ch, grid, ue)
    b_ref = np.concatenate([Me[None] * e_inc, Mm[None] * h_inc]).ravel()
    assert rel_l2(b.cpu().numpy().astype(np.complex128), b_ref) <= TOL[dtype]
    # an electric source alone: the oracle's rhs_from_source
    src = np.concatenate([ue, np.zeros_like(ue)])
    xs = torch.from_numpy(src.ravel()).to(dtype).cuda()
    vie.vie_jm_rhs_from_source(plan, xs, b)
    torch.cuda.synchronize()
    b_ref = jm.rhs_from_source(Gh, Ch, grid, Me, Mm, ue, kappa).ravel()
    assert rel_l2(b.cpu().numpy().astype(np.complex128), b_ref) <= TOL[dtype]
    plan.close()


# planes whose two-buffer pass B does not fit in shared memory (complex128
# 60 x 24, complex64 100 x 24): the one-buffer kernel with a line per warp
@pytest.mark.parametrize("grid,dtype", [((3, 30, 12), torch.complex128), ((3, 50, 12), torch.complex64)])
def test_jm_large_plane_matches_oracle(grid, dtype):
    plan, Me, Mm = _plan(grid, 44)
    kappa = plan.info()["kappa"]
    Gh, Ch = _oracle_spectra(grid, kappa)
    u = np.concatenate([workloads.random_currents(grid, seed=45), workloads.random_currents(grid, seed=46)])
    x = torch.from_numpy(u.ravel()).to(dtype).cuda()
    y = torch.empty_like(x)
    vie.vie_jm_matvec(plan, x, y)
    torch.cuda.synchronize()
    y_ref = jm.matvec(Gh, Ch, grid, Me, Mm, u, kappa).ravel()
    assert rel_l2(y.cpu().numpy().astype(np.complex128), y_ref) <= TOL[dtype]
    plan.close()


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-5)])
def test_jm_full_size_reciprocity(dtype, tol):
    """The full 600 x 23 x 11 guide with electric and magnetic contrast and
    dense random inputs, a property that holds at any size: the JM-VIE's
    integral part L = [[N, -j kappa K], [j kappa K, N]] (Sec. 3) has N
    symmetric and the curl part K symmetric as a bilinear form (its kernel is
    odd), so L^T = S L S with S = diag(I, -I) (reciprocity with magnetic
    currents): v^T L u = (S u)^T L (S v).  L w is recovered as
    diag(M_eps, M_mu)^{-1} (w - A w)."""
    wl = workloads.waveguide()
    nx, ny, nz = grid = wl.grid
    rng = np.random.Generator(np.random.PCG64(64))
    eps = wl.eps_bg * (2.0 + 3.0 * rng.random((nz, ny, nx))) - 1j * rng.random((nz, ny, nx))
    mu = 2.0 + rng.random((nz, ny, nx)) - 0.5j * rng.random((nz, ny, nx))
    plan = vie.vie_plan_create(grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, eps)
    vie.vie_set_permeability(plan, mu)
    Me = op.contrast_M(op.chi_from_permittivity(eps, wl.eps_bg))
    Mm = jm.mu_contrast(mu)
    Mi = np.concatenate([np.broadcast_to(1.0 / Me, (3, nz, ny, nx)), np.broadcast_to(1.0 / Mm, (3, nz, ny, nx))]).ravel()
    np_dtype = np.complex128 if dtype == torch.complex128 else np.complex64
    n3 = 3 * nx * ny * nz
    sgn = np.concatenate([np.ones(n3), -np.ones(n3)])

    def L(w):
        x = torch.from_numpy(w).to(dtype).cuda()
        y = torch.empty_like(x)
        vie.vie_jm_matvec(plan, x, y)
        torch.cuda.synchronize()
        return (w - y.cpu().numpy().astype(np.complex128)) * Mi

    u = np.concatenate([workloads.random_currents(grid, seed=65), workloads.random_currents(grid, seed=66)]).ravel()
    v = np.concatenate([workloads.random_currents(grid, seed=67), workloads.random_currents(grid, seed=68)]).ravel()
    u = u.astype(np_dtype).astype(np.complex128)
    v = v.astype(np_dtype).astype(np.complex128)
    Lu, LSv = L(u), L(sgn * v)
    a, b = np.dot(v, Lu), np.dot(sgn * u, LSv)
    assert abs(a - b) <= tol * np.linalg.norm(v) * np.linalg.norm(Lu), (a, b)
    plan.close()


def test_jm_zero_permeability_contrast_decouples():
    """mu_r = 1 and zero magnetic input: the electric half of the JM operator
    is the J-VIE operator, the magnetic half is M_mu (...) = 0 plus u_m = 0."""
    grid = (12, 5, 4)
    plan = vie.vie_plan_create(grid, 0.03, K0, 2.085)
    vie.vie_set_permittivity(plan, workloads.random_permittivity(grid, seed=5))
    vie.vie_set_permeability(plan, np.ones((4, 5, 12), complex))
    ue = workloads.random_currents(grid, seed=6)
    u = torch.from_numpy(np.concatenate([ue, np.zeros_like(ue)]).ravel()).cuda()
    y = torch.empty_like(u)
    vie.vie_jm_matvec(plan, u, y)
    yj = torch.empty(3 * plan.n_vox, dtype=torch.complex128, device="cuda")
    vie.vie_matvec(plan, u[:3 * plan.n_vox].contiguous(), yj)
    torch.cuda.synchronize()
    assert rel_l2(y[:3 * plan.n_vox].cpu().numpy(), yj.cpu().numpy()) <= 1e-13
    assert torch.count_nonzero(y[3 * plan.n_vox:]).item() == 0


@pytest.mark.parametrize("mode,tol", [(vie.VIE_SOLVE_FP64, 1e-11), (vie.VIE_SOLVE_MIXED, 1e-8)])
def test_jm_solve_matches_dense_lu(mode, tol):
    grid = (4, 3, 3)
    plan, Me, Mm = _plan(grid, 51, h=0.05)
    kappa = plan.info()["kappa"]
    A = jm.dense_A(grid, kappa, Me, Mm)
    rhs = np.concatenate([workloads.random_currents(grid, seed=52), workloads.random_currents(grid, seed=53)])
    x_lu = np.linalg.solve(A, rhs.ravel())
    b = torch.from_numpy(rhs.ravel()).cuda()
    x = torch.zeros_like(b)
    info = vie.vie_jm_solve(plan, b, x, tol, mode=mode, restart=40)
    assert info["converged"] and info["residual"] <= tol
    assert rel_l2(x.cpu().numpy(), x_lu) <= np.linalg.cond(A) * tol
    # host buffers
    xh = np.zeros_like(rhs.ravel())
    info = vie.vie_jm_solve(plan, rhs.ravel().copy(), xh, tol, mode=mode, restart=40)
    assert info["converged"] and rel_l2(xh, x_lu) <= np.linalg.cond(A) * tol


def test_jm_zero_backscatter_on_gpu():
    """An 8^3-voxel cube with eps_r = mu_r, solved on the GPU: the far field
    towards the source vanishes (zero-backscatter theorem), to the solver's
    precision; with mu_r = 1 it does not."""
    grid = (8, 8, 8)
    h = 0.4 / 8
    out = []
    for mu in (3.0 - 0.5j, 1.0 + 0j):
        plan = vie.vie_plan_create(grid, h, K0, 1.0)
        vie.vie_set_permittivity(plan, np.full((8, 8, 8), 3.0 - 0.5j))
        vie.vie_set_permeability(plan, np.full((8, 8, 8), mu))
        kappa = plan.info()["kappa"]
        Me = np.full((8, 8, 8), op.contrast_M(2.0 - 0.5j))
        Mm = np.full((8, 8, 8), jm.mu_contrast(mu))
        b = torch.from_numpy(jm.rhs_plane_wave_x(grid, kappa, Me, Mm).ravel()).cuda()
        x = torch.zeros_like(b)
        info = vie.vie_jm_solve(plan, b, x, 1e-11, mode=vie.VIE_SOLVE_FP64, restart=60)
        assert info["converged"]
        u = x.cpu().numpy().reshape(6, 8, 8, 8)
        C = op.voxel_coords(grid) + 0.5
        F = []
        for s in (np.array([0.0, 0.0, -1.0]), np.array([0.0, 0.0, 1.0])):
            ph = np.exp(1j * kappa * (C @ s))
            We = u[:3].reshape(3, -1) @ ph
            Wm = u[3:].reshape(3, -1) @ ph
            F.append(We - s * (s @ We) - np.cross(s, Wm))
        out.append(np.linalg.norm(F[0]) / np.linalg.norm(F[1]))
        plan.close()
    assert out[0] < 1e-8 and out[1] > 1e-2, out


def _guide_R(L_vox, matched, body=40, degree=2):
    """R of the axis field of a strip guide with a graded absorber of L_vox
    voxels against the same model with a 90-voxel absorber (the round-trip
    target 1e-10 with D = 2, or D = 4 with matched magnetic loss, Sec. 4.3)."""
    fields = {}
    for L in (L_vox, 90):
        wl = workloads.waveguide(nx=body + L, absorber_len_um=L * 0.02, degree=degree, src_x_um=0.2)
        ab = wl.absorbers[0]
        D = 4.0 if matched else 2.0
        e2 = op.eps2_max_from_rrt(1e-10, degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core, D=D)
        absorbers = [dict(x0=ab.x0, length=ab.length, degree=degree, eps2_max=e2)]
        plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
        vie.vie_set_permittivity(plan, wl.eps, absorbers)
        n3 = 3 * plan.n_vox
        if matched:
            vie.vie_set_permeability(plan, None)
            src = torch.zeros(2 * n3, dtype=torch.complex128, device="cuda")
            src[:n3] = torch.from_numpy(wl.src.ravel()).cuda()
            b = torch.empty_like(src)
            vie.vie_jm_rhs_from_source(plan, src, b)
            x = torch.zeros_like(b)
            info = vie.vie_jm_solve(plan, b, x, 1e-9, mode=vie.VIE_SOLVE_MIXED, restart=60)
            xe = x[:n3].contiguous()
        else:
            src = torch.from_numpy(wl.src.ravel()).cuda()
            b = torch.empty_like(src)
            vie.vie_rhs_from_source(plan, src, b)
            xe = torch.zeros_like(b)
            info = vie.vie_solve(plan, b, xe, 1e-9, mode=vie.VIE_SOLVE_MIXED, restart=60)
        assert info["converged"]
        fields[L] = vie.vie_axis_field(plan, xe, body)
        plan.close()
    return vie.vie_reflection(fields[90], fields[L_vox])


def test_matched_absorber_reflects_less():
    """Sec. 5.1: matching the impedance with magnetic loss (mu'' = eps''/eps')
    lowers the reflection of the same-length absorber (the paper reports about
    a factor 100 for long absorbers; here a qualitative factor)."""
    R_e = _guide_R(30, matched=False)
    R_em = _guide_R(30, matched=True)
    print(f"R electric {R_e:.3e}, electric + magnetic {R_em:.3e}, ratio {R_e / R_em:.1f}")
    assert R_em < R_e / 3, (R_e, R_em)
