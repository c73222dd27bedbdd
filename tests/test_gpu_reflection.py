"""Reflection coefficient and fields from actual solves (Sec. 5.1): the GPU
solves a strip guide with a short graded absorber and the same guide with a
long reference absorber, forms the axis fields (Sec. 3, E = J / (c_e chi))
and R = sum |E_ref - E_L|^2 / sum |E_ref|^2 over the guide before the
absorbers; the FP64 oracle does the same with its own operator, GMRES and
metrics.  Both in complex128 GMRES and in mixed precision.

Tolerances (stated for the benchmark's accuracy targets):
* R: |R_gpu - R_oracle| <= 0.05 R_oracle + 1e-11;
* field (whole solution vector, relative L2): <= 1e-9 for complex128 GMRES
  to 1e-11, <= 1e-5 for mixed precision to 1e-6 (a solve to relative residual
  tol is within cond(A) tol of the exact solution; cond(A) of these short
  guides is O(10))."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle import gmres, greens, metrics
from oracle import operator as op
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu

BODY = 40            # voxels of guide before the absorber (0.8 um at h = 20 nm)
N_KEEP = BODY        # R is taken over the axis voxels with x_c < BODY


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def _guide(L_vox, degree=2):
    wl = workloads.waveguide(nx=BODY + L_vox, absorber_len_um=L_vox * 0.02, degree=degree, src_x_um=0.2)
    ab = wl.absorbers[0]
    e2 = op.eps2_max_from_rrt(1e-10, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
    return wl, [dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2)]


@pytest.fixture(scope="module")
def oracle_solutions():
    """Oracle solutions (complex128 GMRES to 1e-12) of the short-absorber
    guide and the reference guide, with their axis fields."""
    out = {}
    for key, L in (("L", 30), ("ref", 90)):
        wl, ab = _guide(L)
        chi = op.chi_from_permittivity(wl.eps, wl.eps_bg, ab)
        M = op.contrast_M(chi)
        Gh = op.green_spectrum(greens.octant_table(wl.kappa, wl.grid), wl.grid, tuple(2 * v for v in wl.grid))
        b = op.rhs_from_source(Gh, wl.grid, M, wl.src).ravel()
        x, info = gmres.gmres(lambda v: op.matvec(Gh, wl.grid, M, v).ravel(), b, tol=1e-12, restart=200,
                              maxiter=5000)
        assert info["converged"]
        out[key] = (x, metrics.axis_field(x, chi, N_KEEP))
    out["R"] = metrics.reflection_coefficient(out["ref"][1], out["L"][1])
    return out


def _gpu_solve(L, mode, tol):
    wl, ab = _guide(L)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, ab)
    src = torch.from_numpy(wl.src.ravel()).cuda()
    b = torch.empty_like(src)
    vie.vie_rhs_from_source(plan, src, b)
    x = torch.zeros_like(b)
    info = vie.vie_solve(plan, b, x, tol, mode=mode, restart=100)
    assert info["converged"] and info["residual"] <= tol, info
    e = vie.vie_axis_field(plan, x, N_KEEP)
    chi = op.chi_from_permittivity(wl.eps, wl.eps_bg, ab)
    return plan, x, e, chi


@pytest.mark.parametrize("mode,tol,field_tol", [(vie.VIE_SOLVE_FP64, 1e-11, 1e-9),
                                                (vie.VIE_SOLVE_MIXED, 1e-6, 1e-5)])
def test_reflection_and_fields_from_solves_match_oracle(oracle_solutions, mode, tol, field_tol):
    plan_l, x_l, e_l, chi_l = _gpu_solve(30, mode, tol)
    plan_r, x_r, e_r, _ = _gpu_solve(90, mode, tol)
    err_l = rel_l2(x_l.cpu().numpy(), oracle_solutions["L"][0])
    err_r = rel_l2(x_r.cpu().numpy(), oracle_solutions["ref"][0])
    R = vie.vie_reflection(e_r, e_l)
    R_ref = oracle_solutions["R"]
    print(f"mode {mode} tol {tol}: field errors {err_l:.2e} {err_r:.2e}; R gpu {R:.6e} oracle {R_ref:.6e}")
    assert err_l <= field_tol and err_r <= field_tol, (err_l, err_r)
    assert abs(R - R_ref) <= 0.05 * R_ref + 1e-11, (R, R_ref)
    # the axis field the GPU forms equals the oracle's formula on the GPU solution
    np.testing.assert_allclose(e_l.cpu().numpy(), metrics.axis_field(x_l.cpu().numpy(), chi_l, N_KEEP),
                               rtol=1e-13, atol=0)
    plan_l.close()
    plan_r.close()


def test_reflection_falls_with_absorber_length():
    """Physics sanity of the absorber path on the GPU (Sec. 4.3, 5.1): at
    fixed round-trip target a longer absorber reflects less (the transition
    reflection falls with L), and R is well below 1."""
    _, _, e_ref, _ = _gpu_solve(90, vie.VIE_SOLVE_MIXED, 1e-7)
    Rs = []
    for L in (15, 30):
        _, _, e_l, _ = _gpu_solve(L, vie.VIE_SOLVE_MIXED, 1e-7)
        Rs.append(vie.vie_reflection(e_ref, e_l))
    assert Rs[1] < Rs[0], Rs
    assert Rs[1] < 1e-2, Rs
    assert math.isfinite(Rs[0])
