"""GPU block-circulant preconditioner (Sec. 5.4) against the FP64 oracle
(oracle/circulant.py): z = W^{-1} v on grids with one and several LU panels,
ragged solve blocks and x lengths that are not 5-smooth; solves with it."""
import functools
import math

import numpy as np
import pytest
import torch

from oracle import circulant as circ
from oracle import operator as op
from paper_1803_06237_gb300 import build, learned, vie, workloads

pytestmark = pytest.mark.gpu
K0 = 2 * math.pi / 1.55
H = 0.02
EPS_BG = 2.085


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


@functools.lru_cache(maxsize=None)
def _oracle_what(grid, seed):
    """The oracle's W_hat(w) blocks (and their largest condition number) for
    the random contrast of _plan_with_contrast(grid, seed)."""
    chi = op.chi_from_permittivity(workloads.random_permittivity(grid, seed=seed), EPS_BG)
    kappa = K0 * math.sqrt(EPS_BG) * H
    What = circ.blocks_hat(circ.circulant_blocks(grid, kappa, op.contrast_M(chi)))
    return What, max(np.linalg.cond(What[w]) for w in range(grid[0]))


def _plan_with_contrast(grid, seed):
    plan = vie.vie_plan_create(grid, H, K0, EPS_BG)
    chi = op.chi_from_permittivity(workloads.random_permittivity(grid, seed=seed), EPS_BG)
    vie.vie_set_contrast(plan, chi)
    return plan, op.contrast_M(chi)


# (nx, ny, nz): R = 3 ny nz unknowns per slice; nb = 32 panels; nx with
# prime factors 7, 11, 13 (FFT stages that sum those radices directly):
# 7, 13, 350 = 2 5^2 7, 550 = 2 5^2 11, 91 = 7 13; (6, 23, 11): the strip's
# cross-section, R = 759 unknowns per slice (24 panels, a ragged last one),
# the factorisation of the benchmark guide
@pytest.mark.parametrize("grid", [(7, 3, 2), (13, 4, 3), (20, 6, 2), (24, 8, 5), (9, 11, 4), (350, 3, 2),
                                  (550, 2, 2), (91, 5, 3), (6, 23, 11)])
@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("fp16", [False, True])
def test_apply_matches_oracle(grid, dtype, fp16):
    """complex64 factors: rounding error times the blocks' condition number;
    complex-half factors (unit roundoff 2^-11): the same bound with that
    roundoff."""
    plan, M = _plan_with_contrast(grid, 3)
    c = vie.vie_circulant_create(plan, vie.VIE_CIRC_FP16_FACTORS if fp16 else vie.VIE_CIRC_DEFAULT)
    What, cond = _oracle_what(grid, 3)
    v = workloads.random_currents(grid, seed=4).astype(dtype)
    vd = torch.from_numpy(v.ravel()).cuda()
    zd = torch.empty_like(vd)
    vie.vie_circulant_apply(c, vd, zd)
    torch.cuda.synchronize()
    z = zd.cpu().numpy().reshape(3, grid[2], grid[1], grid[0]).astype(np.complex128)
    z_ref = circ.apply_inverse(What, v.astype(np.complex128))
    tol = (4e-3 if fp16 else 2e-6) * cond
    assert np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref) < tol


def test_zero_contrast_is_identity():
    grid = (12, 3, 2)
    plan = vie.vie_plan_create(grid, H, K0, EPS_BG)
    vie.vie_set_contrast(plan, np.zeros((grid[2], grid[1], grid[0]), np.complex128))
    c = vie.vie_circulant_create(plan)
    v = torch.from_numpy(workloads.random_currents(grid, seed=5).astype(np.complex64).ravel()).cuda()
    z = torch.empty_like(v)
    vie.vie_circulant_apply(c, v, z)
    torch.cuda.synchronize()
    assert (torch.linalg.vector_norm(z - v) / torch.linalg.vector_norm(v)).item() < 1e-5


def test_stale_after_contrast_change():
    grid = (8, 3, 2)
    plan, _ = _plan_with_contrast(grid, 6)
    c = vie.vie_circulant_create(plan)
    chi = op.chi_from_permittivity(workloads.random_permittivity(grid, seed=7), EPS_BG)
    vie.vie_set_contrast(plan, chi)
    v = torch.zeros(3 * plan.n_vox, dtype=torch.complex64, device="cuda")
    with pytest.raises(vie.VieError):
        vie.vie_circulant_apply(c, v, torch.empty_like(v))


def test_other_plan_rejected():
    grid = (8, 3, 2)
    plan_a, _ = _plan_with_contrast(grid, 8)
    plan_b, _ = _plan_with_contrast(grid, 9)
    c = vie.vie_circulant_create(plan_a)
    with pytest.raises(vie.VieError):
        vie.vie_set_circulant_preconditioner(plan_b, c)


def _guide_problem(nx, absorber_um):
    wl = workloads.waveguide(nx=nx, absorber_len_um=absorber_um, src_x_um=min(1.0, nx * H / 4))
    return learned.setup_problem(wl)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_preconditioned_solve_small_guide(mode):
    """A 160 x 23 x 11 strip guide: the preconditioned solve reaches the true
    residual 1e-6 in a fraction of the plain solve's steps, and both give the
    same solution."""
    plan, b = _guide_problem(160, 1.0)
    m = vie.VIE_SOLVE_FP64 if mode == "fp64" else vie.VIE_SOLVE_MIXED
    x0 = torch.zeros_like(b)
    i0 = vie.vie_solve(plan, b, x0, 1e-6, mode=m, restart=30)
    c = vie.vie_circulant_create(plan)
    vie.vie_set_circulant_preconditioner(plan, c)
    x1 = torch.zeros_like(b)
    i1 = vie.vie_solve(plan, b, x1, 1e-6, mode=m, restart=30, use_preconditioner=True)
    assert i0["converged"] and i1["converged"] and i1["residual"] <= 1e-6
    assert not i1["fallback"]
    assert i1["iterations"] * 4 <= i0["iterations"]
    assert (torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0)).item() < 1e-5
    vie.vie_set_circulant_preconditioner(plan, None)


@pytest.mark.parametrize("fp16", [False, True])
def test_full_size_guide_solve(fp16):
    """The 600 x 23 x 11 benchmark guide (R = 759 unknowns per slice, 24 LU
    panels): the preconditioned mixed solve converges to 1e-6 in few steps
    and agrees with the plain solve, with complex64 or complex-half factors."""
    plan, b = _guide_problem(600, 4.0)
    c = vie.vie_circulant_create(plan, vie.VIE_CIRC_FP16_FACTORS if fp16 else vie.VIE_CIRC_DEFAULT)
    info = vie.vie_circulant_info(c)
    assert info["device_bytes"] >= 600 * 759 * 759 * (4 if fp16 else 8)
    vie.vie_set_circulant_preconditioner(plan, c)
    x1 = torch.zeros_like(b)
    i1 = vie.vie_solve(plan, b, x1, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, use_preconditioner=True)
    assert i1["converged"] and i1["residual"] <= 1e-6 and not i1["fallback"]
    assert i1["iterations"] <= 80
    vie.vie_set_circulant_preconditioner(plan, None)
    x0 = torch.zeros_like(b)
    i0 = vie.vie_solve(plan, b, x0, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30)
    assert i0["converged"]
    assert (torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0)).item() < 1e-5


def test_batch_solve_with_per_plan_preconditioners():
    """Three uneven guides solved together, each with its own block-circulant
    preconditioner (complex-half factors): every problem converges and
    matches its plain solve."""
    plans, bs = [], []
    for nx, L in ((120, 0.6), (150, 1.0), (200, 1.4)):
        p, b = _guide_problem(nx, L)
        plans.append(p)
        bs.append(b)
    xs0 = [torch.zeros_like(b) for b in bs]
    st0, i0 = vie.vie_solve_batch(plans, bs, xs0, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30)
    circs = [vie.vie_circulant_create(p, vie.VIE_CIRC_FP16_FACTORS) for p in plans]
    for p, c in zip(plans, circs):
        vie.vie_set_circulant_preconditioner(p, c)
    xs1 = [torch.zeros_like(b) for b in bs]
    st1, i1 = vie.vie_solve_batch(plans, bs, xs1, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, use_preconditioner=True)
    assert st0 == 0 and st1 == 0
    for a, c, x0, x1 in zip(i0, i1, xs0, xs1):
        assert c["converged"] and c["residual"] <= 1e-6 and not c["fallback"]
        assert c["iterations"] * 2 <= a["iterations"]   # short guides: the guide ends weigh more
        assert (torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0)).item() < 1e-5
    for p in plans:
        vie.vie_set_circulant_preconditioner(p, None)
