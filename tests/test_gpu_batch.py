"""Batched problems: shared-spectrum plans, the grouped operator and the
batched solver, checked against single-problem calls and the oracle."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import oracle_matvec, rel_l2
from oracle import operator as op
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu
K0 = 2 * math.pi / 1.55


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def _guide(nx, L_vox, degree, e2, seed):
    wl = workloads.waveguide(nx=nx, absorber_len_um=L_vox * 0.02, src_x_um=0.2)
    ab = [dict(x0=float(nx - L_vox), length=float(L_vox), degree=degree, eps2_max=e2)]
    return wl, ab


def test_clone_shares_spectrum_and_outlives_base():
    wl, ab = _guide(50, 15, 2, 2.0, 1)
    base = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    clone = vie.vie_plan_clone(base)
    vie.vie_set_permittivity(clone, wl.eps, ab)
    ref = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(ref, wl.eps, ab)
    x = torch.from_numpy(workloads.random_currents(wl.grid, seed=3).ravel()).cuda()
    base.close()                       # the clone keeps the shared spectra alive
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    vie.vie_matvec(clone, x, y1)
    vie.vie_matvec(ref, x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_grouped_operator_equals_single_calls(dtype):
    plans, xs = [], []
    for k, nx in enumerate((40, 60, 40, 60, 40)):
        wl, ab = _guide(nx, 10 + k, k % 4, 0.5 + k, k)
        p = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
        vie.vie_set_permittivity(p, wl.eps, ab)
        plans.append(p)
        xs.append(torch.from_numpy(workloads.random_currents(wl.grid, seed=10 + k).ravel()).to(dtype).cuda())
    ys = [torch.empty_like(x) for x in xs]
    vie.vie_matvec_batch(plans, xs, ys)
    for p, x, y in zip(plans, xs, ys):
        y1 = torch.empty_like(x)
        vie.vie_matvec(p, x, y1)
        torch.cuda.synchronize()
        assert torch.equal(y, y1)


@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_grouped_operator_large_planes(dtype):
    """Three plans whose y-z plane takes the split pass B (4 x 200 x 12:
    circulant 8 x 400 x 24), grouped in one launch per pass: equal to single
    calls bit for bit and to the oracle."""
    grid = (4, 200, 12)
    base = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    plans = [base, vie.vie_plan_clone(base), vie.vie_plan_clone(base)]
    xs, Ms = [], []
    for k, p in enumerate(plans):
        eps = workloads.random_permittivity(grid, seed=90 + k)
        vie.vie_set_permittivity(p, eps)
        Ms.append(op.contrast_M(op.chi_from_permittivity(eps, 2.085)))
        xs.append(torch.from_numpy(workloads.random_currents(grid, seed=95 + k).ravel()).to(dtype).cuda())
    ys = [torch.empty_like(x) for x in xs]
    vie.vie_matvec_batch(plans, xs, ys)
    kappa = base.info()["kappa"]
    tol = 1e-12 if dtype == torch.complex128 else 2e-6
    for p, x, y, M in zip(plans, xs, ys, Ms):
        y1 = torch.empty_like(x)
        vie.vie_matvec(p, x, y1)
        torch.cuda.synchronize()
        assert torch.equal(y, y1)
        ref = oracle_matvec(grid, kappa, M, x.cpu().numpy().astype(np.complex128).reshape(3, 12, 200, 4)).ravel()
        assert rel_l2(y.cpu().numpy().astype(np.complex128), ref) <= tol


@pytest.mark.parametrize("resident", [False, True])
@pytest.mark.parametrize("mode,tol", [(vie.VIE_SOLVE_MIXED, 1e-6), (vie.VIE_SOLVE_FP64, 1e-8)])
def test_batched_solve_matches_single_solves_and_oracle(mode, tol, resident):
    """Four uneven guides solved together (the host loop between cycles, or
    the whole solve as one graph launch with device-side decisions) against
    single solves and the oracle's residual."""
    specs = [(60, 15, 0, 0.5), (80, 20, 2, 2.0), (60, 25, 3, 2.0), (100, 30, 1, 0.5)]
    plans, bs, wls = [], [], []
    for nx, L, d, e2 in specs:
        wl, ab = _guide(nx, L, d, e2, nx)
        p = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
        vie.vie_set_permittivity(p, wl.eps, ab)
        src = torch.from_numpy(wl.src.ravel()).cuda()
        b = torch.empty_like(src)
        vie.vie_rhs_from_source(p, src, b)
        plans.append(p)
        bs.append(b)
        wls.append((wl, ab))
    xs = [torch.zeros_like(b) for b in bs]
    st, infos = vie.vie_solve_batch(plans, bs, xs, tol, mode=mode, restart=40, resident=resident)
    assert st == 0
    for p, b, x, info, (wl, ab) in zip(plans, bs, xs, infos, wls):
        assert info["converged"] and info["residual"] <= tol
        x1 = torch.zeros_like(b)
        i1 = vie.vie_solve(p, b, x1, tol, mode=mode, restart=40)
        assert i1["converged"]
        assert rel_l2(x.cpu().numpy(), x1.cpu().numpy()) <= 100 * tol
        # true residual with the oracle operator
        M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg, ab))
        r = oracle_matvec(wl.grid, wl.kappa, M, x.cpu().numpy().reshape(3, *wl.grid[::-1])).ravel() - b.cpu().numpy()
        assert np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy()) <= 2 * tol


def test_resident_solve_time_limit_and_single_problem():
    """The device-resident solve checks its time limit on the device at each
    refinement step: a limit of a microsecond stops a batch of two with
    VIE_ERR_TIMEOUT (x holds the iterate reached); a single problem solved
    resident takes the same steps as the host loop and reaches the same x."""
    specs = [(60, 15, 2, 2.0), (80, 20, 2, 2.0)]
    plans, bs = [], []
    for nx, L, d, e2 in specs:
        wl, ab = _guide(nx, L, d, e2, nx)
        p = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
        vie.vie_set_permittivity(p, wl.eps, ab)
        src = torch.from_numpy(wl.src.ravel()).cuda()
        b = torch.empty_like(src)
        vie.vie_rhs_from_source(p, src, b)
        plans.append(p)
        bs.append(b)
    xs = [torch.zeros_like(b) for b in bs]
    st, infos = vie.vie_solve_batch(plans, bs, xs, 1e-10, mode=vie.VIE_SOLVE_MIXED, restart=30, resident=True,
                                    timeout_s=1e-6, raise_on_not_converged=False)
    assert st == 5, st
    for info in infos:
        assert not info["converged"]
    x1 = torch.zeros_like(bs[0])
    x2 = torch.zeros_like(bs[0])
    i1 = vie.vie_solve(plans[0], bs[0], x1, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30, resident=True)
    i2 = vie.vie_solve(plans[0], bs[0], x2, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30)
    assert i1["converged"] and i2["converged"]
    assert i1["iterations"] == i2["iterations"]
    assert rel_l2(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-6
