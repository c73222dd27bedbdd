"""Failure detection made on the host (no GPU fault is provoked): non-finite
contrast input, non-finite network parameters uploaded from the host (the
network's output is replaced and the solver drops it and still converges),
the host-side solve timeout, and solves on host buffers and with caller
weights through the C ABI."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu
K0 = 2 * math.pi / 1.55


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def _guide_plan(nx=60):
    wl = workloads.waveguide(nx=nx, absorber_len_um=0.4, src_x_um=0.2)
    ab = [dict(x0=nx - 20.0, length=20.0, degree=2, eps2_max=2.0)]
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, ab)
    src = torch.from_numpy(wl.src.ravel()).cuda()
    b = torch.empty_like(src)
    vie.vie_rhs_from_source(plan, src, b)
    return plan, b


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), complex(0.0, float("nan"))])
def test_non_finite_contrast_is_rejected(bad):
    grid = (6, 5, 4)
    plan = vie.vie_plan_create(grid, 0.03, K0, 2.085)
    chi = np.full((4, 5, 6), 0.5 + 0.1j)
    chi[2, 3, 1] = bad
    with pytest.raises(vie.VieError) as ei:
        vie.vie_set_contrast(plan, chi)
    assert ei.value.status == 6          # VIE_ERR_NONFINITE
    eps = np.full((4, 5, 6), 4.0 + 0j)
    eps[0, 0, 0] = bad
    with pytest.raises(vie.VieError) as ei:
        vie.vie_set_permittivity(plan, eps)
    assert ei.value.status == 6


def test_non_finite_network_parameters_fall_back_to_plain_gmres():
    """Parameters with a NaN uploaded from the host (in the output layer: a
    NaN in a hidden layer is cut off by the next ReLU): every application
    replaces the output by its input and flags it (vie_net_status = 1); a
    solve with that network drops it (info fallback) and still converges to
    the same solution as the unpreconditioned solve."""
    plan, b = _guide_plan()
    params = np.zeros(vie.vie_net_param_count(), np.float32)
    params[:1000] = np.random.default_rng(1).standard_normal(1000).astype(np.float32) * 0.05
    params[-1] = np.nan                     # bias of the last output channel
    net = vie.vie_net_create(params)
    v = torch.from_numpy(workloads.random_currents((60, 23, 11), seed=3).astype(np.complex64).ravel()).cuda()
    z = torch.empty_like(v)
    vie.vie_net_apply(net, plan, v, z)
    torch.cuda.synchronize()
    assert vie.vie_net_status(net, clear=True) == 1
    assert torch.equal(z, v)
    x0 = torch.zeros_like(b)
    ref = vie.vie_solve(plan, b, x0, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30)
    vie.vie_set_preconditioner(plan, params)          # the plan's own copy, from host weights
    x1 = torch.zeros_like(b)
    info = vie.vie_solve(plan, b, x1, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, use_preconditioner=True)
    assert info["converged"] and info["fallback"] and info["residual"] <= 1e-6
    assert rel_l2(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-4
    assert ref["converged"]
    vie.vie_set_preconditioner(plan, None)
    with pytest.raises(vie.VieError):                  # nothing set any more
        vie.vie_solve(plan, b, x1, 1e-6, use_preconditioner=True)


def test_weights_preconditioner_matches_network_object():
    """vie_set_preconditioner(plan, weights, bytes) builds the same
    preconditioner as a network object with those parameters."""
    plan, b = _guide_plan()
    params = np.zeros(vie.vie_net_param_count(), np.float32)
    params[:] = np.random.default_rng(2).standard_normal(params.size).astype(np.float32) * 1e-3
    net = vie.vie_net_create(params)
    vie.vie_set_preconditioner_net(plan, net)
    xa = torch.zeros_like(b)
    ia = vie.vie_solve(plan, b, xa, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, use_preconditioner=True)
    vie.vie_set_preconditioner(plan, params)
    xb = torch.zeros_like(b)
    ib = vie.vie_solve(plan, b, xb, 1e-6, mode=vie.VIE_SOLVE_MIXED, restart=30, use_preconditioner=True)
    assert abs(ia["iterations"] - ib["iterations"]) <= 1 and ia["fallback"] == ib["fallback"]
    assert ib["converged"] and rel_l2(xb.cpu().numpy(), xa.cpu().numpy()) <= 1e-5
    with pytest.raises(vie.VieError) as ei:
        vie.vie_set_preconditioner(plan, params[:-1])
    assert ei.value.status == 1


def test_solve_timeout_returns_the_current_iterate():
    plan, b = _guide_plan()
    x = torch.zeros_like(b)
    info = vie.vie_solve(plan, b, x, 1e-10, mode=vie.VIE_SOLVE_FP64, restart=30, timeout_s=1e-9,
                         raise_on_not_converged=False)
    assert info["status"] == 5 and not info["converged"]        # VIE_ERR_TIMEOUT
    assert "exceeded" in vie.vie_last_error()
    assert np.isfinite(x.cpu().numpy()).all()
    # the plan stays usable: the same solve without the limit converges
    info = vie.vie_solve(plan, b, x, 1e-8, mode=vie.VIE_SOLVE_FP64, restart=30)
    assert info["converged"]


def test_solve_on_host_buffers_matches_device_solve():
    plan, b = _guide_plan()
    xd = torch.zeros_like(b)
    idev = vie.vie_solve(plan, b, xd, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30)
    bh = b.cpu().numpy().copy()
    xh = np.zeros_like(bh)
    ihost = vie.vie_solve(plan, bh, xh, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30)
    assert ihost["converged"] and abs(ihost["iterations"] - idev["iterations"]) <= 1
    assert rel_l2(xh, xd.cpu().numpy()) <= 1e-6
    # warm start from a host initial guess: no iterations needed
    iw = vie.vie_solve(plan, bh, xh, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30, x0_given=True)
    assert iw["converged"] and iw["iterations"] == 0
    # batch entry point on host buffers
    plan2, b2 = _guide_plan(nx=50)
    bs = [bh, b2.cpu().numpy().copy()]
    xs = [np.zeros_like(v) for v in bs]
    st, infos = vie.vie_solve_batch([plan, plan2], bs, xs, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30)
    assert st == 0 and all(i["converged"] for i in infos)
    assert rel_l2(xs[0], xd.cpu().numpy()) <= 1e-6


def test_grid_barrier_wait_runs_out_and_reports():
    """The solver's cooperative Gram-Schmidt step separates its phases with a
    grid barrier whose waits are bounded: with one block missing, the others
    give up after the limit and set the abort word (which the solver reports
    as VIE_ERR_TIMEOUT); with every block present the barrier completes.
    The context stays usable."""
    import time
    t0 = time.perf_counter()
    assert vie.vie_probe_grid_barrier(3, 50.0) is True
    assert time.perf_counter() - t0 < 30.0
    assert vie.vie_probe_grid_barrier(-1, 50.0) is False
    x = torch.ones(8, device="cuda")
    assert float(x.sum().item()) == 8.0
