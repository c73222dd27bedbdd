"""Training and use of the learned right preconditioner (host orchestration).

Every numerical step runs in libvie: the operator and the solver produce the
training pairs, and the network's forward, backward and Adam kernels train
it.  This module only chooses the problems, keeps the pairs and calls the
library in order.

Pairs: for a problem A x = b with solution x*, plain GMRES cycles (restart
``restart``, complex64 inner solves inside FP64 refinement) from x = 0 give
iterates x_k; each yields (r_k, e_k) with e_k = x* - x_k and r_k = A e_k
(complex64 operator), so A e_k = r_k holds by construction.  The
preconditioner is z = r + Net(r); the network is trained so that z matches
e_k (squared error relative to |e_k|^2, both scaled by the RMS of r_k).  The
identity (Net = 0) has loss |e_k - r_k|^2 / |e_k|^2, reported by
``identity_loss`` as the level training has to beat.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import vie, workloads


@dataclasses.dataclass
class Pair:
    plan: object
    r: object      # complex64 CUDA vector
    e: object


def _absorbers(wl):
    out = []
    for ab in wl.absorbers:
        e2 = ab.eps2_max if ab.eps2_max is not None else vie.vie_eps2_from_round_trip(
            ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
        out.append(dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2, direction=ab.direction))
    return out


def setup_problem(wl, base_plan=None):
    """Plan (a clone of base_plan when the grid matches), contrast and the
    right-hand side of the workload's source.  Returns (plan, b)."""
    import torch
    if base_plan is not None and tuple(base_plan.n) == tuple(wl.grid):
        plan = vie.vie_plan_clone(base_plan)
    else:
        plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, _absorbers(wl))
    src = torch.from_numpy(np.ascontiguousarray(wl.src.ravel())).cuda()
    b = torch.empty_like(src)
    vie.vie_rhs_from_source(plan, src, b)
    return plan, b


def make_pairs(seeds, grid=(160, 40, 11), restart=20, cycles=12, tol=1e-6):
    """Training pairs from plain solves of seeded random strip/bend guides."""
    import torch
    pairs = []
    base = None
    for seed in seeds:
        wl = workloads.random_guide(seed, *grid)
        plan, b = setup_problem(wl, base)
        if base is None:
            base = plan
        xs = torch.zeros_like(b)
        vie.vie_solve(plan, b, xs, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart, raise_on_not_converged=False)
        x = torch.zeros_like(b)
        for _ in range(cycles):
            vie.vie_solve(plan, b, x, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart, max_iters=restart,
                          max_outer=1, x0_given=True, raise_on_not_converged=False)
            e = (xs - x).to(torch.complex64)
            if torch.linalg.vector_norm(e).item() == 0.0:
                break
            r = torch.empty_like(e)
            vie.vie_matvec(plan, e, r)
            pairs.append(Pair(plan, r, e))
    return pairs


def make_pairs_many(seeds, grid=(160, 40, 11), restart=10, cycles=20, tol=1e-6):
    """make_pairs for many problems with bounded device memory: one plan
    solves the problems in turn (its permittivity reset for each, so one
    solver workspace serves all), and each problem keeps a clone of it that
    holds only its contrast and operator workspace, which the network reads
    chi from during training.  Returns (pairs, solver plan)."""
    import torch
    pairs = []
    solver = None
    for seed in seeds:
        wl = workloads.random_guide(seed, *grid)
        if solver is None:
            solver, b = setup_problem(wl)
        else:
            vie.vie_set_permittivity(solver, wl.eps, _absorbers(wl))
            src = torch.from_numpy(np.ascontiguousarray(wl.src.ravel())).cuda()
            b = torch.empty_like(src)
            vie.vie_rhs_from_source(solver, src, b)
        keep = vie.vie_plan_clone(solver)
        vie.vie_set_permittivity(keep, wl.eps, _absorbers(wl))
        xs = torch.zeros_like(b)
        vie.vie_solve(solver, b, xs, tol, mode=vie.VIE_SOLVE_MIXED, restart=30, raise_on_not_converged=False)
        x = torch.zeros_like(b)
        for _ in range(cycles):
            vie.vie_solve(solver, b, x, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart, max_iters=restart,
                          max_outer=1, x0_given=True, raise_on_not_converged=False)
            e = (xs - x).to(torch.complex64)
            if torch.linalg.vector_norm(e).item() <= 1e-5 * torch.linalg.vector_norm(xs).item():
                break
            r = torch.empty_like(e)
            vie.vie_matvec(keep, e, r)
            pairs.append(Pair(keep, r, e))
    return pairs, solver


def mean_loss(net, pairs) -> float:
    """Mean loss of the network over pairs (gradients are accumulated and
    then cleared)."""
    vals = [vie.vie_net_accumulate(net, p.plan, p.r, p.e) for p in pairs]
    vie.vie_net_zero_grad(net)
    return float(np.mean(vals))


def identity_loss(pairs) -> float:
    """Mean of |e - r|^2 / |e|^2 over the pairs: the loss of z = r."""
    import torch
    vals = [(torch.linalg.vector_norm(p.e - p.r) ** 2 / torch.linalg.vector_norm(p.e) ** 2).item() for p in pairs]
    return float(np.mean(vals))


def train(net, pairs, steps, lr=1e-3, batch=4, seed=0, log_every=0):
    """Adam on mini-batches of pairs; returns the per-step mean loss."""
    rng = np.random.default_rng(seed)
    losses = []
    for step in range(steps):
        vie.vie_net_zero_grad(net)
        idx = rng.choice(len(pairs), size=min(batch, len(pairs)), replace=False)
        tot = 0.0
        for i in idx:
            p = pairs[i]
            tot += vie.vie_net_accumulate(net, p.plan, p.r, p.e)
        vie.vie_net_adam_step(net, lr, 1.0 / len(idx))
        losses.append(tot / len(idx))
        if log_every and step % log_every == 0:
            print(f"step {step} loss {losses[-1]:.4f}", flush=True)
    return losses
