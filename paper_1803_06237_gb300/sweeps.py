"""Parameter studies of Sec. 5 on the GPU (host orchestration only: every
solve, field and metric runs in libvie).

* ``rl_sweep``: the absorber-length study of Sec. 5.1 on the 13.5 um strip
  (810 x 30 x 12 voxels of 50/3 nm): for each monomial degree d and length L
  the reflection coefficient R(L) = |E_inf - E_L|^2 / |E_inf|^2 along the
  centre axis of the guide, E_inf from the longest absorber, and the slope of
  log R against log L, which Sec. 4.3 predicts to approach -2 (d + 1); with
  ``matched`` the absorbers also carry the matched magnetic loss of Sec. 4.2
  (JM-VIE), which Sec. 5.1 reports to lower R by about a factor 100.
* ``bragg_sweep``: the transmission spectrum of the N-period Bragg grating of
  Sec. 5.2: one plan per wavelength (the spectra depend on k), the
  wavelengths solved together through the batch path, T(lambda) = sum |E|^2
  over a voxel plane behind the grating.

Both precondition with the block-circulant matrix of Sec. 5.4 (complex-half
factors) and solve in mixed precision to a true FP64 residual ``tol``.
"""
from __future__ import annotations

import time

import numpy as np

from . import learned, vie, workloads


def _solve(wl, tol, restart=30, factors_fp16=True):
    """Plan, contrast, right-hand side, block-circulant preconditioner and a
    mixed-precision solve of one workload.  Returns (plan, x, info)."""
    import torch
    plan, b = learned.setup_problem(wl)
    c = vie.vie_circulant_create(plan, vie.VIE_CIRC_FP16_FACTORS if factors_fp16 else vie.VIE_CIRC_DEFAULT)
    vie.vie_set_circulant_preconditioner(plan, c)
    x = torch.zeros_like(b)
    info = vie.vie_solve(plan, b, x, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart, use_preconditioner=True,
                         raise_on_not_converged=False)
    vie.vie_set_circulant_preconditioner(plan, None)
    c.close()
    return plan, x, info


def _solve_matched(wl, tol, restart=60):
    """The same strip with magnetic loss matched to the electric one (Sec. 4.2,
    mu'' = eps''/eps'), the round-trip target met with D = 4 (Sec. 4.3): the
    JM-VIE driven by the electric sheet, mixed precision, no preconditioner.
    Returns (plan, electric half of the solution, info)."""
    import torch
    ab = wl.absorbers[0]
    e2 = vie.vie_eps2_from_round_trip(ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core, 4.0)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, [dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2)])
    vie.vie_set_permeability(plan, None)
    n3 = 3 * plan.n_vox
    src = torch.zeros(2 * n3, dtype=torch.complex128, device="cuda")
    src[:n3] = torch.from_numpy(np.ascontiguousarray(wl.src.ravel())).cuda()
    b = torch.empty_like(src)
    vie.vie_jm_rhs_from_source(plan, src, b)
    x = torch.zeros_like(b)
    info = vie.vie_jm_solve(plan, b, x, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart,
                            raise_on_not_converged=False)
    return plan, x[:n3].contiguous(), info


def fit_slope(L, R, lo=None, hi=None, floor=1e-12):
    """Least-squares slope of log R against log L over the lengths in
    [lo, hi] whose R lies above ``floor`` (None if fewer than two remain).
    The study fits between twice the shortest length and half the reference
    length: the shortest absorbers are not yet adiabatic, and as L approaches
    the reference length E_L approaches E_inf itself."""
    L = np.asarray(L, float)
    R = np.asarray(R, float)
    keep = (R > floor) & (L >= (lo if lo is not None else -np.inf)) & (L <= (hi if hi is not None else np.inf))
    L, R = L[keep], R[keep]
    if L.size < 2:
        return None
    A = np.vstack([np.log(L), np.ones(L.size)]).T
    s, _ = np.linalg.lstsq(A, np.log(R), rcond=None)[0]
    return float(s)


def rl_sweep(lengths_nm, degrees=(0, 1, 2), r_rt=1e-25, ref_nm=9450.0, tol=1e-8, body_nm=13500.0,
             h_nm=50.0 / 3.0, matched=False):
    """R(L) for each degree (Sec. 5.1), electric loss only (J-VIE with the
    block-circulant preconditioner) or with matched magnetic loss (JM-VIE,
    ``matched``).  Returns a dict with, per degree, the lengths (nm), R, solve
    statistics and the fitted slope."""
    t0 = time.perf_counter()
    nb = int(round(body_nm / h_nm))
    solve = _solve_matched if matched else _solve
    out = {"lengths_nm": list(map(float, lengths_nm)), "r_rt": r_rt, "reference_nm": ref_nm, "tol": tol,
           "grid_body": [nb, int(round(500 / h_nm)), int(round(200 / h_nm))], "h_nm": h_nm,
           "loss": "electric and matched magnetic (JM-VIE)" if matched else "electric (J-VIE)", "degrees": {}}
    for d in degrees:
        plan, x, info = solve(workloads.strip_rl(ref_nm, d, r_rt, h_nm=h_nm, length_nm=body_nm), tol)
        e_ref = vie.vie_axis_field(plan, x, nb)
        plan.close()
        Rs, iters, res = [], [], []
        for L in lengths_nm:
            plan, x, info = solve(workloads.strip_rl(L, d, r_rt, h_nm=h_nm, length_nm=body_nm), tol)
            Rs.append(vie.vie_reflection(e_ref, vie.vie_axis_field(plan, x, nb)))
            iters.append(info["iterations"])
            res.append(info["residual"])
            plan.close()
        lo, hi = 2.0 * min(lengths_nm), 0.5 * ref_nm
        out["degrees"][str(d)] = {"R": Rs, "iterations": iters, "true_residual_max": max(res),
                                  "slope": fit_slope(lengths_nm, Rs, lo, hi), "slope_window_nm": [lo, hi],
                                  "slope_predicted": -2.0 * (d + 1)}
    out["seconds"] = time.perf_counter() - t0
    return out


def bragg_sweep(lambdas_um, periods=100, tol=1e-6, batch=8, restart=30):
    """Transmission T(lambda) through the Bragg grating (Sec. 5.2), the
    wavelengths solved ``batch`` at a time with per-plan block-circulant
    preconditioners.  Returns wavelengths, T, T / max T and solve statistics."""
    import torch
    t0 = time.perf_counter()
    T, iters, res, conv = [], [], [], []
    grid = None
    for i0 in range(0, len(lambdas_um), batch):
        lams = lambdas_um[i0:i0 + batch]
        plans, bs, circs, slices = [], [], [], []
        for lam in lams:
            wl = workloads.bragg_grating(lam, periods=periods)
            grid = wl.grid
            plan, b = learned.setup_problem(wl)
            c = vie.vie_circulant_create(plan, vie.VIE_CIRC_FP16_FACTORS)
            vie.vie_set_circulant_preconditioner(plan, c)
            plans.append(plan)
            bs.append(b)
            circs.append(c)
            slices.append(int(wl.name.split("_x")[1]))
        xs = [torch.zeros_like(b) for b in bs]
        st, infos = vie.vie_solve_batch(plans, bs, xs, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart,
                                        use_preconditioner=True, raise_on_not_converged=False)
        for plan, x, info, ix in zip(plans, xs, infos, slices):
            T.append(vie.vie_slice_power(plan, x, ix))
            iters.append(info["iterations"])
            res.append(info["residual"])
            conv.append(bool(info["converged"]))
        for plan, c in zip(plans, circs):
            vie.vie_set_circulant_preconditioner(plan, None)
            c.close()
            plan.close()
        del xs, bs
    Tn = (np.asarray(T) / max(T)).tolist()
    return {"lambdas_um": list(map(float, lambdas_um)), "T": T, "T_normalised": Tn, "grid": list(grid),
            "periods": periods, "iterations": iters, "true_residual_max": max(res), "converged": sum(conv),
            "tol": tol, "seconds": time.perf_counter() - t0}


def microring_sweep(count=16, tol=1e-4, restart=30, max_iters=8000, timeout_s=900.0):
    """The ring resonator beside a bus (800 x 600 x 11 voxels of 20 nm,
    cubic absorbers at both bus ends) at ``count`` wavelengths in
    [1.54, 1.56] um, one plan per wavelength, all solved together by one
    mixed-precision batch call (no preconditioner: the block-circulant one
    would need 19,800^2 x 800 complex values).  Reports per wavelength the
    steps, the true residual and the power through the voxel plane 1 um
    before the output absorber, T(lambda) = sum |E|^2 there.  Restarted
    GMRES(30) stagnates on the resonator near a relative residual of 1e-4
    (1.3e-4 after 6000 steps at 1.54 and 1.56 um), hence the default
    tolerance."""
    import torch
    t0 = time.perf_counter()
    lams = workloads.microring_wavelengths(count)
    plans, bs, xs, ixs = [], [], [], []
    for lam in lams:
        wl = workloads.microring(lambda_um=lam)
        plan, b = learned.setup_problem(wl)
        plans.append(plan)
        bs.append(b)
        xs.append(torch.zeros_like(b))
        ixs.append(int(round(wl.grid[0] - wl.absorbers[1].length - 1.0 / wl.h_um)))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    st, infos = vie.vie_solve_batch(plans, bs, xs, tol, mode=vie.VIE_SOLVE_MIXED, restart=restart,
                                    max_iters=max_iters, timeout_s=timeout_s, raise_on_not_converged=False)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    T = [vie.vie_slice_power(p, x, ix) for p, x, ix in zip(plans, xs, ixs)]
    device_bytes = sum(p.info()["device_bytes"] for p in plans)
    for p in plans:
        p.close()
    Tn = (np.asarray(T) / max(T)).tolist()
    return {"lambdas_um": lams, "grid": [800, 600, 11], "tol": tol, "restart": restart, "status": st,
            "iterations": [i["iterations"] for i in infos], "converged": sum(bool(i["converged"]) for i in infos),
            "true_residual": [i["residual"] for i in infos], "T": T, "T_normalised": Tn,
            "plan_setup_s": t1 - t0, "solve_s": t2 - t1, "solve_device_ms": infos[0]["time_ms"],
            "plans_device_bytes": device_bytes}


def band_gap(lambdas_um, T_normalised, level=0.5):
    """Centre and width of the widest contiguous run of wavelengths whose
    normalised transmission is below ``level`` (None if there is none)."""
    lam = np.asarray(lambdas_um)
    low = np.asarray(T_normalised) < level
    best, cur = None, None
    for i, v in enumerate(low):
        if v:
            cur = (cur[0], i) if cur else (i, i)
            if best is None or cur[1] - cur[0] > best[1] - best[0]:
                best = cur
        else:
            cur = None
    if best is None:
        return None
    a, b = lam[best[0]], lam[best[1]]
    return {"centre_um": float(0.5 * (a + b)), "width_um": float(b - a), "level": level}
