"""Restarted GMRES and flexible GMRES in FP64 (oracle).

Test infrastructure only (see ``oracle/__init__``).

The paper solves the discrete J-VIE with GMRES at relative tolerance 1e-8
(Sec. 5 opening; Sec. 5.4 "Numerical aspects", which also shows unrestarted
GMRES histories).  The oracle is the textbook algorithm: Arnoldi with modified
Gram-Schmidt, Givens rotations on the Hessenberg matrix, the small
least-squares problem solved by back substitution, restart after ``restart``
steps.  With a right preconditioner P (possibly nonlinear) the flexible variant
keeps z_j = P(v_j) and updates x with Z y instead of V y.

Pins (tests/test_oracle_gmres.py): the solution matches an LU solve of the
dense matrix within the stated tolerance bound; the Arnoldi relation
A Z_m = V_{m+1} H_m holds to rounding; the Givens residual estimate equals the
true residual norm; full GMRES on an n x n system converges in at most n steps.
"""
from __future__ import annotations

import numpy as np


def fgmres(A, b, precond=None, x0=None, tol=1e-8, restart=50, maxiter=1000,
           record_arnoldi=False):
    """Solve A x = b.  ``A`` and ``precond`` are callables on flat complex128
    vectors.  Stops when ||b - A x|| / ||b|| <= tol (true residual checked at
    every restart and at the end).  Returns (x, info)."""
    b = np.asarray(b, dtype=np.complex128).ravel()
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.asarray(x0, np.complex128).ravel().copy()
    bnorm = np.linalg.norm(b)
    info = {"iterations": 0, "restarts": 0, "residuals": [], "converged": False}
    if bnorm == 0.0:
        info["converged"] = True
        return np.zeros(n, dtype=np.complex128), info
    P = precond if precond is not None else (lambda v: v)
    total = 0
    while total < maxiter:
        r = b - A(x)
        beta = np.linalg.norm(r)
        info["residuals"].append(beta / bnorm)
        if beta / bnorm <= tol:
            info["converged"] = True
            break
        m = min(restart, maxiter - total)
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.float64)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = P(V[j])
            w = A(Z[j])
            for i in range(j + 1):              # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if record_arnoldi:
                info.setdefault("H_raw", []).append(H[: j + 2, j].copy())
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                  # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.hypot(abs(a), abs(bb))
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            elif abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(bb) / den
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            info["residuals"].append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or total >= maxiter:
                break
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):     # back substitution
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + y @ Z[:j_done]
        info["restarts"] += 1
        if record_arnoldi:
            info["last_cycle"] = {"V": V[: j_done + 1], "Z": Z[:j_done]}
    else:
        r = b - A(x)
        info["residuals"].append(np.linalg.norm(r) / bnorm)
        info["converged"] = info["residuals"][-1] <= tol
    info["iterations"] = total
    info["final_residual"] = np.linalg.norm(b - A(x)) / bnorm
    info["converged"] = info["final_residual"] <= tol
    return x, info


def gmres(A, b, x0=None, tol=1e-8, restart=50, maxiter=1000):
    """Unpreconditioned restarted GMRES (FGMRES with the identity)."""
    return fgmres(A, b, None, x0, tol, restart, maxiter)
