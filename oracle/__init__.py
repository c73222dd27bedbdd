"""FP64 CPU oracle for the FFT-accelerated J-VIE operator of
"Adiabatic absorbers in photonics simulations with the volume integral
equation method" (arXiv:1803.06237).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (the CUDA library and its Python binding) never imports,
links or calls anything here, and nothing here imports the product path.

Modules
-------
greens     Galerkin entries T_pq(Delta) of the discrete operator N (Sec. 3.1,
           Eq. for N_ij = <N P_j, P_i>) by singularity-aware quadrature.
operator   dense assembly of I - M_eps N on tiny grids, the circulant-embedded
           FFT matvec (Sec. 5.4, "Numerical aspects"), contrast and absorber
           (Sec. 4.1-4.2), and the right-hand side of the J-VIE.
gmres      restarted GMRES / flexible GMRES with MGS Arnoldi and Givens
           rotations in FP64 (Sec. 5 solver, Sec. 5.4 discussion).
metrics    field on the centre axis and the reflection coefficient R (Sec. 5.1).

Everything is written for clarity: plain NumPy/SciPy in float64/complex128,
no blocking, no fusion.  Parity of every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against closed forms,
invariants and brute force; see each module's header for its pins.
"""
