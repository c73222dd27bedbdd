"""GPU parity of the setup (Toeplitz entries) and the J-VIE operator
application against the FP64 CPU oracle, through the C ABI.

Tolerances: complex128 path, relative L2 <= 1e-12 (FP64 FFTs of length up to
~1.4e6 accumulate ~1e-15 per element; the entries agree to ~1e-15 relative);
complex64 path, relative L2 <= 2e-6 (FP32 unit roundoff 6e-8 times the ~20
butterfly stages and the 3x3 multiply, with margin), element-wise
|y_gpu - y| <= 1e-5 max|y|.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from gpu_helpers import oracle_matvec, oracle_sparse_apply, rel_l2
from oracle import greens
from oracle import operator as op
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-6
K0 = 2 * math.pi / 1.55


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()
    assert torch.cuda.is_available()


def _apply(plan, x, dtype, mode="operator"):
    xd = torch.from_numpy(np.ascontiguousarray(x.ravel())).to(dtype).cuda()
    yd = torch.empty_like(xd)
    if mode == "operator":
        vie.vie_matvec(plan, xd, yd)
    else:
        vie.vie_rhs_from_source(plan, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("grid,h,eps_bg", [((5, 4, 3), 0.4 / 12, 1.0), ((12, 12, 12), 0.4 / 12, 1.0),
                                           ((9, 23, 11), 0.02, 2.085)])
def test_toeplitz_entries_match_oracle(grid, h, eps_bg):
    plan = vie.vie_plan_create(grid, h, K0, eps_bg)
    T_gpu = vie.vie_get_toeplitz(plan)
    kappa = plan.info()["kappa"]
    T_ref = greens.octant_table(kappa, grid)
    scale = np.abs(T_ref).max()
    assert np.abs(T_gpu - T_ref).max() <= 1e-13 * scale
    # far entries separately, relative to their own size
    far = np.abs(T_ref).max(axis=0) < 1e-2 * scale
    if far.any():
        d = np.abs(T_gpu - T_ref)[:, far].max() / np.abs(T_ref)[:, far].max()
        assert d < 1e-12


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, TOL64), (torch.complex64, TOL32)])
def test_cube_matvec_matches_oracle(dtype, tol):
    wl = workloads.cube(12)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    eps = workloads.random_permittivity(wl.grid, seed=21)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(wl.grid, seed=22)
    y = _apply(plan, x, dtype)
    M = op.contrast_M(op.chi_from_permittivity(eps, wl.eps_bg))
    y_ref = oracle_matvec(wl.grid, wl.kappa, M, x).ravel()
    assert rel_l2(y, y_ref) <= tol
    assert np.abs(y - y_ref).max() <= 5 * tol * np.abs(y_ref).max()


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 3, 5), (7, 1, 1), (1, 1, 9), (13, 4, 6), (3, 7, 2), (31, 2, 3)])
@pytest.mark.parametrize("flags", [vie.VIE_PLAN_DEFAULT, vie.VIE_PLAN_CIRC_2N])
def test_ragged_grids(grid, flags):
    two_n_smooth = all(_smooth(2 * v) for v in grid)
    if flags == vie.VIE_PLAN_CIRC_2N and not two_n_smooth:
        with pytest.raises(vie.VieError) as ei:
            vie.vie_plan_create(grid, 0.02, K0, 2.085, flags)
        assert ei.value.status == 1
        return
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085, flags)
    m = plan.info()["m"]
    assert all(mi >= 2 * ni - 1 for mi, ni in zip(m, grid))
    eps = workloads.random_permittivity(grid, seed=31)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=32)
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    y_ref = oracle_matvec(grid, plan.info()["kappa"], M, x).ravel()
    assert rel_l2(_apply(plan, x, torch.complex128), y_ref) <= TOL64
    assert rel_l2(_apply(plan, x, torch.complex64), y_ref) <= TOL32


def _smooth(m):
    for f in (2, 3, 5):
        while m % f == 0:
            m //= f
    return m == 1


def test_zero_contrast_is_identity_bitwise():
    grid = (10, 6, 4)
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    x = workloads.random_currents(grid, seed=3)
    for dt in (torch.complex128, torch.complex64):
        y = _apply(plan, x, dt)
        assert np.array_equal(y, x.ravel().astype(dt == torch.complex64 and np.complex64 or np.complex128))


def _waveguide_section(nx):
    wl = workloads.waveguide(nx=nx, absorber_len_um=nx * 0.02 / 3, src_x_um=min(1.0, nx * 0.02 / 4))
    ab = wl.absorbers[0]
    e2 = op.eps2_max_from_rrt(1e-10, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
    absorbers = [dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2)]
    return wl, absorbers


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, TOL64), (torch.complex64, TOL32)])
def test_waveguide_section_with_absorber(dtype, tol):
    wl, absorbers = _waveguide_section(60)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    x = workloads.random_currents(wl.grid, seed=41)
    M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg, absorbers))
    y_ref = oracle_matvec(wl.grid, wl.kappa, M, x).ravel()
    assert rel_l2(_apply(plan, x, dtype), y_ref) <= tol


def test_rhs_from_source_matches_oracle():
    wl, absorbers = _waveguide_section(40)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    src = workloads.gaussian_sheet(wl.grid, 10, 10.0)
    M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg, absorbers))
    b_ref = oracle_matvec(wl.grid, wl.kappa, M, src, mode="rhs").ravel()
    assert rel_l2(_apply(plan, src, torch.complex128, mode="rhs"), b_ref) <= TOL64
    assert rel_l2(_apply(plan, src, torch.complex64, mode="rhs"), b_ref) <= TOL32


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, TOL64), (torch.complex64, 1e-5)])
def test_full_size_waveguide_sampled(dtype, tol):
    """600 x 23 x 11 guide, the launch configuration of the benchmark: sparse
    input, 240 sampled outputs summed directly by the oracle."""
    wl = workloads.waveguide()
    ab = wl.absorbers[0]
    e2 = op.eps2_max_from_rrt(ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
    absorbers = [dict(x0=ab.x0, length=ab.length, degree=ab.degree, eps2_max=e2)]
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    x = workloads.sparse_currents(wl.grid, seed=51, nnz=20)
    y = _apply(plan, x, dtype)
    idx = workloads.sample_indices(wl.grid, seed=52, count=200)
    nzv = np.flatnonzero(x.ravel())
    idx = np.unique(np.concatenate([idx, nzv, nzv + 1]))
    idx = idx[idx < 3 * wl.n_voxels]
    M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg, absorbers))
    ref = oracle_sparse_apply(wl.kappa, wl.grid, M, x, idx)
    assert np.abs(y[idx] - ref).max() <= tol * np.abs(ref).max()
    # far from every source the response is small but must still match in absolute terms
    assert np.isfinite(y).all()


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 2e-5)])
def test_full_size_reciprocity(dtype, tol):
    """The full 600 x 23 x 11 guide with dense random inputs, a property that
    holds at any size: the dyadic Green's function is symmetric under the
    exchange of source and observation point, so the Galerkin operator N
    (Sec. 3.1) is complex symmetric, u^T N v = v^T N u.  N v is recovered as
    M^{-1} (v - A v) from applications of A = I - M N, every voxel's contrast
    with |M| >= 1/2."""
    wl = workloads.waveguide()
    nx, ny, nz = grid = wl.grid
    rng = np.random.Generator(np.random.PCG64(61))
    eps = wl.eps_bg * (2.0 + 3.0 * rng.random((nz, ny, nx))) - 1j * rng.random((nz, ny, nx))
    plan = vie.vie_plan_create(grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, eps)
    Mi = np.broadcast_to(1.0 / op.contrast_M(op.chi_from_permittivity(eps, wl.eps_bg)), (3, nz, ny, nx)).ravel()
    np_dtype = np.complex128 if dtype == torch.complex128 else np.complex64
    u = workloads.random_currents(grid, seed=62).astype(np_dtype).astype(np.complex128)
    v = workloads.random_currents(grid, seed=63).astype(np_dtype).astype(np.complex128)
    Nu = (u.ravel() - _apply(plan, u, dtype)) * Mi
    Nv = (v.ravel() - _apply(plan, v, dtype)) * Mi
    a, b = np.dot(u.ravel(), Nv), np.dot(v.ravel(), Nu)
    assert abs(a - b) <= tol * np.linalg.norm(u) * np.linalg.norm(Nv), (a, b)
    plan.close()


@pytest.mark.parametrize("flags", [0, 2])
def test_full_size_dense_complex64_matches_complex128(flags):
    """The full 600 x 23 x 11 guide with a dense random input and random
    contrast: the complex64 path (its x passes with five lines per block, one
    block per SM: the default three-factor forward and four-step inverse, and
    whatever the tuner picks) against the complex128 path (pinned to the
    oracle by the sampled test above), element by element."""
    wl = workloads.waveguide()
    grid = wl.grid
    eps = workloads.random_permittivity(grid, seed=73)
    plan = vie.vie_plan_create(grid, wl.h_um, wl.k0_per_um, wl.eps_bg, flags)
    if flags == vie.VIE_PLAN_AUTOTUNE:
        assert plan.info()["tune_candidates"] > 0
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=74).astype(np.complex64).astype(np.complex128)
    y64 = _apply(plan, x, torch.complex128)
    y32 = _apply(plan, x, torch.complex64)
    assert rel_l2(y32, y64) <= TOL32
    assert np.abs(y32 - y64).max() <= 1e-5 * np.abs(y64).max()
    plan.close()


def test_bad_inputs_report_errors():
    grid = (4, 3, 2)
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    eps = np.full((2, 3, 4), 2.0 + 0j)
    eps[1, 1, 1] = 0.0     # eps_r = 0 -> M = chi / (1 + chi) undefined
    with pytest.raises(vie.VieError) as ei:
        vie.vie_set_permittivity(plan, eps)
    assert ei.value.status == 6
    x = torch.zeros(2 * 3 * 24, dtype=torch.complex128, device="cuda")
    rc = vie.load().vie_matvec(plan.handle, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(x.data_ptr() + 16), vie.VIE_C128, None)
    assert rc == 1 and "overlap" in vie.vie_last_error()


def _smooth_at_least(n):
    m = max(1, n)
    while not _smooth(m):
        m += 1
    return m


# (ny, nz) whose circulant sizes hit each compiled register pass-B pair
@pytest.mark.parametrize("ny,nz", [(12, 12), (23, 11), (24, 11), (25, 11), (15, 11), (20, 11), (13, 11),
                                   (23, 13), (24, 13), (12, 13)])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, TOL64), (torch.complex64, TOL32)])
def test_register_pass_b_sizes(ny, nz, dtype, tol):
    grid = (5, ny, nz)
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    m = plan.info()["m"]
    assert m[1] == _smooth_at_least(2 * ny - 1) and m[2] == _smooth_at_least(2 * nz - 1)
    eps = workloads.random_permittivity(grid, seed=ny * 100 + nz)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=ny + nz)
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    y_ref = oracle_matvec(grid, plan.info()["kappa"], M, x).ravel()
    assert rel_l2(_apply(plan, x, dtype), y_ref) <= tol


# nx whose Mx hits each compiled four-step x-pass factorisation, and the
# three-factor one (Mx = 1200: 600 with the line length compiled in, 599
# without)
@pytest.mark.parametrize("nx", [300, 360, 450, 563, 675, 750, 800, 600, 599, 200])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, TOL64), (torch.complex64, TOL32)])
def test_four_step_x_sizes(nx, dtype, tol):
    grid = (nx, 3, 2)
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    assert plan.info()["m"][0] == _smooth_at_least(2 * nx - 1)
    eps = workloads.random_permittivity(grid, seed=nx)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=nx + 1)
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    y_ref = oracle_matvec(grid, plan.info()["kappa"], M, x).ravel()
    assert rel_l2(_apply(plan, x, dtype), y_ref) <= tol


@pytest.mark.parametrize("grid", [(13, 4, 6), (1, 1, 9), (150, 23, 11), (600, 3, 2)])
def test_autotuned_plan_matches_oracle(grid):
    """Any circulant size M >= 2n - 1 embeds the Toeplitz operator exactly
    (Sec. 3), so the tuner's choice changes the time, never the result."""
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085, vie.VIE_PLAN_AUTOTUNE)
    info = plan.info()
    assert info["tune_candidates"] >= 1 and info["tune_ms"] > 0
    assert all(mi >= 2 * ni - 1 and _smooth(mi) for mi, ni in zip(info["m"], grid))
    assert info["x_lines_per_block"] in (0, 2, 4, 5, -1, -2, -5)
    assert info["x_lines_per_block_inverse"] in (0, 2, 4, 5, -1, -2, -5)
    eps = workloads.random_permittivity(grid, seed=41)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=42)
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    y_ref = oracle_matvec(grid, info["kappa"], M, x).ravel()
    assert rel_l2(_apply(plan, x, torch.complex128), y_ref) <= TOL64
    assert rel_l2(_apply(plan, x, torch.complex64), y_ref) <= TOL32
    # a clone keeps the tuned shapes
    clone = vie.vie_plan_clone(plan)
    ci = clone.info()
    assert ci["m"] == info["m"] and ci["x_lines_per_block"] == info["x_lines_per_block"]
    assert ci["x_lines_per_block_inverse"] == info["x_lines_per_block_inverse"]
    vie.vie_set_permittivity(clone, eps)
    assert rel_l2(_apply(clone, x, torch.complex64), y_ref) <= TOL32


@pytest.mark.parametrize("grid", [(4, 200, 12), (3, 300, 6), (5, 97, 13), (4, 100, 7), (2, 150, 20),
                                  (3, 200, 23)])
def test_large_plane_pass_b_grids(grid):
    """y-z planes larger than one CTA's shared memory (complex64 from My Mz
    ~ 4.7e3, complex128 from ~2.3e3; (4, 100, 7) only in complex128): the
    split pass B (y along lines, z-stage kernel, inverse y) where Mz has a
    z-stage kernel, else (Mz = 40, 45) the pass on a cluster of 2-8 CTAs
    sharing the plane in distributed shared memory.  Ragged tiles, folded
    images at kxf = 0 and Mx / 2."""
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    eps = workloads.random_permittivity(grid, seed=61)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=62)
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    y_ref = oracle_matvec(grid, plan.info()["kappa"], M, x).ravel()
    assert rel_l2(_apply(plan, x, torch.complex128), y_ref) <= TOL64
    assert rel_l2(_apply(plan, x, torch.complex64), y_ref) <= TOL32


def _absorber_dicts(wl):
    out = []
    for ab in wl.absorbers:
        e2 = op.eps2_max_from_rrt(ab.r_rt, ab.degree, ab.length * wl.h_um, wl.k0_per_um, wl.eps_core)
        out.append(dict(x0=ab.x0, length=ab.length, degree=ab.degree, direction=ab.direction, eps2_max=e2))
    return out


@pytest.fixture(scope="module")
def microring_plan():
    wl = workloads.microring()
    absorbers = _absorber_dicts(wl)
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    assert plan.info()["m"] == (1600, 1200, 24)
    vie.vie_set_permittivity(plan, wl.eps, absorbers)
    M = op.contrast_M(op.chi_from_permittivity(wl.eps, wl.eps_bg, absorbers))
    return wl, plan, M


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, TOL64), (torch.complex64, 1e-5)])
def test_full_size_microring_sampled(microring_plan, dtype, tol):
    """800 x 600 x 11 ring resonator (circulant 1600 x 1200 x 24, pass B on
    CTA clusters): sparse input, sampled outputs summed directly by the
    oracle, including the neighbours of every source entry."""
    wl, plan, M = microring_plan
    x = workloads.sparse_currents(wl.grid, seed=71, nnz=16)
    y = _apply(plan, x, dtype)
    idx = workloads.sample_indices(wl.grid, seed=72, count=200)
    nzv = np.flatnonzero(x.ravel())
    nx, ny = wl.grid[0], wl.grid[1]
    idx = np.unique(np.concatenate([idx, nzv, nzv + 1, nzv + nx, nzv + nx * ny]))
    idx = idx[idx < 3 * wl.n_voxels]
    ref = oracle_sparse_apply(wl.kappa, wl.grid, M, x, idx)
    assert np.abs(y[idx] - ref).max() <= tol * np.abs(ref).max()
    assert np.isfinite(y).all()


def _apply_static(plan, x, dtype):
    xd = torch.from_numpy(np.ascontiguousarray(x.ravel())).to(dtype).cuda()
    yd = torch.empty_like(xd)
    vie.vie_matvec_static_scratch(plan, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128)


def test_static_workspace_large_plane():
    """16 x 600 x 11 (circulant 32 x 1200 x 24): the plan's workspace holds the
    split pass B's buffer; the 16 MiB static workspace holds it in complex64
    but not in complex128, where the same plan falls back to the cluster
    pass.  All four routes agree with the oracle."""
    grid = (16, 600, 11)
    plan = vie.vie_plan_create(grid, 0.02, K0, 2.085)
    assert plan.info()["m"] == (32, 1200, 24)
    eps = workloads.random_permittivity(grid, seed=81)
    vie.vie_set_permittivity(plan, eps)
    x = workloads.random_currents(grid, seed=82)
    M = op.contrast_M(op.chi_from_permittivity(eps, 2.085))
    y_ref = oracle_matvec(grid, plan.info()["kappa"], M, x).ravel()
    for dtype, tol in ((torch.complex128, TOL64), (torch.complex64, TOL32)):
        assert rel_l2(_apply(plan, x, dtype), y_ref) <= tol
        assert rel_l2(_apply_static(plan, x, dtype), y_ref) <= tol
