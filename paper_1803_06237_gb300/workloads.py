"""Seeded synthetic inputs shaped like the paper's waveguide workloads.

This module only generates data: grids, permittivity maps, absorber
parameters, source sheets and random vectors.  It holds none of the method's
arithmetic (no contrast, no absorber profile, no Green function), so both the
CUDA path and the FP64 oracle can take their inputs from it.

Every generator takes an explicit seed and uses NumPy's PCG64.

Workloads (sizes in units of the voxel size h unless stated):

* ``cube``       lossless dielectric cube eps = 12.25 in vacuum, 12^3 voxels,
                 side 0.4 um (h = 33.3 nm), lambda0 = 1.55 um, x-polarised
                 plane wave along +z.
* ``waveguide``  Si strip eps = 12.11 (core 460 x 220 nm = 23 x 11 voxels) in
                 eps_bg = 2.085, h = 20 nm, 600 x 23 x 11 voxels (12 um),
                 quadratic absorber over the last 4 um (x0 = 400, L = 200)
                 with round-trip target R_rt = 1e-10, y-polarised Gaussian
                 current sheet (waist 200 nm) on the voxel plane x = 1 um.
* ``batch48``    48 guides of the same cross-section: absorber length
                 {1,2,4,6,8,10} um x degree {0,1,2,3} x eps''_max {0.5, 2};
                 nx = 250 + 50 L[um] (a 5 um body plus the absorber).
* ``microring``  ring resonator, R = 5 um, 450 x 220 nm strips, 200 nm gap
                 to a straight bus along x, h = 20 nm, 800 x 600 x 11 voxels,
                 cubic absorbers over the first and last 4 um in x, y-sheet
                 on the bus 1 um inside the left absorber's end; 16
                 wavelengths in [1.54, 1.56] um (``microring_wavelengths``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LAMBDA0_UM = 1.55


@dataclasses.dataclass
class Absorber:
    x0: float            # start of the absorber, units of h from the low-x edge
    length: float        # absorber length L, units of h
    degree: int          # d in s(u) = u^d
    eps2_max: float | None = None   # eps''_max if given directly
    r_rt: float | None = None       # else: target round-trip reflection
    direction: int = +1


@dataclasses.dataclass
class Workload:
    name: str
    grid: tuple           # (nx, ny, nz)
    h_um: float
    k0_per_um: float
    eps_bg: float
    eps: np.ndarray       # relative permittivity per voxel, (nz, ny, nx) complex
    absorbers: list
    source: str           # "plane_wave_x" or "sheet"
    src: np.ndarray | None = None   # impressed current (3, nz, ny, nx) for "sheet"
    eps_core: float = 0.0

    @property
    def n_voxels(self) -> int:
        return int(np.prod(self.grid))

    @property
    def kappa(self) -> float:
        """k h with k = k0 sqrt(eps_bg) (dimensionless)."""
        return self.k0_per_um * math.sqrt(self.eps_bg) * self.h_um


def _k0() -> float:
    return 2.0 * math.pi / LAMBDA0_UM


def cube(n: int = 12) -> Workload:
    eps = np.full((n, n, n), 12.25 + 0j)
    return Workload("cube", (n, n, n), 0.4 / n, _k0(), 1.0, eps, [], "plane_wave_x",
                    eps_core=12.25)


def gaussian_sheet(grid, ix: int, waist_vox: float, comp: int = 1) -> np.ndarray:
    """Impressed current: exp(-((y - yc)^2 + (z - zc)^2) / waist^2) on the
    voxel plane ``ix``, component ``comp`` (1 = y), voxel-centre coordinates,
    centred on the cross-section."""
    nx, ny, nz = grid
    y = np.arange(ny) + 0.5 - ny / 2.0
    z = np.arange(nz) + 0.5 - nz / 2.0
    prof = np.exp(-(z[:, None] ** 2 + y[None, :] ** 2) / waist_vox**2)
    src = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    src[comp, :, :, ix] = prof
    return src


def waveguide(nx: int = 600, ny: int = 23, nz: int = 11, h_um: float = 0.02,
              absorber_len_um: float = 4.0, degree: int = 2, eps2_max=None,
              r_rt: float = 1e-10, src_x_um: float = 1.0, waist_um: float = 0.2,
              eps_core: float = 12.11, eps_bg: float = 2.085,
              name: str = "waveguide") -> Workload:
    eps = np.full((nz, ny, nx), eps_core + 0j)
    L = absorber_len_um / h_um
    ab = Absorber(x0=nx - L, length=L, degree=degree,
                  eps2_max=eps2_max, r_rt=None if eps2_max is not None else r_rt)
    src = gaussian_sheet((nx, ny, nz), int(round(src_x_um / h_um)), waist_um / h_um)
    return Workload(name, (nx, ny, nz), h_um, _k0(), eps_bg, eps, [ab], "sheet", src,
                    eps_core=eps_core)


def batch48():
    """The 48 uneven guides (list of Workload)."""
    out = []
    for L in (1, 2, 4, 6, 8, 10):
        for d in (0, 1, 2, 3):
            for e2 in (0.5, 2.0):
                nx = 250 + 50 * L
                out.append(waveguide(nx=nx, absorber_len_um=float(L), degree=d,
                                     eps2_max=e2, name=f"guide_L{L}_d{d}_e{e2}"))
    return out


def random_currents(grid, seed: int, dtype=np.complex128) -> np.ndarray:
    """Complex normal vector of shape (3, nz, ny, nx)."""
    nx, ny, nz = grid
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((2, 3, nz, ny, nx))
    return (v[0] + 1j * v[1]).astype(dtype)


def random_permittivity(grid, seed: int, lossy: bool = True) -> np.ndarray:
    """eps per voxel: real part U[1, 13], imaginary part -U[0, 2] if lossy."""
    nx, ny, nz = grid
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.uniform(1.0, 13.0, (nz, ny, nx))
    im = -rng.uniform(0.0, 2.0, (nz, ny, nx)) if lossy else np.zeros((nz, ny, nx))
    return re + 1j * im


def sparse_currents(grid, seed: int, nnz: int) -> np.ndarray:
    """Vector with ``nnz`` random non-zero (voxel, component) entries."""
    nx, ny, nz = grid
    rng = np.random.Generator(np.random.PCG64(seed))
    v = np.zeros(3 * nx * ny * nz, dtype=np.complex128)
    idx = rng.choice(v.size, size=nnz, replace=False)
    v[idx] = rng.standard_normal(nnz) + 1j * rng.standard_normal(nnz)
    return v.reshape(3, nz, ny, nx)


def sample_indices(grid, seed: int, count: int) -> np.ndarray:
    """Distinct flat (component, voxel) output indices to spot-check."""
    n = 3 * int(np.prod(grid))
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


def random_guide(seed: int, nx: int = 160, ny: int = 40, nz: int = 11, h_um: float = 0.02,
                 eps_core: float = 12.11, eps_bg: float = 2.085, absorber_len_um: float = 1.0,
                 r_rt: float = 1e-10) -> Workload:
    """Seeded strip or circular-bend waveguide (width U[350, 550] nm, all nz
    layers core, i.e. 220 nm at h = 20 nm) on an nx x ny x nz grid, with a
    quadratic absorber over the last ``absorber_len_um`` and a Gaussian
    y-sheet 0.4 um from the left end.  Bends have radius U[2, 5] um and start
    at a random x in the first third of the guide."""
    rng = np.random.Generator(np.random.PCG64(seed))
    width = rng.uniform(0.35, 0.55) / h_um                 # in voxels
    yc = ny / 2.0 + rng.uniform(-2.0, 2.0)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    X, Y = np.meshgrid(x, y)                               # (ny, nx)
    if rng.random() < 0.5:
        inside = np.abs(Y - yc) <= width / 2
    else:
        R = rng.uniform(2.0, 5.0) / h_um
        x0 = rng.uniform(0.0, nx / 3.0)
        sign = 1.0 if rng.random() < 0.5 else -1.0
        # straight for x < x0, then an arc of radius R bending towards +/- y
        cy = yc + sign * R
        d_arc = np.abs(np.hypot(X - x0, Y - cy) - R)
        inside = np.where(X < x0, np.abs(Y - yc) <= width / 2, d_arc <= width / 2)
    eps = np.full((nz, ny, nx), eps_bg + 0j)
    eps[:, inside] = eps_core
    L = absorber_len_um / h_um
    ab = Absorber(x0=nx - L, length=L, degree=2, r_rt=r_rt)
    src = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    ix = int(round(0.4 / h_um))
    zz = np.arange(nz) + 0.5 - nz / 2.0
    prof = np.exp(-(zz[:, None] ** 2 + (y[None, :] - yc) ** 2) / (0.2 / h_um) ** 2)
    src[1, :, :, ix] = prof
    return Workload(f"guide_{seed}", (nx, ny, nz), h_um, _k0(), eps_bg, eps, [ab], "sheet", src, eps_core=eps_core)


def microring(nx: int = 800, ny: int = 600, nz: int = 11, h_um: float = 0.02, radius_um: float = 5.0,
              width_um: float = 0.45, gap_um: float = 0.2, absorber_len_um: float = 4.0, degree: int = 3,
              r_rt: float = 1e-10, eps_core: float = 12.11, eps_bg: float = 2.085,
              lambda_um: float = LAMBDA0_UM) -> Workload:
    """Ring resonator beside a straight bus (all nz layers core).  The bus
    runs along x with its centre 20 voxels from the low-y edge; the ring is
    centred in x, its centre-line radius ``radius_um``, with ``gap_um``
    between the bus and the ring edges.  The absorbers span the full
    cross-section over their x range, so at this grid size they also reach
    the ring's outermost x sides."""
    w = width_um / h_um
    R = radius_um / h_um
    yb = 20.0
    yc = yb + w + gap_um / h_um + R
    xc = nx / 2.0
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    X, Y = np.meshgrid(x, y)                               # (ny, nx)
    inside = (np.abs(Y - yb) <= w / 2) | (np.abs(np.hypot(X - xc, Y - yc) - R) <= w / 2)
    eps = np.full((nz, ny, nx), eps_bg + 0j)
    eps[:, inside] = eps_core
    L = absorber_len_um / h_um
    abs_ = [Absorber(x0=L, length=L, degree=degree, r_rt=r_rt, direction=-1),
            Absorber(x0=nx - L, length=L, degree=degree, r_rt=r_rt, direction=+1)]
    src = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    ix = int(round(L + 1.0 / h_um))
    zz = np.arange(nz) + 0.5 - nz / 2.0
    src[1, :, :, ix] = np.exp(-(zz[:, None] ** 2 + (y[None, :] - yb) ** 2) / (0.2 / h_um) ** 2)
    return Workload("microring", (nx, ny, nz), h_um, 2.0 * math.pi / lambda_um, eps_bg, eps, abs_, "sheet",
                    src, eps_core=eps_core)


def strip_rl(absorber_nm: float, degree: int, r_rt: float = 1e-25, h_nm: float = 50.0 / 3.0,
             length_nm: float = 13500.0, width_nm: float = 500.0, height_nm: float = 200.0,
             src_x_um: float = 1.0, eps_core: float = 12.11, eps_bg: float = 2.085) -> Workload:
    """The absorber-length study of Sec. 5.1: a strip 13.5 um x 500 x 200 nm
    (810 x 30 x 12 voxels of 50/3 nm) with an absorber of ``absorber_nm``
    appended at the right end (all core voxels), the round-trip target
    ``r_rt`` and the monomial degree; Gaussian y-sheet source at x = 1 um."""
    h_um = h_nm / 1000.0
    nb = int(round(length_nm / h_nm))
    L = int(round(absorber_nm / h_nm))
    ny, nz = int(round(width_nm / h_nm)), int(round(height_nm / h_nm))
    nx = nb + L
    eps = np.full((nz, ny, nx), eps_core + 0j)
    ab = Absorber(x0=float(nb), length=float(L), degree=degree, r_rt=r_rt)
    src = gaussian_sheet((nx, ny, nz), int(round(src_x_um / h_um)), 0.2 / h_um)
    return Workload(f"strip_L{absorber_nm:.0f}_d{degree}", (nx, ny, nz), h_um, _k0(), eps_bg, eps, [ab], "sheet",
                    src, eps_core=eps_core)


def bragg_grating(lambda_um: float, periods: int = 100, period_nm: float = 320.0, width_nm: float = 500.0,
                  dwidth_nm: float = 40.0, height_nm: float = 220.0, lead_periods: int = 10,
                  tail_um: float = 1.0, absorber_um: float = 2.2, degree: int = 2, r_rt: float = 1e-10,
                  h_nm: float = 20.0, eps_core: float = 12.11, eps_bg: float = 2.085) -> Workload:
    """The Bragg grating of Sec. 2.2 / 5.2 at h = 20 nm: a strip of width W
    whose width alternates between W + dW and W - dW every half period (each
    edge moves by dW/2 = one voxel), N periods, preceded by a uniform
    lead-in of 10 periods and followed by ``tail_um`` of uniform guide, with
    quadratic absorbers of ``absorber_um`` on both ends; height 220 nm.  A
    Gaussian y-sheet a quarter of the wavelength in silicon into the lead-in
    excites it.  Returns the workload; ``slice_x`` (the voxel plane half way
    through the tail, where the transmission is taken) is stored in
    ``wl.name`` as ``bragg_x<slice_x>``."""
    h_um = h_nm / 1000.0
    La = int(round(absorber_um / h_um))
    lead = int(round(lead_periods * period_nm / h_nm))
    per = int(round(period_nm / h_nm))
    tail = int(round(tail_um / h_um))
    nx = La + lead + periods * per + tail + La
    wmax = int(round((width_nm + dwidth_nm) / h_nm))
    ny, nz = wmax, int(round(height_nm / h_nm))
    wide = np.ones(ny, bool)
    narrow = np.zeros(ny, bool)
    d = int(round(dwidth_nm / h_nm))
    narrow[d:ny - d] = True
    core = np.zeros((ny, nx), bool)
    nominal = np.zeros(ny, bool)
    nominal[d // 2:ny - d // 2] = True
    x0 = La + lead
    for ix in range(nx):
        if x0 <= ix < x0 + periods * per:
            core[:, ix] = wide if ((ix - x0) % per) < per // 2 else narrow
        else:
            core[:, ix] = nominal
    eps = np.full((nz, ny, nx), eps_bg + 0j)
    eps[:, core] = eps_core
    abs_ = [Absorber(x0=float(La), length=float(La), degree=degree, r_rt=r_rt, direction=-1),
            Absorber(x0=float(nx - La), length=float(La), degree=degree, r_rt=r_rt, direction=+1)]
    lam_si = lambda_um / math.sqrt(eps_core)
    ix = La + int(round(0.25 * lam_si / h_um))
    zz = np.arange(nz) + 0.5 - nz / 2.0
    yy = np.arange(ny) + 0.5 - ny / 2.0
    src = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    src[1, :, :, ix] = np.exp(-(zz[:, None] ** 2 + yy[None, :] ** 2) / (0.2 / h_um) ** 2)
    slice_x = x0 + periods * per + tail // 2
    return Workload(f"bragg_x{slice_x}", (nx, ny, nz), h_um, 2.0 * math.pi / lambda_um, eps_bg, eps, abs_,
                    "sheet", src, eps_core=eps_core)


def microring_wavelengths(count: int = 16, lo_um: float = 1.54, hi_um: float = 1.56) -> list:
    """``count`` equally spaced wavelengths in [lo, hi] (um)."""
    return [lo_um + (hi_um - lo_um) * i / (count - 1) for i in range(count)]
