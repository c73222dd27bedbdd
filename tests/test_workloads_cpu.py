"""Host checks of the seeded input generators (paper_1803_06237_gb300/workloads.py)."""
import math

import numpy as np

from paper_1803_06237_gb300 import workloads


def test_microring_geometry():
    """800 x 600 x 11 ring resonator: core areas close to those of the
    continuous shapes, the 200 nm gap kept, absorbers at both x ends."""
    wl = workloads.microring()
    nx, ny, nz = wl.grid
    assert (nx, ny, nz) == (800, 600, 11) and abs(wl.h_um - 0.02) < 1e-12
    core = np.abs(wl.eps - wl.eps_bg) > 0
    assert (core == core[0]).all()                     # every layer is core
    c = core[0]
    h = wl.h_um
    w = 0.45 / h
    bus_rows = np.flatnonzero(c[:, 0])                  # x = 0 sees only the bus
    assert abs(len(bus_rows) - w) <= 1.0
    ring = c.copy()
    ring[bus_rows, :] = False
    area_ring = 2 * math.pi * (5.0 / h) * w
    assert abs(ring.sum() - area_ring) <= 0.02 * area_ring
    # gap: nearest ring voxel centre above the bus edge
    ys = np.nonzero(ring)[0]
    gap_vox = ys.min() - bus_rows.max() - 1
    assert abs(gap_vox - 0.2 / h) <= 1.0
    left, right = wl.absorbers
    L = 4.0 / h
    assert left.direction == -1 and left.x0 == L and left.length == L and left.degree == 3
    assert right.direction == 1 and right.x0 == nx - L and right.length == L and right.degree == 3
    # the source sheet sits on the bus, 1 um inside the left absorber's end
    ix = np.flatnonzero(np.abs(wl.src[1]).sum(axis=(0, 1)))
    assert list(ix) == [int(round(L + 1.0 / h))]
    prof = np.abs(wl.src[1, nz // 2, :, ix[0]])
    assert abs(int(np.argmax(prof)) - (bus_rows.min() + bus_rows.max()) / 2) <= 1.0


def test_microring_wavelengths():
    lam = workloads.microring_wavelengths()
    assert len(lam) == 16 and abs(lam[0] - 1.54) < 1e-12 and abs(lam[-1] - 1.56) < 1e-12
    assert np.allclose(np.diff(lam), 0.02 / 15)
