"""Pins for oracle.metrics (Sec. 5.1 reflection coefficient) by closed forms
that do not restate R's own formula."""
import math

import numpy as np

from oracle import metrics


def test_reflection_coefficient_limits():
    rng = np.random.default_rng(0)
    E = rng.standard_normal((3, 50)) + 1j * rng.standard_normal((3, 50))
    assert metrics.reflection_coefficient(E, E) == 0.0
    assert metrics.reflection_coefficient(E, 0 * E) == 1.0


def test_reflection_of_a_standing_wave_is_the_reflected_power():
    """A guide mode exp(-j beta x) plus a reflected wave r exp(+j beta x): over
    a whole number of half-periods of the mode the cross term vanishes and
    R = |r|^2, whatever the phase of r and the number of field components."""
    for beta, npts, r in ((2 * math.pi / 40, 100, 0.3 * np.exp(0.7j)),      # 5 half-periods, 20 samples each
                          (2 * math.pi / 12, 60, 1e-3j),
                          (2 * math.pi / 30, 45, 0.05 - 0.02j)):
        x = np.arange(npts) + 0.5
        mode = np.exp(-1j * beta * x)
        refl = np.exp(+1j * beta * x)
        pol = np.array([0.2, 1.0, -0.1j])[:, None]
        E_inf = pol * mode
        E_L = pol * (mode + r * refl)
        assert abs(metrics.reflection_coefficient(E_inf, E_L) - abs(r) ** 2) <= 1e-13 * abs(r) ** 2


def test_reflection_is_phase_sensitive():
    """A field equal to the reference up to a phase phi and an amplitude a
    gives R = |1 - a exp(j phi)|^2 = 1 + a^2 - 2 a cos(phi) (R compares fields,
    not powers)."""
    rng = np.random.default_rng(5)
    E = rng.standard_normal((3, 37)) + 1j * rng.standard_normal((3, 37))
    for a, phi in ((1.0, 0.3), (0.9, 0.0), (1.2, math.pi), (1.0, 2.0)):
        R = metrics.reflection_coefficient(E, a * np.exp(1j * phi) * E)
        assert abs(R - (1 + a * a - 2 * a * math.cos(phi))) < 1e-13


def test_axis_field_is_current_over_contrast():
    chi = np.full((3, 5, 8), 2.0 + 0.5j)
    w = np.arange(3 * 3 * 5 * 8, dtype=complex).reshape(3, 3, 5, 8)
    E = metrics.axis_field(w, chi, 6)
    np.testing.assert_allclose(E, w[:, 1, 2, :6] / (2.0 + 0.5j))


def test_slice_power_counts_the_structure_only():
    """A field E = 2 + 1j in every voxel of the structure (w = chi E) gives
    T = |E|^2 times the number of structure voxels of the plane times 3
    components; cladding voxels (chi = 0) contribute nothing."""
    chi = np.zeros((3, 4, 6), complex)
    chi[:, 1:3, :] = 1.5 - 0.2j
    E = 2.0 + 1.0j
    w = np.broadcast_to(chi * E, (3, 3, 4, 6)).copy()
    w[:, :, 0, :] = 7.0             # values outside the structure are ignored
    for ix in (0, 5):
        assert abs(metrics.slice_power(w, chi, ix) - 3 * 6 * abs(E) ** 2) < 1e-12
