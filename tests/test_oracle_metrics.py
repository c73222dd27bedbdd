"""Pins for oracle.metrics (Sec. 5.1 reflection coefficient)."""
import numpy as np

from oracle import metrics


def test_reflection_coefficient_cases():
    rng = np.random.default_rng(0)
    E = rng.standard_normal((3, 50)) + 1j * rng.standard_normal((3, 50))
    assert metrics.reflection_coefficient(E, E) == 0.0
    assert metrics.reflection_coefficient(E, 0 * E) == 1.0
    d = 1e-3 * (rng.standard_normal((3, 50)) + 0j)
    expect = np.sum(np.abs(d) ** 2) / np.sum(np.abs(E) ** 2)
    assert abs(metrics.reflection_coefficient(E, E + d) - expect) < 1e-18
    assert abs(metrics.reflection_coefficient(7 * E, 7 * (E + d)) - expect) < 1e-18


def test_axis_field_is_current_over_contrast():
    chi = np.full((3, 5, 8), 2.0 + 0.5j)
    w = np.arange(3 * 3 * 5 * 8, dtype=complex).reshape(3, 3, 5, 8)
    E = metrics.axis_field(w, chi, 6)
    np.testing.assert_allclose(E, w[:, 1, 2, :6] / (2.0 + 0.5j))
