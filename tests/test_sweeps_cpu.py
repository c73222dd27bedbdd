"""Host-side analysis of the Sec. 5 studies (no GPU): the slope fit of
log R against log L (Sec. 4.3 predicts -2 (d + 1)) and the band-gap read-out
of a transmission spectrum (Sec. 5.2)."""
import numpy as np

from paper_1803_06237_gb300 import sweeps


def test_fit_slope_of_a_power_law():
    L = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    assert abs(sweeps.fit_slope(L, 3e-4 * L ** -4.0) + 4.0) < 1e-12
    R = 3e-4 * L ** -4.0
    R[-1] = 1e-3                       # outside the window: ignored
    assert abs(sweeps.fit_slope(L, R, 2.0, 8.0) + 4.0) < 1e-12
    assert sweeps.fit_slope(L, np.full(5, 1e-15)) is None
    # values at or below the floor are left out of the fit
    R = 2.0 * L ** -6.0
    R[2] = 1e-13
    assert abs(sweeps.fit_slope(L, R) + 6.0) < 1e-12


def test_band_gap_takes_the_widest_run_below_the_level():
    lam = np.linspace(1.50, 1.60, 11)
    T = np.array([1.0, 0.9, 0.3, 0.9, 0.2, 0.1, 0.05, 0.2, 0.8, 1.0, 1.0])
    gap = sweeps.band_gap(lam, T)
    assert abs(gap["centre_um"] - 1.555) < 1e-12 and abs(gap["width_um"] - 0.03) < 1e-12
    assert sweeps.band_gap(lam, np.ones(11)) is None
    # a single point below the level is a gap of zero width
    T1 = np.ones(11)
    T1[3] = 0.1
    g1 = sweeps.band_gap(lam, T1)
    assert abs(g1["centre_um"] - lam[3]) < 1e-12 and g1["width_um"] == 0.0
