"""GPU axis field and reflection coefficient (Sec. 5.1) against the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import metrics
from oracle import operator as op
from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def test_axis_field_and_reflection_match_oracle():
    grid = (40, 23, 11)
    wl = workloads.waveguide(nx=40, absorber_len_um=0.2, src_x_um=0.1)
    ab = [dict(x0=30.0, length=10.0, degree=2, eps2_max=3.0)]
    plan = vie.vie_plan_create(grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, ab)
    chi = op.chi_from_permittivity(wl.eps, wl.eps_bg, ab)
    w1 = workloads.random_currents(grid, seed=91)
    w2 = w1 + 1e-3 * workloads.random_currents(grid, seed=92)
    n_keep = 30
    e1 = vie.vie_axis_field(plan, torch.from_numpy(w1.ravel()).cuda(), n_keep)
    e2 = vie.vie_axis_field(plan, torch.from_numpy(w2.ravel()).cuda(), n_keep)
    r1 = metrics.axis_field(w1, chi, n_keep)
    r2 = metrics.axis_field(w2, chi, n_keep)
    np.testing.assert_allclose(e1.cpu().numpy(), r1, rtol=1e-14, atol=0)
    R = vie.vie_reflection(e1, e2)
    R_ref = metrics.reflection_coefficient(r1, r2)
    assert abs(R - R_ref) <= 1e-12 * R_ref
    assert vie.vie_reflection(e1, e1) == 0.0


def test_slice_power_matches_oracle():
    grid = (30, 9, 5)
    eps = np.full((5, 9, 30), 2.085 + 0j)
    eps[1:4, 2:7, :] = 12.11
    plan = vie.vie_plan_create(grid, 0.02, 2 * math.pi / 1.55, 2.085)
    ab = [dict(x0=20.0, length=10.0, degree=2, eps2_max=3.0)]
    vie.vie_set_permittivity(plan, eps, ab)
    chi = op.chi_from_permittivity(eps, 2.085, ab)
    w = workloads.random_currents(grid, seed=93)
    wd = torch.from_numpy(w.ravel()).cuda()
    for ix in (0, 7, 25, 29):
        T = vie.vie_slice_power(plan, wd, ix)
        T_ref = metrics.slice_power(w, chi, ix)
        assert abs(T - T_ref) <= 1e-12 * T_ref
