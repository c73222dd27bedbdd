"""Reduced versions of the parameter studies of Sec. 5 on the GPU
(paper_1803_06237_gb300/sweeps.py): the absorber-length study of Sec. 5.1
(R falls with the absorber length, faster for a smoother profile) and the
Bragg-grating transmission of Sec. 5.2 through the batch path (the batched
solve of several wavelengths equals their single solves)."""
import pytest
import torch

from paper_1803_06237_gb300 import build, learned, sweeps, vie, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def test_reflection_falls_with_absorber_length_and_degree():
    """A 1.5 um strip (90 x 30 x 12 voxels of 50/3 nm) with absorbers of 225,
    450 and 900 nm against a 1800 nm reference, d = 0 and 1, R_rt = 1e-25."""
    out = sweeps.rl_sweep([225.0, 450.0, 900.0], degrees=(0, 1), r_rt=1e-25, ref_nm=1800.0, tol=1e-9,
                          body_nm=1500.0)
    R0 = out["degrees"]["0"]["R"]
    R1 = out["degrees"]["1"]["R"]
    print(out)
    assert R0[0] > R0[1] > R0[2] and R1[0] > R1[1] > R1[2], (R0, R1)
    assert R1[-1] < R0[-1]
    for d in ("0", "1"):
        assert out["degrees"][d]["true_residual_max"] <= 1e-9


def test_bragg_batch_equals_single_solves():
    """Three wavelengths of a 10-period grating solved together (one plan,
    spectrum and preconditioner per wavelength) give the transmission of
    their single solves."""
    lams = [1.52, 1.545, 1.57]
    out = sweeps.bragg_sweep(lams, periods=10, tol=1e-8, batch=3)
    assert out["converged"] == 3
    for lam, T in zip(lams, out["T"]):
        wl = workloads.bragg_grating(lam, periods=10)
        plan, b = learned.setup_problem(wl)
        x = torch.zeros_like(b)
        info = vie.vie_solve(plan, b, x, 1e-8, mode=vie.VIE_SOLVE_MIXED, restart=30)
        assert info["converged"]
        T1 = vie.vie_slice_power(plan, x, int(wl.name.split("_x")[1]))
        assert abs(T1 - T) <= 1e-5 * T, (lam, T, T1)
        plan.close()
