"""The allocation-free operator entry point, vie_matvec_static_scratch.

It serves callers that cannot allocate device memory where they apply the
operator (memory owned by another allocator or held to a fixed budget), by
running the operator on a static workspace inside the library.  These tests
call it through the C ABI and compare it with vie_matvec, twice in a row, so
that leftover contents of the shared workspace from one call cannot leak into
the next, and check in a fresh process that the first call reserves no device
memory.  The file is named to be collected last.
"""
import ctypes
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from paper_1803_06237_gb300 import build, vie, workloads

pytestmark = pytest.mark.gpu

# same tolerances as the operator parity tests (relative L2)
TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    vie.load()


def _raw_call(plan, x, y, dtype_code):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return vie.load().vie_matvec_static_scratch(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                                ctypes.c_void_p(y.data_ptr()), dtype_code, stream)


@pytest.mark.parametrize("dtype,code", [(torch.complex128, vie.VIE_C128), (torch.complex64, vie.VIE_C64)])
def test_static_workspace_matches_matvec_twice(dtype, code):
    wl = workloads.waveguide()          # 600 x 23 x 11: the benchmark's plan
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps, [dict(x0=400.0, length=200.0, degree=2, eps2_max=7.4)])
    for seed in (1, 2):
        x = torch.from_numpy(workloads.random_currents(wl.grid, seed=seed).ravel()).to(dtype).cuda()
        y_ref = torch.empty_like(x)
        vie.vie_matvec(plan, x, y_ref)
        y = torch.full_like(x, float("nan"))
        assert _raw_call(plan, x, y, code) == 0, vie.vie_last_error()
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(y - y_ref) / torch.linalg.vector_norm(y_ref)).item()
        assert err <= TOL[dtype], err
    plan.close()


def test_static_workspace_rejects_plans_beyond_its_size():
    # 3 * ny * nz * Mx complex128 values must fit in 16 MiB; 3*50*40*200*16 B = 19.2 MB does not
    plan = vie.vie_plan_create((100, 50, 40), 0.02, 2 * math.pi / 1.55, 2.085)
    assert plan.info()["m"][0] == 200
    n3 = 3 * plan.n_vox
    x = torch.zeros(n3, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert _raw_call(plan, x, y, vie.VIE_C128) == 1
    assert "static workspace" in vie.vie_last_error()
    plan.close()


_FRESH = textwrap.dedent("""
    import ctypes, sys
    import torch
    sys.path.insert(0, {root!r})
    from paper_1803_06237_gb300 import vie, workloads
    torch.cuda.init()
    wl = workloads.waveguide()
    plan = vie.vie_plan_create(wl.grid, wl.h_um, wl.k0_per_um, wl.eps_bg)
    vie.vie_set_permittivity(plan, wl.eps)
    x = torch.from_numpy(workloads.random_currents(wl.grid, seed=3).ravel()).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = vie.load().vie_matvec_static_scratch(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()), vie.VIE_C64,
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    print("STATUS", st, "FREE_BEFORE", free0, "FREE_AFTER", free1)
""")


def test_first_call_in_fresh_process_reserves_no_memory():
    """A process that made a plan and never applied the operator: its first
    static-workspace call must not change the device's free memory (the plan
    creation already loaded the library part that holds the static array)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("STATUS")][-1].split()
    status, free0, free1 = int(line[1]), int(line[3]), int(line[5])
    assert status == 0
    assert free1 == free0, (free0, free1, free0 - free1)
