"""The no-allocation Poisson entry point against the plan-based one.

ibm_poisson_solve_noalloc serves callers that may not allocate device
memory while solving (their GPU memory belongs to a pool or framework that
only lends out its own buffers, or a cudaMalloc mid-run is not acceptable).
It must give the same answer as ibm_poisson_solve on an FP32 plan with the
same refinement count, within the FP32 parity tolerance used everywhere
else, and must not be disturbed by what the previous call left in the
shared static scratch -- so two different right-hand sides are solved back
to back.  This file is collected last so that a failure here does not stop
the other GPU tests.
"""

import numpy as np
import pytest

from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, grid, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("shape,refine", [((128, 128, 128), 1), ((48, 40, 96), 2), ((32, 32, 32), 0)])
def test_noalloc_matches_plan_solve_twice(shape, refine):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, refine)
    try:
        for call, wl in enumerate((40, 41)):
            b = synth.rhs_lowpass_noise(nx, ny, nz, kmax=12.0, workload=wl).astype(np.float32)
            rhs = torch.from_numpy(b).cuda()
            want = torch.empty_like(rhs)
            got = torch.full_like(rhs, float("nan"))
            ibm.ibm_poisson_solve(plan, rhs, want)
            ibm.ibm_poisson_solve_noalloc(nx, ny, nz, g[3:], refine, rhs, got)
            torch.cuda.synchronize()
            err = rel_l2(got.double().cpu().numpy(), want.double().cpu().numpy())
            assert err <= TOL_FP32, (call, err)
    finally:
        ibm.ibm_plan_destroy(plan)


def test_noalloc_rejects_grids_beyond_the_scratch():
    g = grid(256, 256, 256)
    x = torch.zeros(16, device="cuda")
    y = torch.zeros(16, device="cuda")
    with pytest.raises(ibm.IbmError) as e:
        ibm.ibm_poisson_solve_noalloc(256, 256, 256, g[3:], 1, x, y)
    assert e.value.code == ibm.IBM_ERR_ARG
    assert "scratch" in str(e.value)
