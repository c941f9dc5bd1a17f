"""The no-allocation Poisson entry point against the plan-based one and the oracle.

ibm_poisson_solve_noalloc serves callers that may not allocate device
memory while solving (their GPU memory belongs to a pool or framework that
only lends out its own buffers, or a cudaMalloc mid-run is not acceptable).
It must give the same answer as ibm_poisson_solve on an FP32 plan with the
same refinement count, and both must match the FP64 oracle within the FP32
parity tolerance used everywhere else.  It must not be disturbed by what
the previous call left in the shared static scratch, so two different
right-hand sides are solved back to back, and it reports a clean device
error word through its status argument.  The shapes cover the one-CTA plane
transforms (128^3, 48x40x96, 32^3) and a 256x8x256 grid whose planes take
the split x / z passes, as a plan of that shape does.  This file is
collected last so that a failure here does not stop the other GPU tests.
"""

import ctypes

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, grid, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("shape,refine", [((128, 128, 128), 1), ((48, 40, 96), 2), ((32, 32, 32), 0),
                                          ((256, 8, 256), 1)])
def test_noalloc_matches_plan_solve_and_oracle_twice(shape, refine):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, refine)
    try:
        for call, wl in enumerate((40, 41)):
            b = synth.rhs_lowpass_noise(nx, ny, nz, kmax=12.0, workload=wl).astype(np.float32)
            ref, _ = O.poisson_solve(b.astype(np.float64), g)
            rhs = torch.from_numpy(b).cuda()
            want = torch.empty_like(rhs)
            got = torch.full_like(rhs, float("nan"))
            status = ctypes.c_int(-1)
            ibm.ibm_poisson_solve(plan, rhs, want)
            ibm.ibm_poisson_solve_noalloc(nx, ny, nz, g[3:], refine, rhs, got, status=status)
            torch.cuda.synchronize()
            assert status.value == 0, (call, status.value)
            got_h, want_h = got.double().cpu().numpy(), want.double().cpu().numpy()
            err_plan = rel_err(got_h, want_h)
            assert err_plan <= TOL_FP32, (call, err_plan)
            err_oracle = rel_err(got_h, ref)
            assert err_oracle <= TOL_FP32, (call, err_oracle)
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
