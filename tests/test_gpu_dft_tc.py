"""Tensor-core DFT plane transforms (plane mode -1) against the oracle.

FP32 plans whose planes are short (nx, nz in {8, 16, 24, 32, 48, 64}) can
run the x-z transforms as dense DFT matrix products on the tensor cores
(split-TF32 operands, FP32 accumulation).  The solves in that mode are
compared with the oracle's eigen-solves (Poisson and the three Helmholtz
field kinds, wall-bounded and triply periodic) and with the FFT plane
modes: after one refinement step the FP32 bar (1e-6 relative L2); without
refinement the error stays at the FFT path's order.  Shapes cover every
supported length, non-square planes, a plane count that leaves the last
group of planes partly empty, and the three-field stage launches.
"""

import os

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, dev, grid, host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DFT = -1

SHAPES = [(8, 9, 8), (16, 16, 16), (24, 11, 24), (32, 32, 32), (48, 20, 48), (64, 10, 64),
          (64, 10, 32), (32, 13, 64), (16, 33, 48), (48, 11, 8)]


def _plan(nx, ny, nz, g, refine, mode, bc=None):
    os.environ["IBM_PLANE_MODE"] = str(mode)
    try:
        if bc is None:
            return ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, refine)
        return ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, refine, bc=bc)
    finally:
        del os.environ["IBM_PLANE_MODE"]


def _poisson(plan, b32):
    rhs = dev(b32, torch.float32)
    phi = torch.empty_like(rhs)
    ibm.ibm_poisson_solve(plan, rhs, phi)
    torch.cuda.synchronize()
    return host(phi)


@pytest.mark.parametrize("shape", SHAPES)
def test_dft_mode_solves_match_oracle(shape):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    b = synth.white_noise(nx, ny, nz, workload=91, stream=0) + 0.3
    b32 = b.astype(np.float32).astype(np.float64)
    ref, _ = O.poisson_solve(b32, g)
    errs = {}
    for refine in (0, 1):
        for mode in (DFT, 0):
            plan = _plan(nx, ny, nz, g, refine, mode)
            try:
                errs[(refine, mode)] = rel_err(_poisson(plan, b32), ref)
                if refine == 1 and mode == DFT:
                    for kind in (ibm.IBM_FIELD_CELL_NEUMANN, ibm.IBM_FIELD_CELL_DIRICHLET,
                                 ibm.IBM_FIELD_FACE_DIRICHLET):
                        href = O.helmholtz_solve(b32, g, 0.01, kind)
                        rhs = dev(b32, torch.float32)
                        u = torch.empty_like(rhs)
                        ibm.ibm_helmholtz_solve(plan, 0.01, kind, rhs, u)
                        torch.cuda.synchronize()
                        got = host(u)
                        if kind == ibm.IBM_FIELD_FACE_DIRICHLET:
                            got, href = got[1:], href[1:]
                        assert rel_err(got, href) <= TOL_FP32, (kind, rel_err(got, href))
                ibm.ibm_plan_check(plan)
            finally:
                ibm.ibm_plan_destroy(plan)
    assert errs[(1, DFT)] <= TOL_FP32, errs
    # unrefined: the DFT products' rounding stays within a few times the FFT path's
    assert errs[(0, DFT)] <= 5.0 * errs[(0, 0)] + 1e-7, errs


def test_dft_mode_listed_only_for_short_fp32_planes():
    g = grid(128, 8, 128)
    with pytest.raises(ibm.IbmError) as e:
        _plan(128, 8, 128, g, 1, DFT)
    assert e.value.code == ibm.IBM_ERR_UNSUPPORTED
    g = grid(32, 8, 32)
    os.environ["IBM_PLANE_MODE"] = str(DFT)
    try:
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_plan_create(32, 8, 32, g[3:], ibm.IBM_FP64, 0)
        assert e.value.code == ibm.IBM_ERR_UNSUPPORTED
    finally:
        del os.environ["IBM_PLANE_MODE"]


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 12, 16), (64, 12, 64)])
def test_dft_mode_triply_periodic(shape):
    nx, ny, nz = shape
    g = grid(nx, ny, nz, Ly=3.0)
    b = synth.white_noise(nx, ny, nz, workload=92, stream=0) + 0.4
    b32 = b.astype(np.float32).astype(np.float64)
    ref, _ = O.poisson_solve(b32, g, ybc=O.PERIODIC)
    plan = _plan(nx, ny, nz, g, 1, DFT, bc=ibm.IBM_BC_TRIPLY_PERIODIC)
    try:
        assert rel_err(_poisson(plan, b32), ref) <= TOL_FP32
        href = O.helmholtz_solve(b32, g, 0.02, O.PERIODIC)
        rhs = dev(b32, torch.float32)
        u = torch.empty_like(rhs)
        ibm.ibm_helmholtz_solve(plan, 0.02, ibm.IBM_FIELD_PERIODIC, rhs, u)
        torch.cuda.synchronize()
        assert rel_err(host(u), href) <= TOL_FP32
    finally:
        ibm.ibm_plan_destroy(plan)


def test_dft_mode_in_place_and_repeated():
    """rhs == phi, and ten solves in a row give identical bytes."""
    nx, ny, nz = 32, 24, 32
    g = grid(nx, ny, nz)
    b32 = (synth.white_noise(nx, ny, nz, workload=93, stream=0) + 0.1).astype(np.float32).astype(np.float64)
    ref, _ = O.poisson_solve(b32, g)
    plan = _plan(nx, ny, nz, g, 1, DFT)
    try:
        x = dev(b32, torch.float32)
        ibm.ibm_poisson_solve(plan, x, x)
        torch.cuda.synchronize()
        assert rel_err(host(x), ref) <= TOL_FP32
        rhs = dev(b32, torch.float32)
        outs = []
        for _ in range(10):
            phi = torch.empty_like(rhs)
            ibm.ibm_poisson_solve(plan, rhs, phi)
            outs.append(phi)
        torch.cuda.synchronize()
        assert all(torch.equal(outs[0], o) for o in outs[1:])
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("path", ["tensor_memory", "bulk_copy"])
def test_bounded_wait_runs_out_and_plan_stays_usable(path):
    """A wait that cannot complete gives up after its limit, reports
    IBM_ERR_TIMEOUT through the plan's error word and leaves the context
    usable: the same plan then solves (in the tensor-core DFT mode) to the
    oracle.  Two paths: a wait on an mbarrier that nothing completes while
    the CTA holds tensor memory (the tensor-core kernels' wait, which frees
    the memory before returning), and a wait on a real in-bounds bulk copy
    whose barrier expects twice its bytes (the tile kernels' wait, which
    waits once more for copies in flight before returning; two limits)."""
    import time
    code = {"tensor_memory": ibm.IBM_SELFTEST_TENSOR_MEMORY, "bulk_copy": ibm.IBM_SELFTEST_BULK_COPY}[path]
    nx, ny, nz = 32, 16, 32
    g = grid(nx, ny, nz)
    plan = _plan(nx, ny, nz, g, 1, DFT)
    try:
        t0 = time.perf_counter()
        ibm.ibm_selftest_timeout(plan, 50.0, path=code)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert 0.04 <= dt < 5.0, dt
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_plan_check(plan)
        assert e.value.code == ibm.IBM_ERR_TIMEOUT
        ibm.ibm_plan_check(plan)  # the word was cleared
        b32 = (synth.white_noise(nx, ny, nz, workload=94, stream=0) + 0.2).astype(np.float32).astype(np.float64)
        ref, _ = O.poisson_solve(b32, g)
        assert rel_err(_poisson(plan, b32), ref) <= TOL_FP32
        ibm.ibm_plan_check(plan)
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_selftest_timeout(plan, 0.0, path=code)
        assert e.value.code == ibm.IBM_ERR_ARG
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_selftest_timeout(plan, 10.0, path=7)
        assert e.value.code == ibm.IBM_ERR_ARG
    finally:
        ibm.ibm_plan_destroy(plan)
