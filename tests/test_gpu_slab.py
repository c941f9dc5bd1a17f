"""GPU parity of the fused slab solve path against the FP64 oracle.

FP32 plans on wall-bounded grids with ny and nz in {64, 128, 256} solve
single fields in three passes: x rows into a kx-major spectrum, one cluster
kernel per kx slab (z transforms, the segmented y sweep with its carries
crossing the cluster, the FP64 zero mode), x rows back.  Every (ny, nz)
pair, i.e. every cluster size (2, 4, 8 CTAs) and z length, is solved here
against the oracle, with ragged and radix-3 x lengths, non-zero-mean
right-hand sides (the removed mean), in place, with 0, 1 and 2 refinement
steps, and for the Helmholtz kinds the path takes (cell Neumann, cell
Dirichlet) next to the one it leaves to the split passes (face Dirichlet).
The slab and split paths of the same plan agree to FP32 rounding.
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

SLAB_SHAPES = [
    (48, 64, 64),     # 2-CTA clusters, radix-3 x
    (384, 64, 128),   # longest radix-3 x row
    (16, 64, 256),
    (256, 128, 64),   # 4-CTA clusters
    (12, 128, 256),
    (96, 256, 128),   # 8-CTA clusters
    (24, 256, 64),
    (16, 256, 256),   # 8-CTA clusters, 256-point z rows (the 256^3 configuration's slabs)
    (48, 256, 256),
]


def _plan(shape, refine, slab=True):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    old = os.environ.get("IBM_SLAB")
    os.environ["IBM_SLAB"] = "1" if slab else "0"
    try:
        return ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, refine), g
    finally:
        if old is None:
            del os.environ["IBM_SLAB"]
        else:
            os.environ["IBM_SLAB"] = old


@pytest.mark.parametrize("shape", SLAB_SHAPES)
@pytest.mark.parametrize("refine", [0, 1, 2])
def test_slab_poisson_matches_oracle(shape, refine):
    nx, ny, nz = shape
    plan, g = _plan(shape, refine)
    try:
        b = (synth.white_noise(nx, ny, nz, workload=51, stream=refine) + 0.25).astype(np.float32)
        ref, mean_b = O.poisson_solve(b.astype(np.float64), g)
        rhs = dev(b, torch.float32)
        phi = torch.empty_like(rhs)
        info = ibm.ibm_poisson_solve(plan, rhs, phi, info=True)
        err = rel_err(host(phi), ref)
        # without refinement the FP32 sweep and transforms alone (about
        # 1e-6 at 256 rows); with it the benchmark spec's 1e-6
        assert err <= (TOL_FP32 if refine else 1e-5), (shape, refine, err)
        # the plane sums come from FP32 transforms of nx nz values: ~log2(nx nz) eps32 relative
        assert abs(info["removed_mean"] - mean_b) <= 1e-5 * abs(mean_b), (info["removed_mean"], mean_b)
        assert info["refine_iters"] == refine
        assert info["phase_ms"]["forward"] > 0 and info["phase_ms"]["pencil"] > 0
        print("slab", shape, refine, err)
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("shape", [(48, 64, 64), (256, 128, 64), (96, 256, 128)])
def test_slab_and_split_paths_agree_in_place(shape):
    """The slab path in place (rhs == phi) against the split passes of a plan
    made with IBM_SLAB=0, both one refinement step."""
    nx, ny, nz = shape
    b = synth.rhs_lowpass_noise(nx, ny, nz, kmax=8.0, workload=52).astype(np.float32)
    outs = []
    for slab in (True, False):
        plan, g = _plan(shape, 1, slab)
        try:
            x = dev(b, torch.float32)
            ibm.ibm_poisson_solve(plan, x, x)
            torch.cuda.synchronize()
            outs.append(host(x))
            ibm.ibm_plan_check(plan)
        finally:
            ibm.ibm_plan_destroy(plan)
    ref, _ = O.poisson_solve(b.astype(np.float64), grid(nx, ny, nz))
    assert rel_err(outs[0], ref) <= TOL_FP32
    assert rel_err(outs[0], outs[1]) <= TOL_FP32


@pytest.mark.parametrize("shape", [(48, 64, 64), (12, 128, 256), (96, 256, 128), (16, 256, 256)])
@pytest.mark.parametrize("bc", [ibm.IBM_FIELD_CELL_NEUMANN, ibm.IBM_FIELD_CELL_DIRICHLET,
                                ibm.IBM_FIELD_FACE_DIRICHLET])
@pytest.mark.parametrize("c", [5e-6, 0.05])
def test_slab_helmholtz_matches_oracle(shape, bc, c):
    nx, ny, nz = shape
    plan, g = _plan(shape, 1)
    try:
        r = synth.white_noise(nx, ny, nz, workload=53, stream=bc).astype(np.float32).astype(np.float64)
        ref = O.helmholtz_solve(r, g, c, bc)
        rhs = dev(r, torch.float32)
        u = torch.empty_like(rhs)
        ibm.ibm_helmholtz_solve(plan, c, bc, rhs, u)
        torch.cuda.synchronize()
        assert rel_err(host(u), ref) <= TOL_FP32
    finally:
        ibm.ibm_plan_destroy(plan)


# The refinement's first pass for 256-point x rows runs in its streaming
# form (each CTA walks up a range of y planes for one block of 32 z rows, x
# planes staged in a ring of shared-memory slots, residual and transform in
# two warp groups); IBM_RES_STREAM=0 keeps the block form.  Shapes with one
# CTA per 4 planes (ny = 64), several z blocks per plane and 64 to 256 z
# rows, against the oracle and against the block form.
STREAM_SHAPES = [(256, 64, 64), (256, 128, 128), (256, 64, 256)]


def _with_env(name, value, fn):
    old = os.environ.get(name)
    os.environ[name] = value
    try:
        return fn()
    finally:
        if old is None:
            del os.environ[name]
        else:
            os.environ[name] = old


@pytest.mark.parametrize("shape", STREAM_SHAPES)
@pytest.mark.parametrize("refine", [1, 2])
def test_stream_residual_poisson_matches_oracle(shape, refine):
    nx, ny, nz = shape
    plan, g = _plan(shape, refine)
    try:
        b = (synth.white_noise(nx, ny, nz, workload=54, stream=refine) + 0.5).astype(np.float32)
        ref, _ = O.poisson_solve(b.astype(np.float64), g)
        rhs = dev(b, torch.float32)
        phi = torch.empty_like(rhs)
        ibm.ibm_poisson_solve(plan, rhs, phi)
        torch.cuda.synchronize()
        ibm.ibm_plan_check(plan)
        err = rel_err(host(phi), ref)
        assert err <= TOL_FP32, (shape, refine, err)
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("bc", [ibm.IBM_FIELD_CELL_NEUMANN, ibm.IBM_FIELD_CELL_DIRICHLET])
@pytest.mark.parametrize("c", [5e-6, 0.05])
def test_stream_residual_helmholtz_matches_oracle(bc, c):
    shape = (256, 64, 128)
    nx, ny, nz = shape
    plan, g = _plan(shape, 1)
    try:
        r = synth.white_noise(nx, ny, nz, workload=55, stream=bc).astype(np.float32).astype(np.float64)
        ref = O.helmholtz_solve(r, g, c, bc)
        rhs = dev(r, torch.float32)
        u = torch.empty_like(rhs)
        ibm.ibm_helmholtz_solve(plan, c, bc, rhs, u)
        torch.cuda.synchronize()
        ibm.ibm_plan_check(plan)
        assert rel_err(host(u), ref) <= TOL_FP32
    finally:
        ibm.ibm_plan_destroy(plan)


def test_stream_and_block_residual_agree():
    shape = (256, 128, 64)
    nx, ny, nz = shape
    b = synth.rhs_lowpass_noise(nx, ny, nz, kmax=8.0, workload=56).astype(np.float32)
    plan, g = _plan(shape, 1)
    try:
        def solve():
            x = torch.empty((ny, nz, nx), device="cuda", dtype=torch.float32)
            ibm.ibm_poisson_solve(plan, dev(b, torch.float32), x)
            torch.cuda.synchronize()
            ibm.ibm_plan_check(plan)
            return host(x)
        streamed = solve()
        block = _with_env("IBM_RES_STREAM", "0", solve)
    finally:
        ibm.ibm_plan_destroy(plan)
    ref, _ = O.poisson_solve(b.astype(np.float64), g)
    assert rel_err(streamed, ref) <= TOL_FP32
    # the same FP32 residual, summed in the same order: both forms agree to
    # the rounding of the correction (about 1e-2 of a 1e-6 correction)
    assert rel_err(streamed, block) <= 1e-7
