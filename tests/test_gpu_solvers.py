"""GPU parity of the Poisson and Helmholtz solves against the FP64 oracle.

Every case builds a seeded synthetic right-hand side, runs the CUDA path
through the C ABI and compares element by element with the oracle
(relative L2).  Shapes cover the one-CTA-per-plane transform path, the
split x/z path (planes larger than shared memory), radix-3 sizes, ragged
pencil tiles and the smallest supported grid.
"""

import math
import os

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, TOL_FP64, dev, grid, host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [
    (32, 32, 32),     # workload-0 grid, plane path
    (8, 8, 8),        # smallest grid
    (12, 10, 24),     # radix 3, odd ny, ragged pencil tile
    (48, 40, 48),     # radix 3
    (96, 33, 64),     # mixed shape, odd ny
    (256, 12, 256),   # plane larger than shared memory (split x/z path)
    (384, 9, 32),     # longest radix-3 row, split path
    (16, 200, 24),    # pencils of 200: FP32 split-component block solve, FP64 serial sweep
    (32, 300, 16),    # pencils longer than 256: serial sweep in both precisions
]


def _plan(nx, ny, nz, g, prec, refine=1):
    return ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, refine)


@pytest.mark.parametrize("shape", SHAPES)
def test_poisson_fp64_matches_oracle(shape):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    b = synth.white_noise(nx, ny, nz, workload=10, stream=0) + 0.3
    ref, mean_b = O.poisson_solve(b, g)
    plan = _plan(nx, ny, nz, g, ibm.IBM_FP64)
    try:
        rhs = dev(b, torch.float64)
        phi = torch.empty_like(rhs)
        info = ibm.ibm_poisson_solve(plan, rhs, phi, info=True)
        assert rel_err(host(phi), ref) <= TOL_FP64
        assert abs(info["removed_mean"] - mean_b) <= 1e-12 * max(1.0, abs(mean_b))
        assert info["rel_residual"] < 1e-12
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("refine", [1, 2])
def test_poisson_fp32_refined_matches_oracle(shape, refine):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    b32 = synth.white_noise(nx, ny, nz, workload=11, stream=0).astype(np.float32)
    ref, _ = O.poisson_solve(b32.astype(np.float64), g)
    plan = _plan(nx, ny, nz, g, ibm.IBM_FP32_REFINED, refine)
    try:
        rhs = dev(b32, torch.float32)
        phi = torch.empty_like(rhs)
        info = ibm.ibm_poisson_solve(plan, rhs, phi, info=True)
        assert rel_err(host(phi), ref) <= TOL_FP32
        assert info["refine_iters"] == refine
    finally:
        ibm.ibm_plan_destroy(plan)


def test_poisson_workload0_eigen_rhs_both_precisions():
    """Workload 0: 32^3, sum of 4 grid eigenfunctions + noise 1e-3."""
    g = grid(32, 32, 32)
    b, _ = synth.rhs_eigen_sum(32, 32, 32, workload=0)
    for prec, dt, tol in ((ibm.IBM_FP64, torch.float64, TOL_FP64), (ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32)):
        bb = b.astype(np.float32).astype(np.float64) if dt == torch.float32 else b
        ref, _ = O.poisson_solve(bb, g)
        plan = _plan(32, 32, 32, g, prec)
        try:
            rhs = dev(bb, dt)
            phi = torch.empty_like(rhs)
            ibm.ibm_poisson_solve(plan, rhs, phi)
            torch.cuda.synchronize()
            assert rel_err(host(phi), ref) <= tol
        finally:
            ibm.ibm_plan_destroy(plan)


def test_poisson_in_place_and_128_lowpass():
    """Workload 1 right-hand side (128^3 low-passed noise), rhs == phi."""
    g = grid(128, 128, 128)
    b = synth.rhs_lowpass_noise(128, 128, 128, kmax=32.0, workload=1).astype(np.float32)
    ref, _ = O.poisson_solve(b.astype(np.float64), g)
    plan = _plan(128, 128, 128, g, ibm.IBM_FP32_REFINED, 1)
    try:
        x = dev(b, torch.float32)
        info = ibm.ibm_poisson_solve(plan, x, x, info=True)
        err = rel_err(host(x), ref)
        assert err <= TOL_FP32, (err, info)
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("shape", [(32, 32, 32), (12, 10, 24), (256, 12, 256), (48, 17, 96), (24, 129, 16)])
@pytest.mark.parametrize("bc", [ibm.IBM_FIELD_CELL_NEUMANN, ibm.IBM_FIELD_CELL_DIRICHLET,
                                ibm.IBM_FIELD_FACE_DIRICHLET])
@pytest.mark.parametrize("c", [5e-6, 0.05])
def test_helmholtz_matches_oracle(shape, bc, c):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    r = synth.white_noise(nx, ny, nz, workload=12, stream=bc)
    for prec, dt, tol in ((ibm.IBM_FP64, torch.float64, TOL_FP64), (ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32)):
        rr = r.astype(np.float32).astype(np.float64) if dt == torch.float32 else r
        ref = O.helmholtz_solve(rr, g, c, bc)
        plan = _plan(nx, ny, nz, g, prec, 1)
        try:
            rhs = dev(rr, dt)
            u = torch.empty_like(rhs)
            ibm.ibm_helmholtz_solve(plan, c, bc, rhs, u)
            torch.cuda.synchronize()
            got = host(u)
            assert rel_err(got, ref) <= tol, (prec, rel_err(got, ref))
            if bc == ibm.IBM_FIELD_FACE_DIRICHLET:
                assert np.all(got[0] == 0.0)
        finally:
            ibm.ibm_plan_destroy(plan)


# Planes with a cluster transform (C CTAs per plane exchanging rows and
# columns through distributed shared memory), each solved in every plane
# mode the shape has: 0 split x/z passes, 1 one CTA per plane, 2/4/8 cluster.
PLANE_MODE_SHAPES = [
    (64, 10, 64), (96, 9, 96), (128, 12, 128), (192, 8, 192), (256, 9, 256),
    (384, 8, 256), (256, 8, 128), (128, 8, 256), (384, 8, 384), (512, 8, 256),
]


def _plan_in_mode(nx, ny, nz, g, prec, refine, mode):
    os.environ["IBM_PLANE_MODE"] = str(mode)
    try:
        return ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, refine)
    except ibm.IbmError as e:
        assert e.code == ibm.IBM_ERR_UNSUPPORTED
        return None
    finally:
        del os.environ["IBM_PLANE_MODE"]


@pytest.mark.parametrize("shape", PLANE_MODE_SHAPES)
def test_every_plane_mode_matches_oracle(shape):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    b = synth.white_noise(nx, ny, nz, workload=13, stream=0) + 0.2
    b32 = b.astype(np.float32).astype(np.float64)
    ref64, _ = O.poisson_solve(b, g)
    ref32, _ = O.poisson_solve(b32, g)
    href = O.helmholtz_solve(b32, g, 0.01, ibm.IBM_FIELD_CELL_DIRICHLET)
    ran = set()
    for mode in (0, 1, 2, 4, 8):
        for prec, dt, tol, bb, ref in ((ibm.IBM_FP64, torch.float64, TOL_FP64, b, ref64),
                                       (ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32, b32, ref32)):
            plan = _plan_in_mode(nx, ny, nz, g, prec, 1, mode)
            if plan is None:
                continue
            ran.add(mode)
            try:
                rhs = dev(bb, dt)
                phi = torch.empty_like(rhs)
                ibm.ibm_poisson_solve(plan, rhs, phi)
                torch.cuda.synchronize()
                assert rel_err(host(phi), ref) <= tol, (mode, prec, rel_err(host(phi), ref))
                if prec == ibm.IBM_FP32_REFINED:
                    u = torch.empty_like(rhs)
                    ibm.ibm_helmholtz_solve(plan, 0.01, ibm.IBM_FIELD_CELL_DIRICHLET, rhs, u)
                    torch.cuda.synchronize()
                    assert rel_err(host(u), href) <= tol, (mode, rel_err(host(u), href))
                ibm.ibm_plan_check(plan)
            finally:
                ibm.ibm_plan_destroy(plan)
    assert 0 in ran and any(m >= 2 for m in ran), ran


PENCIL_MODE_SHAPES = [(32, 32, 32), (12, 10, 24), (48, 17, 96), (24, 129, 16), (16, 200, 24), (32, 300, 16)]


@pytest.mark.parametrize("shape", PENCIL_MODE_SHAPES)
def test_every_pencil_kernel_matches_oracle(shape):
    """IBM_PENCIL_MODE 1 (warp-parallel blocks), 2 (tile sweep), 3 (streaming sweep), 4 (segmented sweep)."""
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    b = synth.white_noise(nx, ny, nz, workload=14, stream=0) + 0.1
    b32 = b.astype(np.float32).astype(np.float64)
    ref64, _ = O.poisson_solve(b, g)
    ref32, _ = O.poisson_solve(b32, g)
    helm = {bc: O.helmholtz_solve(b32, g, 0.02, bc)
            for bc in (ibm.IBM_FIELD_CELL_NEUMANN, ibm.IBM_FIELD_FACE_DIRICHLET)}
    for mode in (1, 2, 3, 4):
        for prec, dt, tol, bb, ref in ((ibm.IBM_FP64, torch.float64, TOL_FP64, b, ref64),
                                       (ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32, b32, ref32)):
            os.environ["IBM_PENCIL_MODE"] = str(mode)
            try:
                plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
            finally:
                del os.environ["IBM_PENCIL_MODE"]
            try:
                rhs = dev(bb, dt)
                phi = torch.empty_like(rhs)
                ibm.ibm_poisson_solve(plan, rhs, phi)
                torch.cuda.synchronize()
                assert rel_err(host(phi), ref) <= tol, (mode, prec, rel_err(host(phi), ref))
                if prec == ibm.IBM_FP32_REFINED:
                    for bc, href in helm.items():
                        u = torch.empty_like(rhs)
                        ibm.ibm_helmholtz_solve(plan, 0.02, bc, rhs, u)
                        torch.cuda.synchronize()
                        assert rel_err(host(u), href) <= tol, (mode, bc, rel_err(host(u), href))
                ibm.ibm_plan_check(plan)
            finally:
                ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("shape", [(32, 256, 32), (16, 500, 16), (24, 129, 16)])
def test_segmented_sweep_unrefined_fp32_accuracy(shape):
    """Without refinement the FP32 error is the sweep's own: the segmented
    sweep (pivot prefix, carries combined across warps) stays within a small
    factor of the single two-ended sweep on long, near-singular pencils."""
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    b32 = synth.white_noise(nx, ny, nz, workload=15, stream=0).astype(np.float32)
    ref, _ = O.poisson_solve(b32.astype(np.float64), g)
    errs = {}
    for mode in (3, 4):
        os.environ["IBM_PENCIL_MODE"] = str(mode)
        try:
            plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, 0)
        finally:
            del os.environ["IBM_PENCIL_MODE"]
        try:
            rhs = dev(b32, torch.float32)
            phi = torch.empty_like(rhs)
            ibm.ibm_poisson_solve(plan, rhs, phi)
            torch.cuda.synchronize()
            errs[mode] = rel_err(host(phi), ref)
        finally:
            ibm.ibm_plan_destroy(plan)
    assert errs[4] <= 1e-5, errs
    assert errs[4] <= 2.0 * errs[3] + 1e-7, errs


def test_fp32_fields_must_be_16_byte_aligned():
    """The four-point residual and the vector loads need 16-byte aligned
    fields: an element-aligned view at an odd offset is refused before any
    launch, the aligned view of the same buffer solves."""
    nx, ny, nz = 32, 24, 16
    g = grid(nx, ny, nz)
    n = nx * ny * nz
    b32 = synth.white_noise(nx, ny, nz, workload=16, stream=0).astype(np.float32)
    ref, _ = O.poisson_solve(b32.astype(np.float64), g)
    plan = _plan(nx, ny, nz, g, ibm.IBM_FP32_REFINED, 2)
    try:
        buf = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        out = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        for off in (1, 3):
            with pytest.raises(ibm.IbmError) as e:
                ibm.ibm_poisson_solve(plan, buf[off:off + n].view(ny, nz, nx), out[off:off + n].view(ny, nz, nx))
            assert e.value.code == ibm.IBM_ERR_ARG
        rhs = buf[4:4 + n].view(ny, nz, nx)
        rhs.copy_(dev(b32, torch.float32))
        phi = out[4:4 + n].view(ny, nz, nx)
        ibm.ibm_poisson_solve(plan, rhs, phi)
        torch.cuda.synchronize()
        assert rel_err(host(phi), ref) <= TOL_FP32
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
@pytest.mark.parametrize("shape", [(32, 24, 16), (48, 17, 96)])
def test_solves_with_wall_data_match_oracle(prec, shape):
    """Inhomogeneous wall data (Appendix B's boundary right-hand sides, BC2.2):
    Poisson with dphi/dy on both walls and Helmholtz with wall values / wall
    slopes for every field kind, against the oracle; rhs left untouched."""
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    tol = TOL_FP64 if prec == ibm.IBM_FP64 else TOL_FP32
    rng = np.random.default_rng(nx + ny)
    b = synth.white_noise(nx, ny, nz, workload=17, stream=0).astype(npdt).astype(np.float64)
    lo, hi = (rng.standard_normal((nz, nx)).astype(npdt).astype(np.float64) for _ in range(2))
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        rhs, glo, ghi = dev(b, dt), dev(lo, dt), dev(hi, dt)
        keep = rhs.clone()
        phi = torch.empty_like(rhs)
        info = ibm.ibm_poisson_solve_bc(plan, rhs, phi, glo, ghi, info=True)
        ref, removed = O.poisson_solve(b, g, q_lo=lo, q_hi=hi)
        assert rel_err(host(phi), ref) <= tol
        assert abs(info["removed_mean"] - removed) <= 1e-5 * max(1.0, abs(removed))
        for bc in (ibm.IBM_FIELD_CELL_NEUMANN, ibm.IBM_FIELD_CELL_DIRICHLET, ibm.IBM_FIELD_FACE_DIRICHLET):
            u = torch.empty_like(rhs)
            ibm.ibm_helmholtz_solve_bc(plan, 0.02, bc, rhs, u, glo, ghi)
            torch.cuda.synchronize()
            href = O.helmholtz_solve(b, g, 0.02, bc, lo, hi)
            assert rel_err(host(u), href) <= tol, bc
            # one wall only
            ibm.ibm_helmholtz_solve_bc(plan, 0.02, bc, rhs, u, None, ghi)
            torch.cuda.synchronize()
            assert rel_err(host(u), O.helmholtz_solve(b, g, 0.02, bc, None, hi)) <= tol, bc
        assert torch.equal(rhs, keep)
        # in place
        ibm.ibm_helmholtz_solve_bc(plan, 0.02, ibm.IBM_FIELD_CELL_DIRICHLET, rhs, rhs, glo, ghi)
        torch.cuda.synchronize()
        assert rel_err(host(rhs), O.helmholtz_solve(b, g, 0.02, ibm.IBM_FIELD_CELL_DIRICHLET, lo, hi)) <= tol
        ibm.ibm_plan_check(plan)
    finally:
        ibm.ibm_plan_destroy(plan)


def test_wall_data_rejected_without_walls():
    g = grid(16, 16, 16)
    plan = ibm.ibm_plan_create(16, 16, 16, g[3:], ibm.IBM_FP64, 0, bc=ibm.IBM_BC_TRIPLY_PERIODIC)
    try:
        x = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_poisson_solve_bc(plan, x, x, x[0], x[0])
        assert e.value.code == ibm.IBM_ERR_UNSUPPORTED
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_helmholtz_solve_bc(plan, 0.1, ibm.IBM_FIELD_CELL_NEUMANN, x, x, x[0], x[0])
        assert e.value.code == ibm.IBM_ERR_UNSUPPORTED
    finally:
        ibm.ibm_plan_destroy(plan)


def test_invalid_arguments_rejected_before_launch():
    g = grid(32, 32, 32)
    with pytest.raises(ibm.IbmError) as e:
        ibm.ibm_plan_create(30, 32, 32, g[3:], ibm.IBM_FP32_REFINED, 1)
    assert e.value.code == ibm.IBM_ERR_ARG
    with pytest.raises(ibm.IbmError):
        ibm.ibm_plan_create(32, 4, 32, g[3:], ibm.IBM_FP32_REFINED, 1)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_plan_create(32, 32, 32, (1.0, -1.0, 1.0), ibm.IBM_FP64, 0)
    plan = _plan(32, 32, 32, g, ibm.IBM_FP64)
    try:
        x = torch.zeros(32 * 32 * 32 + 1, dtype=torch.float64, device="cuda")
        with pytest.raises(ibm.IbmError):
            ibm.ibm_poisson_solve(plan, x[1:].data_ptr() + 4, x.data_ptr())
        with pytest.raises(ibm.IbmError):
            ibm.ibm_helmholtz_solve(plan, -1.0, 0, x, x)
    finally:
        ibm.ibm_plan_destroy(plan)
