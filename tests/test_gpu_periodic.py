"""GPU parity of the triply periodic branch (Sec. 2.3.3, S2) against the oracle.

Plans with bc = IBM_BC_TRIPLY_PERIODIC solve every (kx, kz) pencil by a
Fourier transform along y, a diagonal divide and the inverse transform.
Poisson (mean(phi) = 0, removed mean reported) and Helmholtz (field kind
IBM_FIELD_PERIODIC) are compared element by element with the oracle's
periodic eigen-solves, in FP64 (1e-12) and FP32 with refinement (1e-6), on
shapes that cover radix-3 lengths along every axis, the smallest grid,
one-CTA plane and split x/z transforms, and ragged pencil tiles.
"""

import ctypes
import math

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, TOL_FP64, dev, grid, host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(32, 32, 32), (8, 8, 8), (12, 24, 16), (48, 96, 64), (64, 12, 48), (256, 16, 128), (16, 384, 8)]


def _plan(shape, prec, refine=1):
    g = grid(*shape, Ly=3.0)
    return g, ibm.ibm_plan_create(*shape, g[3:], prec, refine, bc=ibm.IBM_BC_TRIPLY_PERIODIC)


@pytest.mark.parametrize("shape", SHAPES)
def test_periodic_poisson_matches_oracle(shape):
    nx, ny, nz = shape
    b = synth.white_noise(nx, ny, nz, workload=80, stream=0) + 0.4
    for prec, dt, tol in ((ibm.IBM_FP64, torch.float64, TOL_FP64), (ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32)):
        bb = b.astype(np.float32).astype(np.float64) if dt == torch.float32 else b
        g, plan = _plan(shape, prec)
        try:
            ref, mean_b = O.poisson_solve(bb, g, ybc=O.PERIODIC)
            rhs = dev(bb, dt)
            phi = torch.empty_like(rhs)
            info = ibm.ibm_poisson_solve(plan, rhs, phi, info=True)
            err = rel_err(host(phi), ref)
            assert err <= tol, (prec, err)
            assert abs(info["removed_mean"] - mean_b) <= (1e-12 if prec == ibm.IBM_FP64 else 1e-6) * max(1.0, abs(mean_b))
            # FP32 storage of phi alone limits the residual to ~eps32 cond
            assert info["rel_residual"] < (1e-12 if prec == ibm.IBM_FP64 else 1e-2)
            ph = host(phi)
            assert abs(ph.mean()) <= (1e-13 if prec == ibm.IBM_FP64 else 1e-6) * np.abs(ph).max()
        finally:
            ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("c", [5e-6, 0.05])
def test_periodic_helmholtz_matches_oracle(shape, c):
    nx, ny, nz = shape
    r = synth.white_noise(nx, ny, nz, workload=81, stream=1)
    for prec, dt, tol in ((ibm.IBM_FP64, torch.float64, TOL_FP64), (ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32)):
        rr = r.astype(np.float32).astype(np.float64) if dt == torch.float32 else r
        g, plan = _plan(shape, prec)
        try:
            ref = O.helmholtz_solve(rr, g, c, O.PERIODIC)
            rhs = dev(rr, dt)
            u = torch.empty_like(rhs)
            ibm.ibm_helmholtz_solve(plan, c, ibm.IBM_FIELD_PERIODIC, rhs, u)
            torch.cuda.synchronize()
            assert rel_err(host(u), ref) <= tol, (prec, rel_err(host(u), ref))
        finally:
            ibm.ibm_plan_destroy(plan)


def test_periodic_manufactured_mode_in_place():
    """A Fourier mode along every axis comes back exactly (rhs == phi)."""
    shape = (48, 32, 24)
    g, plan = _plan(shape, ibm.IBM_FP64)
    nx, ny, nz, hx, hy, hz = g
    try:
        i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
        phi = (np.cos(2 * math.pi * 5 * j / ny)[:, None, None] * np.sin(2 * math.pi * 3 * k / nz)[None, :, None]
               * np.cos(2 * math.pi * 7 * i / nx)[None, None, :])
        lam = (O.modified_wavenumber_sq(2 * math.pi * 7 / nx, hx) + O.modified_wavenumber_sq(2 * math.pi * 5 / ny, hy)
               + O.modified_wavenumber_sq(2 * math.pi * 3 / nz, hz))
        x = dev(-lam * phi, torch.float64)
        ibm.ibm_poisson_solve(plan, x, x)
        assert rel_err(host(x), phi) < 1e-13
    finally:
        ibm.ibm_plan_destroy(plan)


def test_periodic_plan_rejections():
    g = grid(32, 32, 32)
    with pytest.raises(ibm.IbmError) as e:
        ibm.ibm_plan_create(32, 40, 32, g[3:], ibm.IBM_FP64, 0, bc=ibm.IBM_BC_TRIPLY_PERIODIC)  # ny not 2^a 3^b
    assert e.value.code == ibm.IBM_ERR_ARG
    plan = ibm.ibm_plan_create(32, 32, 32, g[3:], ibm.IBM_FP64, 0, bc=ibm.IBM_BC_TRIPLY_PERIODIC)
    try:
        x = torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda")
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_helmholtz_solve(plan, 0.1, ibm.IBM_FIELD_CELL_DIRICHLET, x, x)
        assert e.value.code == ibm.IBM_ERR_ARG
        X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
        U = torch.zeros_like(X)
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_interp(plan, 4, X, x, x, x, U)
        assert e.value.code == ibm.IBM_ERR_UNSUPPORTED
        st = ibm.ibm_state(*([x.data_ptr()] * 7), 0.0)
        mk = ibm.ibm_markers(0, None, None, None, None, None, 0, (ctypes.c_double * 4)())
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_substep(plan, st, 1, 1e-3, 1e-2, mk)
        assert e.value.code == ibm.IBM_ERR_UNSUPPORTED
    finally:
        ibm.ibm_plan_destroy(plan)
    wall = ibm.ibm_plan_create(32, 32, 32, g[3:], ibm.IBM_FP64, 0)
    try:
        x = torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda")
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_helmholtz_solve(wall, 0.1, ibm.IBM_FIELD_PERIODIC, x, x)
        assert e.value.code == ibm.IBM_ERR_ARG
    finally:
        ibm.ibm_plan_destroy(wall)
