"""GPU parity of one RK stage (ibm_substep, Eq. 2a-2h) against the oracle.

Inputs: a discretely divergence-free random velocity (energy ~ k^-5/3),
random pressure and previous-stage advection, and a sphere of markers with
prescribed motion.  The stage is compared field by field (u, v, w, p, the
stored advection term, the Lagrangian force) with the oracle's rk_stage.

FP32 tolerance (3e-6 relative L2 per field): the stage chains FP32 stencils
(~10 eps32 each), FP32 interpolation/spreading (~2e-6, see gpu_util) whose
force enters u* scaled by dt, three well-conditioned Helmholtz solves
(~1e-7) and a refined Poisson solve (<= 1e-6 on phi, entering u through
(a+b) dt G phi); markers sit at their reference positions (t = 0) so both
sides see identical coordinates.
"""

import math
import os

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import dev, grid, host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_STAGE_FP64 = 1e-11
TOL_STAGE_FP32 = 3e-6
# The stored advection term N = div(u u) in FP32: each flux is a product of
# two-point averages rounded to FP32 (relative error a few eps32 of |u|^2)
# and N is a difference of fluxes over h, of size |u|^2 k; its relative
# error is therefore ~ eps32 / (k h) per point (about 1e-6 for the k <= 16
# content of the 384-cell grids), and the max over 25M points runs several
# times higher (measured: 2.1e-6 L2, 6.3e-6 max at 384x256x256).
TOL_STAGE_FP32_N = 1e-5


def stage_ok(errs, tol, tol_n):
    """Every field within tol, the stored advection terms (N0..N2) within tol_n."""
    return all(v <= (tol_n if k.startswith("N") else tol) for k, v in errs.items())


def _setup(nx, ny, nz, nmk, npdt, wl):
    g = grid(nx, ny, nz)
    u, v, w = synth.div_free_velocity(g, workload=wl, kmax=min(nx, ny, nz) / 4)
    r = np.random.default_rng(wl)
    p = 0.1 * r.standard_normal((ny, nz, nx))
    Np = [0.5 * r.standard_normal((ny, nz, nx)) for _ in range(3)]
    Np[1][0] = 0.0
    X0, dV = synth.fibonacci_sphere(nmk, 0.25, (math.pi + 0.01, 1.0 - 0.013, math.pi + 0.02), g[3])
    cast = lambda a: np.asarray(a).astype(npdt).astype(np.float64)
    return g, [cast(a) for a in (u, v, w, p)], [cast(a) for a in Np], cast(X0), cast(dV)


def _run_gpu(g, fields, Np, X0, dV, stage, dt, nu, motion, params, prec, dt_t, t0, spread=None):
    nx, ny, nz = g[:3]
    n = len(X0)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        if spread is not None:
            ibm.ibm_plan_set_spread(plan, spread)
        d = [dev(a, dt_t) for a in fields]
        dN = [dev(a, dt_t) for a in Np]
        st = ibm.ibm_state(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
                           dN[0].data_ptr(), dN[1].data_ptr(), dN[2].data_ptr(), t0)
        X0d, dVd = dev(X0, dt_t), dev(dV, dt_t)
        X = torch.empty((n, 3), dtype=dt_t, device="cuda")
        Ud = torch.empty_like(X)
        F = torch.empty_like(X)
        mk = ibm.ibm_markers(n, X0d.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(), motion,
                             (ctypes_d4(params)))
        info = ibm.ibm_substep(plan, st, stage, dt, nu, mk, info=True)
        out = dict(u=host(d[0]), v=host(d[1]), w=host(d[2]), p=host(d[3]), N=[host(a) for a in dN],
                   F=host(F), X=host(X), Ud=host(Ud), t=st.t, info=info)
        return out
    finally:
        ibm.ibm_plan_destroy(plan)


def _run_gpu_inout(g, fields, Np, X0, dV, io, stages, dt, nu, params, prec, dt_t):
    """Stages `stages` (a sequence of 1..3) of ibm_substep_inout in a row;
    the outlet planes carry over from stage to stage on the device."""
    nx, ny, nz = g[:3]
    n = len(X0)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        d = [dev(a, dt_t) for a in fields]
        dN = [dev(a, dt_t) for a in Np]
        st = ibm.ibm_state(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), d[3].data_ptr(),
                           dN[0].data_ptr(), dN[1].data_ptr(), dN[2].data_ptr(), 0.0)
        planes = [dev(io[k], dt_t) for k in ("u_out", "v_out", "w_out")]
        dio = ibm.ibm_inout(io["v_in"], io["c_out"], *[t.data_ptr() for t in planes])
        X0d, dVd = dev(X0, dt_t), dev(dV, dt_t)
        X = torch.empty((n, 3), dtype=dt_t, device="cuda")
        Ud = torch.empty_like(X)
        F = torch.empty_like(X)
        mk = ibm.ibm_markers(n, X0d.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                             ibm.IBM_MOTION_TRANSLATE, ctypes_d4(params))
        info = None
        for s in stages:
            info = ibm.ibm_substep_inout(plan, st, dio, s, dt, nu, mk, info=True)
        return dict(u=host(d[0]), v=host(d[1]), w=host(d[2]), p=host(d[3]), N=[host(a) for a in dN],
                    F=host(F), u_out=host(planes[0]), v_out=host(planes[1]), w_out=host(planes[2]), t=st.t,
                    info=info)
    finally:
        ibm.ibm_plan_destroy(plan)


def _inout_data(nx, nz, npdt, seed):
    r = np.random.default_rng(seed)
    cast = lambda a: np.asarray(a).astype(npdt).astype(np.float64)
    return dict(v_in=0.5, c_out=0.6, u_out=cast(0.1 * r.standard_normal((nz, nx))),
                v_out=cast(0.5 + 0.1 * r.standard_normal((nz, nx))), w_out=cast(0.1 * r.standard_normal((nz, nx))))


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 24, 24)])
@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_inout_substep_matches_oracle(shape, stage, prec):
    """Inflow-outflow walls (Sec. 3): one stage, every field and the
    advanced outlet planes against the oracle."""
    nx, ny, nz = shape
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    dt_t = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    tol = TOL_STAGE_FP64 if prec == ibm.IBM_FP64 else TOL_STAGE_FP32
    g, (u, v, w, p), Np, X0, dV = _setup(nx, ny, nz, 800, npdt, wl=50 + stage)
    io = _inout_data(nx, nz, npdt, 60 + stage)
    dt, nu = 1e-3, 1e-2
    params = (0.1, 0.0, 0.0)
    st = dict(u=u, v=v, w=w, p=p, N_prev=tuple(Np), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=params)
    ref, rinfo = O.rk_stage(st, mk, stage, dt, nu, g, inout=io)
    got = _run_gpu_inout(g, [u, v, w, p], Np, X0, dV, io, [stage], dt, nu, params, prec, dt_t)
    errs = {k: rel_err(got[k], ref[k]) for k in ("u", "v", "w", "p")}
    errs.update({"N%d" % c: rel_err(got["N"][c], ref["N_prev"][c]) for c in range(3)})
    errs.update({k: rel_err(got[k], ref["inout"][k]) for k in ("u_out", "v_out", "w_out")})
    errs["F"] = rel_err(got["F"], rinfo["F"])
    assert stage_ok(errs, tol, tol if prec == ibm.IBM_FP64 else TOL_STAGE_FP32_N), errs
    print("stage errors", errs)
    assert np.all(got["v"][0] == npdt(io["v_in"]))
    # outflow = inflow to rounding of the stored outlet plane
    assert abs(got["v_out"].mean() - io["v_in"]) <= (1e-14 if prec == ibm.IBM_FP64 else 1e-6)
    vo = ref["inout"]["v_out"]
    d0 = np.abs(O.divergence(*rinfo["ustar"], g, io["v_in"], vo)).max()
    lim = 1e-11 if prec == ibm.IBM_FP64 else 1e-5
    assert got["info"]["div_max"] <= lim * max(1.0, d0), (got["info"], d0)
    assert abs(got["info"]["div_before"] - d0) <= 1e-3 * d0


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_inout_full_rk_step_matches_oracle(prec):
    """Three stages in a row (one time step): the outlet planes and N^{n-2}
    carry over on the device exactly as in the oracle."""
    nx, ny, nz = 48, 24, 32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    dt_t = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    g, (u, v, w, p), Np, X0, dV = _setup(nx, ny, nz, 500, npdt, wl=71)
    io = _inout_data(nx, nz, npdt, 72)
    dt, nu = 2e-3, 1e-2
    params = (0.1, 0.0, 0.0)
    st = dict(u=u, v=v, w=w, p=p, N_prev=tuple(Np), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=params)
    ref_io = io
    for s in (1, 2, 3):
        st, _ = O.rk_stage(st, mk, s, dt, nu, g, inout=ref_io)
        ref_io = st["inout"]
    got = _run_gpu_inout(g, [u, v, w, p], Np, X0, dV, io, (1, 2, 3), dt, nu, params, prec, dt_t)
    tol = 3 * (TOL_STAGE_FP64 if prec == ibm.IBM_FP64 else TOL_STAGE_FP32)
    errs = {k: rel_err(got[k], st[k]) for k in ("u", "v", "w", "p")}
    errs.update({k: rel_err(got[k], ref_io[k]) for k in ("u_out", "v_out", "w_out")})
    assert stage_ok(errs, tol, tol if prec == ibm.IBM_FP64 else TOL_STAGE_FP32_N), errs
    print("stage errors", errs)
    assert abs(got["t"] - dt) < 1e-15


def test_inout_arguments_rejected():
    g = grid(16, 16, 16)
    plan = ibm.ibm_plan_create(16, 16, 16, g[3:], ibm.IBM_FP64, 1)
    try:
        f = [torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda") for _ in range(7)]
        st = ibm.ibm_state(*[t.data_ptr() for t in f], 0.0)
        pl = [torch.zeros((16, 16), dtype=torch.float64, device="cuda") for _ in range(3)]
        mk = ibm.ibm_markers(0, None, None, None, None, None, ibm.IBM_MOTION_STATIC, ctypes_d4(()))
        bad = [ibm.ibm_inout(0.5, -1.0, *[t.data_ptr() for t in pl]),
               ibm.ibm_inout(float("nan"), 0.5, *[t.data_ptr() for t in pl]),
               ibm.ibm_inout(0.5, 0.5, pl[0].data_ptr(), None, pl[2].data_ptr())]
        for io in bad:
            with pytest.raises(ibm.IbmError):
                ibm.ibm_substep_inout(plan, st, io, 1, 1e-3, 1e-2, mk)
    finally:
        ibm.ibm_plan_destroy(plan)


def ctypes_d4(params):
    import ctypes
    vals = list(params) + [0.0] * (4 - len(params))
    return (ctypes.c_double * 4)(*vals)


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 24, 24)])
@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_substep_matches_oracle(shape, stage, prec):
    nx, ny, nz = shape
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    dt_t = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    tol = TOL_STAGE_FP64 if prec == ibm.IBM_FP64 else TOL_STAGE_FP32
    g, (u, v, w, p), Np, X0, dV = _setup(nx, ny, nz, 800, npdt, wl=30 + stage)
    dt, nu = 1e-3, 1e-2
    motion, params = ibm.IBM_MOTION_TRANSLATE, (0.1, 0.0, 0.0)
    st = dict(u=u, v=v, w=w, p=p, N_prev=tuple(Np), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=params)
    ref, rinfo = O.rk_stage(st, mk, stage, dt, nu, g)
    got = _run_gpu(g, [u, v, w, p], Np, X0, dV, stage, dt, nu, motion, params, prec, dt_t, 0.0)
    errs = {k: rel_err(got[k], ref[k]) for k in ("u", "v", "w", "p")}
    errs.update({"N%d" % c: rel_err(got["N"][c], ref["N_prev"][c]) for c in range(3)})
    errs["F"] = rel_err(got["F"], rinfo["F"])
    assert stage_ok(errs, tol, tol if prec == ibm.IBM_FP64 else TOL_STAGE_FP32_N), errs
    print("stage errors", errs)
    a, b = O.RK_ALPHA[stage - 1], O.RK_BETA[stage - 1]
    assert abs(got["t"] - (a + b) * dt) < 1e-15
    assert np.all(got["v"][0] == 0.0)
    # projection: D u^n vanishes to round-off of the stored fields
    d0 = np.abs(O.divergence(*rinfo["ustar"], g)).max()
    lim = 1e-11 if prec == ibm.IBM_FP64 else 1e-5
    assert got["info"]["div_max"] <= lim * max(1.0, d0), (got["info"], d0)
    assert abs(got["info"]["div_before"] - d0) <= 1e-3 * d0


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_three_field_helmholtz_every_kernel(prec):
    """The three Helmholtz solves of a stage share launches; every plane mode
    of those launches (split, one CTA per plane, 2-CTA cluster, tensor-core
    DFT products) and every
    pencil kernel gives the oracle's stage."""
    nx, ny, nz = 64, 24, 64
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    dt_t = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    tol = TOL_STAGE_FP64 if prec == ibm.IBM_FP64 else TOL_STAGE_FP32
    g, (u, v, w, p), Np, X0, dV = _setup(nx, ny, nz, 300, npdt, wl=37)
    dt, nu = 1e-3, 1e-2
    params = (0.1, 0.0, 0.0)
    st = dict(u=u, v=v, w=w, p=p, N_prev=tuple(Np), t=0.0)
    ref, _ = O.rk_stage(st, dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=params), 2, dt, nu, g)
    for plane_mode, pencil_mode in ((0, 2), (0, 3), (1, 2), (2, 3), (0, 1), (1, 4), (-1, 4)):
        if plane_mode == -1 and prec == ibm.IBM_FP64:
            continue  # the tensor-core DFT mode (-1) exists for FP32 plans only
        os.environ["IBM_PLANE_MODE_FIELDS"] = str(plane_mode)
        os.environ["IBM_PENCIL_MODE"] = str(pencil_mode)
        try:
            got = _run_gpu(g, [u, v, w, p], Np, X0, dV, 2, dt, nu, ibm.IBM_MOTION_TRANSLATE, params, prec, dt_t, 0.0)
        finally:
            del os.environ["IBM_PLANE_MODE_FIELDS"]
            del os.environ["IBM_PENCIL_MODE"]
        errs = {k: rel_err(got[k], ref[k]) for k in ("u", "v", "w", "p")}
        assert stage_ok(errs, tol, tol if prec == ibm.IBM_FP64 else TOL_STAGE_FP32_N), (plane_mode, pencil_mode, errs)
        assert np.all(got["v"][0] == 0.0)


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_marker_motion_heave(prec):
    """L2: heaving plate positions and surface velocity at a stage time."""
    g = grid(32, 32, 32)
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    dt_t = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    X0, dV = synth.flat_plate(10, 20, 1.0, 2.0, (math.pi, 1.0, math.pi), g[3])
    X0 = X0.astype(npdt).astype(np.float64)
    z = np.zeros((32, 32, 32))
    fields = [z.copy() for _ in range(4)]
    Np = [z.copy() for _ in range(3)]
    t0 = 0.37
    params = (0.05, 1.0)
    got = _run_gpu(g, fields, Np, X0, dV.astype(npdt), 1, 1e-3, 1e-2, ibm.IBM_MOTION_HEAVE, params, prec, dt_t, t0)
    Xr, Udr = O.marker_motion(X0, t0, O.MOTION_HEAVE, params)
    tol = 1e-14 if prec == ibm.IBM_FP64 else 1e-7
    assert rel_err(got["X"], Xr) <= tol
    assert rel_err(got["Ud"], Udr) <= tol


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_substep_with_gather_spreading(prec):
    """The RK stage with the deterministic Eulerian-gather spreading gives the
    oracle's stage, and the same bytes on a second run."""
    nx, ny, nz = 32, 32, 32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    dt_t = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    tol = TOL_STAGE_FP64 if prec == ibm.IBM_FP64 else TOL_STAGE_FP32
    g, (u, v, w, p), Np, X0, dV = _setup(nx, ny, nz, 800, npdt, wl=41)
    dt, nu = 1e-3, 1e-2
    params = (0.1, 0.0, 0.0)
    st = dict(u=u, v=v, w=w, p=p, N_prev=tuple(Np), t=0.0)
    ref, _ = O.rk_stage(st, dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=params), 2, dt, nu, g)
    runs = [_run_gpu(g, [u, v, w, p], Np, X0, dV, 2, dt, nu, ibm.IBM_MOTION_TRANSLATE, params, prec, dt_t, 0.0,
                     spread=ibm.IBM_SPREAD_GATHER) for _ in range(2)]
    errs = {k: rel_err(runs[0][k], ref[k]) for k in ("u", "v", "w", "p")}
    assert stage_ok(errs, tol, tol if prec == ibm.IBM_FP64 else TOL_STAGE_FP32_N), errs
    print("stage errors", errs)
    for k in ("u", "v", "w", "p"):
        assert np.array_equal(runs[0][k], runs[1][k]), k
