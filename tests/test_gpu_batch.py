"""Batched solves of many independent grids in one CUDA-graph launch.

Every instance of a mixed-size batch is compared with the FP64 oracle (and
so with what it would give alone), across a change of field pointers (a
new graph) and a repeat of the first pointer set (graph replay), including
an in-place instance.
"""

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, TOL_FP64, dev, grid, host, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DIMS = [(32, 32, 32), (48, 40, 48), (16, 16, 16), (64, 24, 64), (32, 32, 32), (48, 40, 48), (12, 10, 24),
        (96, 33, 64)]


@pytest.mark.parametrize("prec", [ibm.IBM_FP32_REFINED, ibm.IBM_FP64])
def test_batch_matches_oracle_and_replays(prec):
    dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
    npdt = np.float32 if prec == ibm.IBM_FP32_REFINED else np.float64
    tol = TOL_FP32 if prec == ibm.IBM_FP32_REFINED else TOL_FP64
    grids = [grid(*d) for d in DIMS]
    batch = ibm.ibm_batch_create(DIMS, [g[3:] for g in grids], prec, 1)
    try:
        sets = []
        for rep in range(2):
            rhs, phi, ref = [], [], []
            for i, (d, g) in enumerate(zip(DIMS, grids)):
                b = synth.white_noise(*d, workload=50 + rep, stream=i).astype(npdt).astype(np.float64)
                ref.append(O.poisson_solve(b, g)[0])
                r = dev(b, dt)
                rhs.append(r)
                phi.append(r if i == 3 else torch.empty_like(r))  # instance 3 in place
            sets.append((rhs, phi, ref))
        for rhs, phi, ref in sets + sets[:1]:
            ibm.ibm_batch_poisson(batch, rhs, phi)
            torch.cuda.synchronize()
            for i in range(len(DIMS)):
                err = rel_err(host(phi[i]), ref[i])
                assert err <= tol, (i, DIMS[i], err)
            # refill the in-place instance for the replay
            rhs[3].copy_(dev(O.laplacian(ref[3], grids[3], O.NEUMANN), dt))
    finally:
        ibm.ibm_batch_destroy(batch)


def test_batch_rejects_bad_arguments():
    g = grid(32, 32, 32)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_batch_create([(30, 32, 32)], [g[3:]], ibm.IBM_FP32_REFINED, 1)


def _stage_instance(d, i, prec, n_markers):
    """Device state and still marker sphere of one batched-stage instance."""
    import math
    g = grid(*d)
    dt = torch.float32 if prec == ibm.IBM_FP32_REFINED else torch.float64
    u, v, w = synth.div_free_velocity(g, workload=80 + i, kmax=min(d) / 4)
    r = np.random.default_rng(80 + i)
    p = 0.1 * r.standard_normal(u.shape)
    X0, dV = synth.fibonacci_sphere(n_markers, 0.25, (math.pi, 1.0, math.pi), g[3])
    f = [dev(a, dt) for a in (u, v, w, p)] + [torch.zeros(u.shape, dtype=dt, device="cuda") for _ in range(3)]
    st = ibm.ibm_state(*[t.data_ptr() for t in f], 0.0)
    Xd, dVd = dev(X0, dt), dev(dV, dt)
    X, Ud, F = (torch.empty((n_markers, 3), dtype=dt, device="cuda") for _ in range(3))
    mk = ibm.ibm_markers(n_markers, Xd.data_ptr(), dVd.data_ptr(), X.data_ptr(), Ud.data_ptr(), F.data_ptr(),
                         ibm.IBM_MOTION_STATIC, (ctypes_double4)(0.0, 0.0, 0.0, 0.0))
    return g, st, mk, (f, Xd, dVd, X, Ud, F), (u, v, w, p, X0, dV)


import ctypes  # noqa: E402
ctypes_double4 = ctypes.c_double * 4


@pytest.mark.parametrize("prec", [ibm.IBM_FP32_REFINED, ibm.IBM_FP64])
def test_batched_stage_with_markers_equals_instances_alone(prec):
    """ibm_batch_substep: one RK stage of mixed-size instances, each with its
    own still marker sphere (500-2000 markers), as one graph launch; every
    instance's fields equal those of the same stage run alone through
    ibm_substep, over three stages (the second call of a stage replays its
    graph), and the first stage of two instances matches the oracle."""
    dims = [(32, 32, 32), (48, 40, 48), (64, 24, 64), (32, 32, 32), (16, 16, 16), (48, 40, 48)]
    counts = [500, 1200, 2000, 800, 600, 1500]
    grids = [grid(*d) for d in dims]
    batch = ibm.ibm_batch_create(dims, [g[3:] for g in grids], prec, 1)
    # the batch's plans take the kernels its tuner picked, the lone plans the
    # default ones, so FP32 fields differ by rounding that accumulates over
    # the stages: the FP32 stage tolerance (the pressure, defined up to a
    # constant and concentrated at the sphere, carries most of it)
    tol = 3e-6 if prec == ibm.IBM_FP32_REFINED else 1e-11
    try:
        inst = [_stage_instance(d, i, prec, m) for i, (d, m) in enumerate(zip(dims, counts))]
        alone = [_stage_instance(d, i, prec, m) for i, (d, m) in enumerate(zip(dims, counts))]
        plans = [ibm.ibm_plan_create(*d, g[3:], prec, 1) for d, g in zip(dims, grids)]
        try:
            for stage in (1, 2, 3, 1):
                ibm.ibm_batch_substep(batch, [x[1] for x in inst], [x[2] for x in inst], stage, 1e-3, 1e-2)
                for pl, a in zip(plans, alone):
                    ibm.ibm_substep(pl, a[1], stage, 1e-3, 1e-2, a[2])
                torch.cuda.synchronize()
                for i, (x, a) in enumerate(zip(inst, alone)):
                    for c in range(4):
                        e = rel_err(host(x[3][0][c]), host(a[3][0][c]))
                        assert e <= tol, (stage, i, c, e)
                    assert x[1].t == pytest.approx(a[1].t, rel=0, abs=1e-15)
        finally:
            for pl in plans:
                ibm.ibm_plan_destroy(pl)
        # the oracle: a fresh first stage of instances 0 and 2
        for i in (0, 2):
            g, st, mk, keep, (u, v, w, p, X0, dV) = _stage_instance(dims[i], i, prec, counts[i])
            solo = ibm.ibm_batch_create([dims[i]], [grids[i][3:]], prec, 1)
            try:
                ibm.ibm_batch_substep(solo, [st], [mk], 1, 1e-3, 1e-2)
                torch.cuda.synchronize()
            finally:
                ibm.ibm_batch_destroy(solo)
            cast = (lambda a: a.astype(np.float32).astype(np.float64)) if prec == ibm.IBM_FP32_REFINED else (lambda a: a)
            z = np.zeros_like(u)
            ref, _ = O.rk_stage(dict(u=cast(u), v=cast(v), w=cast(w), p=cast(p), N_prev=(z, z, z), t=0.0),
                                dict(X0=cast(X0), dV=cast(dV), kind=O.MOTION_STATIC, params=()), 1, 1e-3, 1e-2, g)
            stol = 3e-6 if prec == ibm.IBM_FP32_REFINED else 1e-11
            for c, k in enumerate("uvwp"):
                assert rel_err(host(keep[0][c]), ref[k]) <= stol, (i, k)
    finally:
        ibm.ibm_batch_destroy(batch)
