"""Continuous-batching server: results alone vs in the mix, admission, failures.

A mix of Poisson, Helmholtz and RK-stage requests of different grids and
precisions is submitted back to back to a multi-stream server; each result
must equal what the same request gives when served alone (one stream, no
other work) within the parity tolerance of its precision, and Poisson
results must match the oracle.  Failure paths are exercised on the host:
cancellation before admission, a request larger than the HBM budget, and
the IBM_FAULT_ADMIT hook that fails one admission.
"""

import ctypes
import math
import os

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, TOL_FP64, grid, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _request(kind, shape, prec, data, out, **kw):
    nx, ny, nz = shape
    g = grid(nx, ny, nz)
    r = ibm.ibm_request()
    r.kind, r.nx, r.ny, r.nz = kind, nx, ny, nz
    r.h = (ctypes.c_double * 3)(*g[3:])
    r.precision, r.refine_iters = prec, kw.get("refine", 1)
    r.c, r.field_bc = kw.get("c", 0.0), kw.get("field_bc", 0)
    r.in_ = data.ctypes.data
    r.out = out.ctypes.data
    r.n_markers = kw.get("n_markers", 0)
    r.X0 = kw["X0"].ctypes.data if "X0" in kw else None
    r.dV = kw["dV"].ctypes.data if "dV" in kw else None
    r.motion = kw.get("motion", 0)
    r.params = (ctypes.c_double * 4)(*(list(kw.get("params", ())) + [0.0] * 4)[:4])
    r.dt, r.nu, r.rk_stage = kw.get("dt", 1e-3), kw.get("nu", 1e-2), kw.get("rk_stage", 1)
    return r


def _mix():
    """(request kwargs, host input) list of mixed kinds, grids and precisions."""
    reqs = []
    rng = np.random.default_rng(7)
    shapes = [(32, 32, 32), (48, 40, 48), (64, 32, 64), (16, 16, 16), (96, 33, 64)]
    for i in range(14):
        shape = shapes[i % len(shapes)]
        prec = ibm.IBM_FP32_REFINED if i % 3 else ibm.IBM_FP64
        if i % 4 == 3:
            data = rng.standard_normal((shape[1], shape[2], shape[0]))
            reqs.append(dict(kind=ibm.IBM_REQ_HELMHOLTZ, shape=shape, prec=prec, data=data,
                             c=0.01, field_bc=ibm.IBM_FIELD_CELL_DIRICHLET))
        elif i % 7 == 5:
            g = grid(*shape)
            u, v, w = synth.div_free_velocity(g, workload=60 + i, kmax=4)
            data = np.stack([u, v, w, 0.05 * rng.standard_normal(u.shape)])
            X0, dV = synth.fibonacci_sphere(300, 0.25, (math.pi, 1.0, math.pi), g[3])
            reqs.append(dict(kind=ibm.IBM_REQ_SUBSTEP, shape=shape, prec=prec, data=data, n_markers=300,
                             X0=np.ascontiguousarray(X0), dV=np.ascontiguousarray(dV),
                             motion=ibm.IBM_MOTION_TRANSLATE, params=(0.1, 0.0, 0.0), rk_stage=1 + i % 3))
        else:
            data = synth.white_noise(*shape, workload=61, stream=i)
            reqs.append(dict(kind=ibm.IBM_REQ_POISSON, shape=shape, prec=prec, data=data))
    for q in reqs:
        q["data"] = np.ascontiguousarray(q["data"], dtype=np.float64)
    return reqs


def _serve(reqs, n_streams, budget=8 << 30):
    srv = ibm.ibm_server_create(budget, n_streams, 1024)
    outs, keep, tickets = [], [], []
    try:
        for q in reqs:
            out = np.zeros_like(q["data"])
            kw = {k: v for k, v in q.items() if k not in ("kind", "shape", "prec", "data")}
            r = _request(q["kind"], q["shape"], q["prec"], q["data"], out, **kw)
            keep.append((r, kw))
            outs.append(out)
            t = ibm.ibm_submit(srv, r)
            assert t is not None
            tickets.append(t)
        results = [ibm.ibm_wait(srv, t, 120.0) for t in tickets]
    finally:
        ibm.ibm_server_destroy(srv)
    return outs, results


def test_results_alone_equal_results_in_the_mix():
    reqs = _mix()
    mixed, res = _serve(reqs, n_streams=6)
    for rc, r in res:
        assert rc == ibm.IBM_OK, (rc, r.status)
        assert r.total_ms >= r.queue_ms >= 0.0 and r.device_ms > 0.0
    for i, q in enumerate(reqs):
        alone, res1 = _serve([q], n_streams=1)
        assert res1[0][0] == ibm.IBM_OK
        tol = TOL_FP64 if q["prec"] == ibm.IBM_FP64 else TOL_FP32
        assert rel_err(mixed[i], alone[0]) <= tol, (i, q["kind"], rel_err(mixed[i], alone[0]))
        if q["kind"] == ibm.IBM_REQ_POISSON:
            g = grid(*q["shape"])
            data = q["data"].astype(np.float32).astype(np.float64) if q["prec"] else q["data"]
            ref, _ = O.poisson_solve(data, g)
            assert rel_err(mixed[i], ref) <= tol


def test_substep_through_server_matches_oracle():
    shape = (32, 32, 32)
    g = grid(*shape)
    u, v, w = synth.div_free_velocity(g, workload=70, kmax=4)
    p = np.zeros_like(u)
    X0, dV = synth.fibonacci_sphere(400, 0.25, (math.pi, 1.0, math.pi), g[3])
    data = np.ascontiguousarray(np.stack([u, v, w, p]))
    q = dict(kind=ibm.IBM_REQ_SUBSTEP, shape=shape, prec=ibm.IBM_FP64, data=data, n_markers=400,
             X0=np.ascontiguousarray(X0), dV=np.ascontiguousarray(dV), motion=ibm.IBM_MOTION_TRANSLATE,
             params=(0.1, 0.0, 0.0), rk_stage=1)
    outs, res = _serve([q], n_streams=1)
    assert res[0][0] == ibm.IBM_OK
    z = np.zeros_like(u)
    st = dict(u=u, v=v, w=w, p=p, N_prev=(z, z, z), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=(0.1, 0.0, 0.0))
    ref, _ = O.rk_stage(st, mk, 1, 1e-3, 1e-2, g)
    for c, k in enumerate(("u", "v", "w", "p")):
        assert rel_err(outs[0][c], ref[k]) <= 1e-11


def test_cancel_budget_and_fault_hook():
    shape = (128, 128, 128)
    big = synth.white_noise(*shape, workload=62, stream=0)
    small = synth.white_noise(16, 16, 16, workload=62, stream=1)
    # one slot: the second request waits in the queue and can be cancelled
    srv = ibm.ibm_server_create(8 << 30, 1, 16)
    try:
        o1, o2, o3 = np.zeros_like(big), np.zeros_like(big), np.zeros_like(small)
        r1 = _request(ibm.IBM_REQ_POISSON, shape, ibm.IBM_FP64, big, o1)
        r2 = _request(ibm.IBM_REQ_POISSON, shape, ibm.IBM_FP64, big, o2)
        r3 = _request(ibm.IBM_REQ_POISSON, (16, 16, 16), ibm.IBM_FP32_REFINED, small, o3)
        t1, t2, t3 = ibm.ibm_submit(srv, r1), ibm.ibm_submit(srv, r2), ibm.ibm_submit(srv, r3)
        cancelled = ibm.ibm_cancel(srv, t3) == ibm.IBM_OK
        assert ibm.ibm_wait(srv, t1, 60.0)[0] == ibm.IBM_OK
        assert ibm.ibm_wait(srv, t2, 60.0)[0] == ibm.IBM_OK
        rc3 = ibm.ibm_wait(srv, t3, 60.0)[0]
        assert rc3 == (ibm.IBM_ERR_CANCELLED if cancelled else ibm.IBM_OK)
    finally:
        ibm.ibm_server_destroy(srv)
    # a request that cannot fit the budget even alone
    srv = ibm.ibm_server_create(1 << 20, 2, 16)
    try:
        o = np.zeros_like(big)
        t = ibm.ibm_submit(srv, _request(ibm.IBM_REQ_POISSON, shape, ibm.IBM_FP32_REFINED, big, o))
        assert ibm.ibm_wait(srv, t, 60.0)[0] == ibm.IBM_ERR_OOM
    finally:
        ibm.ibm_server_destroy(srv)
    # host-side fault hook: the second admission fails, the others succeed
    os.environ["IBM_FAULT_ADMIT"] = "1"
    try:
        srv = ibm.ibm_server_create(8 << 30, 2, 16)
    finally:
        del os.environ["IBM_FAULT_ADMIT"]
    try:
        outs = [np.zeros_like(small) for _ in range(3)]
        ts = [ibm.ibm_submit(srv, _request(ibm.IBM_REQ_POISSON, (16, 16, 16), ibm.IBM_FP32_REFINED, small, o))
              for o in outs]
        codes = [ibm.ibm_wait(srv, t, 60.0)[0] for t in ts]
        assert codes == [ibm.IBM_OK, ibm.IBM_ERR_OOM, ibm.IBM_OK]
    finally:
        ibm.ibm_server_destroy(srv)


def test_device_data_requests_equal_host_fp64_requests():
    """IBM_DATA_DEVICE: requests whose fields and markers are device arrays in
    the plan precision (no host staging, no FP64 conversion) give the results
    of the same requests served from FP64 host buffers, in a concurrent mix,
    and Poisson results match the oracle.  A stage's input stays untouched
    (it runs on a copy in the output)."""
    reqs = _mix()
    host_out, res = _serve(reqs, n_streams=4)
    assert all(rc == ibm.IBM_OK for rc, _ in res)
    srv = ibm.ibm_server_create(8 << 30, 6, 1024)
    keep, tickets, outs = [], [], []
    try:
        for q in reqs:
            dt = torch.float64 if q["prec"] == ibm.IBM_FP64 else torch.float32
            din = torch.from_numpy(q["data"]).to("cuda", dt)
            dout = torch.zeros_like(din)
            kw = {k: v for k, v in q.items() if k not in ("kind", "shape", "prec", "data")}
            dm = {}
            if "X0" in kw:
                dm = dict(X0=torch.from_numpy(kw.pop("X0")).to("cuda", dt), dV=torch.from_numpy(kw.pop("dV")).to("cuda", dt))
            r = _request(q["kind"], q["shape"], q["prec"], q["data"], q["data"], **kw)
            r.in_, r.out, r.data = din.data_ptr(), dout.data_ptr(), ibm.IBM_DATA_DEVICE
            if dm:
                r.X0, r.dV = dm["X0"].data_ptr(), dm["dV"].data_ptr()
            keep.append((r, din, dout, dm))
            t = ibm.ibm_submit(srv, r)
            assert t is not None
            tickets.append(t)
        for t in tickets:
            rc, res1 = ibm.ibm_wait(srv, t, 120.0)
            assert rc == ibm.IBM_OK and res1.device_ms > 0.0
        for (r, din, dout, dm), q, ho in zip(keep, reqs, host_out):
            tol = TOL_FP64 if q["prec"] == ibm.IBM_FP64 else TOL_FP32
            got = dout.double().cpu().numpy()
            assert rel_err(got, ho) <= tol, (q["kind"], rel_err(got, ho))
            assert np.array_equal(din.double().cpu().numpy(),
                                  q["data"].astype(np.float32 if q["prec"] else np.float64).astype(np.float64))
            if q["kind"] == ibm.IBM_REQ_POISSON:
                data = q["data"].astype(np.float32).astype(np.float64) if q["prec"] else q["data"]
                ref, _ = O.poisson_solve(data, grid(*q["shape"]))
                assert rel_err(got, ref) <= tol
    finally:
        ibm.ibm_server_destroy(srv)
    # rejected before admission: aliasing and misaligned device fields, an unknown data kind
    srv = ibm.ibm_server_create(1 << 30, 1, 4)
    try:
        x = torch.zeros(4096, device="cuda")
        r = _request(ibm.IBM_REQ_POISSON, (16, 16, 16), ibm.IBM_FP32_REFINED, np.zeros(1), np.zeros(1))
        r.data, r.in_, r.out = ibm.IBM_DATA_DEVICE, x.data_ptr(), x.data_ptr()
        with pytest.raises(ibm.IbmError):
            ibm.ibm_submit(srv, r)
        r.out = x.data_ptr() + 4
        with pytest.raises(ibm.IbmError):
            ibm.ibm_submit(srv, r)
        r.out, r.data = x.data_ptr() + 8192, 5
        with pytest.raises(ibm.IbmError):
            ibm.ibm_submit(srv, r)
    finally:
        ibm.ibm_server_destroy(srv)


def test_request_with_a_marker_past_the_wall_rule_fails():
    """A stage request whose sphere reaches within the delta support of a wall
    fails with IBM_ERR_ARG (the wall rule), and the server's next request of
    the same shape (the same resident plan) succeeds."""
    shape = (32, 32, 32)
    g = grid(*shape)
    u, v, w = synth.div_free_velocity(g, workload=71, kmax=4)
    data = np.ascontiguousarray(np.stack([u, v, w, np.zeros_like(u)]))
    X0, dV = synth.fibonacci_sphere(200, 0.25, (math.pi, 0.2, math.pi), g[3])  # reaches y = -0.05
    ok0, okdV = synth.fibonacci_sphere(200, 0.25, (math.pi, 1.0, math.pi), g[3])
    srv = ibm.ibm_server_create(2 << 30, 1, 16)
    try:
        outs = [np.zeros_like(data) for _ in range(2)]
        bad = _request(ibm.IBM_REQ_SUBSTEP, shape, ibm.IBM_FP32_REFINED, data, outs[0], n_markers=200,
                       X0=np.ascontiguousarray(X0), dV=np.ascontiguousarray(dV), motion=ibm.IBM_MOTION_STATIC)
        good = _request(ibm.IBM_REQ_SUBSTEP, shape, ibm.IBM_FP32_REFINED, data, outs[1], n_markers=200,
                        X0=np.ascontiguousarray(ok0), dV=np.ascontiguousarray(okdV), motion=ibm.IBM_MOTION_STATIC)
        t1 = ibm.ibm_submit(srv, bad)
        assert ibm.ibm_wait(srv, t1, 60.0)[0] == ibm.IBM_ERR_ARG
        t2 = ibm.ibm_submit(srv, good)
        assert ibm.ibm_wait(srv, t2, 60.0)[0] == ibm.IBM_OK
    finally:
        ibm.ibm_server_destroy(srv)
