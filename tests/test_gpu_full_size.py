"""Parity at the benchmark's full sizes, in the launch configurations the
bench times.

* 128^3 RK stage (the bench's headline workload): FP32 with one refinement
  step, the 20,000-marker Fibonacci sphere translating at 0.1 and the seeded
  divergence-free k^-5/3 velocity; one stage against the oracle's rk_stage,
  element by element (every field, the stored advection and the marker
  force).
* 256^3 Poisson (the solve the roofline target is quoted on): FP32 with one
  refinement step and FP64, the bench's low-passed noise right-hand side,
  against the oracle's eigen-solve element by element.
* 384 x 256 x 256 heaving-plate stage (100,000 markers, pre-aggregated
  spreading): properties that hold at any size (the projected field is
  divergence-free to the FP32 rounding of the stored fields; v stays zero
  on the wall) and, when the host has the memory for the FP64 oracle at
  this size, the oracle's stage element by element.
"""

import math

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import TOL_FP32, TOL_FP64, dev, host, rel_err
from tests.test_gpu_substep import TOL_STAGE_FP32, TOL_STAGE_FP32_N, _run_gpu, stage_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DT, NU = 1e-3, 1e-2


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def _f32(a):
    return np.asarray(a).astype(np.float32).astype(np.float64)


def _stage_errors(got, ref, rinfo):
    errs = {k: rel_err(got[k], ref[k]) for k in ("u", "v", "w", "p")}
    errs.update({"N%d" % c: rel_err(got["N"][c], ref["N_prev"][c]) for c in range(3)})
    errs["F"] = rel_err(got["F"], rinfo["F"])
    return errs


def test_stage_128_full_size():
    g = synth.grid(128, 128, 128)
    u, v, w = synth.div_free_velocity(g, workload=1, kmax=16.0)
    X0, dV = synth.fibonacci_sphere(20000, 0.25, (math.pi, 1.0, math.pi), g[3])
    z = np.zeros_like(u)
    fields = [_f32(a) for a in (u, v, w, z)]
    Np = [z, z, z]
    X0, dV = _f32(X0), _f32(dV)
    st = dict(u=fields[0], v=fields[1], w=fields[2], p=fields[3], N_prev=tuple(Np), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=(0.1, 0.0, 0.0))
    ref, rinfo = O.rk_stage(st, mk, 1, DT, NU, g)
    got = _run_gpu(g, fields, Np, X0, dV, 1, DT, NU, ibm.IBM_MOTION_TRANSLATE, (0.1, 0.0, 0.0),
                   ibm.IBM_FP32_REFINED, torch.float32, 0.0)
    errs = _stage_errors(got, ref, rinfo)
    assert stage_ok(errs, TOL_STAGE_FP32, TOL_STAGE_FP32_N), errs
    print("stage errors", errs)
    assert got["info"]["div_max"] <= 1e-5 * max(1.0, got["info"]["div_before"]), got["info"]


def test_poisson_256_full_size():
    n = 256
    g = synth.grid(n, n, n)
    b = synth.rhs_lowpass_noise(n, n, n, kmax=32.0, workload=1)
    for prec, dt, tol, bb in ((ibm.IBM_FP32_REFINED, torch.float32, TOL_FP32, _f32(b)),
                              (ibm.IBM_FP64, torch.float64, TOL_FP64, b)):
        ref, _ = O.poisson_solve(bb, g)
        plan = ibm.ibm_plan_create(n, n, n, g[3:], prec, 1 if prec == ibm.IBM_FP32_REFINED else 0)
        try:
            rhs = dev(bb, dt)
            phi = torch.empty_like(rhs)
            ibm.ibm_poisson_solve(plan, rhs, phi)
            torch.cuda.synchronize()
            err = rel_err(host(phi), ref)
            assert err <= tol, (prec, err)
            ibm.ibm_plan_check(plan)
        finally:
            ibm.ibm_plan_destroy(plan)


def test_plate_stage_full_size():
    nx, ny, nz = 384, 256, 256
    h = 2 * math.pi / 384
    g = (nx, ny, nz, h, h, h)
    u, v, w = synth.div_free_velocity(g, workload=2, kmax=16.0, rms=0.1)
    X0, dV = synth.flat_plate(250, 400, 1.0, 2.0, (nx * h / 2, ny * h / 2, nz * h / 2), h)
    z = np.zeros_like(u)
    fields = [_f32(a) for a in (u, v, w, z)]
    Np = [z, z, z]
    X0, dV = _f32(X0), _f32(dV)
    got = _run_gpu(g, fields, Np, X0, dV, 1, DT, NU, ibm.IBM_MOTION_HEAVE, (0.5, 1.0), ibm.IBM_FP32_REFINED,
                   torch.float32, 0.0)
    info = got["info"]
    assert info["div_max"] <= 1e-5 * max(1.0, info["div_before"]), info
    assert np.all(got["v"][0] == 0.0)
    for k in ("u", "v", "w", "p"):
        assert np.all(np.isfinite(got[k])), k
    if _mem_available_gb() < 16.0:
        pytest.skip("the FP64 oracle stage at 384x256x256 needs about 8 GB of host memory")
    st = dict(u=fields[0], v=fields[1], w=fields[2], p=fields[3], N_prev=tuple(Np), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_HEAVE, params=(0.5, 1.0))
    ref, rinfo = O.rk_stage(st, mk, 1, DT, NU, g)
    errs = _stage_errors(got, ref, rinfo)
    assert stage_ok(errs, TOL_STAGE_FP32, TOL_STAGE_FP32_N), errs
    print("stage errors", errs)
