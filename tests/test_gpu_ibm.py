"""GPU parity of interpolation (Eq. 2b) and spreading (Eq. 2d) against the oracle."""

import math

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth
import paper_2406_19920_gb300 as ibm
from tests.gpu_util import IBM_INF_RATIO, TOL_IBM_FP32, TOL_IBM_FP64, dev, grid, host
from tests.gpu_util import rel_err as _rel_err


def rel_err(x, ref):
    return _rel_err(x, ref, IBM_INF_RATIO)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    # (nx, ny, nz, markers, radius)
    (32, 32, 32, 1000, 0.25),      # workload-0 sphere
    (64, 48, 96, 4000, 0.4),
    (128, 128, 128, 20000, 0.25),  # workload-1 sphere (dense markers)
    (96, 64, 96, 48000, 0.3),      # above the pre-aggregation threshold (40k markers)
]


def _markers(g, n, radius, wl):
    nx, ny, nz, hx, hy, hz = g
    X, dV = synth.fibonacci_sphere(n, radius, (nx * hx / 2 + 0.013, ny * hy / 2 - 0.007, nz * hz / 2 + 0.021), hx)
    F = synth.marker_forces(n, workload=wl)
    return X, dV, F


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("kernel", [ibm.IBM_DELTA_ROMA3, ibm.IBM_DELTA_PESKIN4])
@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_ATOMIC, ibm.IBM_SPREAD_ATOMIC_DIRECT])
def test_interp_spread_match_oracle(case, kernel, prec, mode):
    """Interpolation and the two atomic spreading kernels (shared-memory
    pre-aggregation per CTA, and the direct global atomics) against the
    oracle."""
    nx, ny, nz, n, radius = case
    g = grid(nx, ny, nz)
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    tol = TOL_IBM_FP64 if prec == ibm.IBM_FP64 else TOL_IBM_FP32
    X, dV, F = _markers(g, n, radius, wl=20 + nx)
    X, dV, F = (a.astype(npdt).astype(np.float64) for a in (X, dV, F))
    r = np.random.default_rng(nx)
    u, v, w = (r.standard_normal((ny, nz, nx)).astype(npdt).astype(np.float64) for _ in range(3))
    v[0] = 0.0
    Uref = O.interp(X, u, v, w, g, kernel)
    fref = O.spread(X, F, dV, g, kernel)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        ibm.ibm_plan_set_delta(plan, kernel)
        ibm.ibm_plan_set_spread(plan, mode)
        Xd, ud, vd, wd = dev(X, dt), dev(u, dt), dev(v, dt), dev(w, dt)
        U = torch.empty((n, 3), dtype=dt, device="cuda")
        ibm.ibm_interp(plan, n, Xd, ud, vd, wd, U)
        fu, fv, fw = (torch.zeros((ny, nz, nx), dtype=dt, device="cuda") for _ in range(3))
        ibm.ibm_spread(plan, n, Xd, dev(F, dt), dev(dV, dt), fu, fv, fw)
        torch.cuda.synchronize()
        assert rel_err(host(U), Uref) <= tol
        for got, ref in zip((fu, fv, fw), fref):
            assert rel_err(host(got), ref) <= tol
        # spreading accumulates: a second call doubles the field
        ibm.ibm_spread(plan, n, Xd, dev(F, dt), dev(dV, dt), fu, fv, fw)
        torch.cuda.synchronize()
        assert rel_err(host(fu), 2 * fref[0]) <= tol
    finally:
        ibm.ibm_plan_destroy(plan)


def test_interp_spread_empty_and_wrap():
    g = grid(16, 16, 16)
    plan = ibm.ibm_plan_create(16, 16, 16, g[3:], ibm.IBM_FP64, 0)
    try:
        z = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
        U = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        ibm.ibm_interp(plan, 0, U, z, z, z, U)
        ibm.ibm_spread(plan, 0, U, U, U, z, z, z)
        # markers straddling the periodic boundaries x = 0 and z = 0
        X = np.array([[0.01, 1.0, 0.02], [2 * math.pi - 0.03, 0.9, 2 * math.pi - 0.01]])
        r = np.random.default_rng(3)
        u, v, w = r.standard_normal((3, 16, 16, 16))
        v[0] = 0
        Uref = O.interp(X, u, v, w, g)
        Ud = torch.empty((2, 3), dtype=torch.float64, device="cuda")
        ibm.ibm_interp(plan, 2, dev(X, torch.float64), dev(u, torch.float64), dev(v, torch.float64),
                       dev(w, torch.float64), Ud)
        torch.cuda.synchronize()
        assert rel_err(host(Ud), Uref) <= TOL_IBM_FP64
    finally:
        ibm.ibm_plan_destroy(plan)


GATHER_CASES = [
    # (nx, ny, nz, markers, radius)
    (32, 32, 32, 1000, 0.25),
    (64, 48, 96, 4000, 0.4),
    (24, 36, 12, 700, 0.3),  # radix 3, bricks straddling the periodic ends
]


@pytest.mark.parametrize("case", GATHER_CASES)
@pytest.mark.parametrize("kernel", [ibm.IBM_DELTA_ROMA3, ibm.IBM_DELTA_PESKIN4])
@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_gather_spread_matches_oracle(case, kernel, prec):
    """IBM_SPREAD_GATHER (Eulerian gather, Sec. 2.3.2's alternative) gives
    the oracle's spread, accumulating into the field like the atomic kernel."""
    nx, ny, nz, n, radius = case
    g = grid(nx, ny, nz)
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    tol = TOL_IBM_FP64 if prec == ibm.IBM_FP64 else TOL_IBM_FP32
    X, dV, F = _markers(g, n, radius, wl=40 + nx)
    X, dV, F = (a.astype(npdt).astype(np.float64) for a in (X, dV, F))
    fref = O.spread(X, F, dV, g, kernel)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        ibm.ibm_plan_set_delta(plan, kernel)
        ibm.ibm_plan_set_spread(plan, ibm.IBM_SPREAD_GATHER)
        Xd, Fd, dVd = dev(X, dt), dev(F, dt), dev(dV, dt)
        fu, fv, fw = (torch.zeros((ny, nz, nx), dtype=dt, device="cuda") for _ in range(3))
        ibm.ibm_spread(plan, n, Xd, Fd, dVd, fu, fv, fw)
        torch.cuda.synchronize()
        for got, ref in zip((fu, fv, fw), fref):
            assert rel_err(host(got), ref) <= tol
        assert np.all(host(fv)[0] == 0.0)  # v's wall face is not an unknown
        ibm.ibm_spread(plan, n, Xd, Fd, dVd, fu, fv, fw)
        torch.cuda.synchronize()
        assert rel_err(host(fu), 2 * fref[0]) <= tol
        ibm.ibm_plan_check(plan)
    finally:
        ibm.ibm_plan_destroy(plan)


def test_gather_spread_is_bitwise_reproducible():
    """Dense markers (20k on a 128^3 sphere): the gathered field is the same
    bytes on every call; it agrees with the atomic kernel to rounding."""
    nx = ny = nz = 128
    n = 20000
    g = grid(nx, ny, nz)
    X, dV, F = _markers(g, n, 0.25, wl=77)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], ibm.IBM_FP32_REFINED, 1)
    try:
        Xd, Fd, dVd = dev(X, torch.float32), dev(F, torch.float32), dev(dV, torch.float32)

        def spread(mode):
            ibm.ibm_plan_set_spread(plan, mode)
            f = [torch.zeros((ny, nz, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
            ibm.ibm_spread(plan, n, Xd, Fd, dVd, *f)
            torch.cuda.synchronize()
            return f

        runs = [spread(ibm.IBM_SPREAD_GATHER) for _ in range(4)]
        for r in runs[1:]:
            for a, b in zip(runs[0], r):
                assert torch.equal(a, b)
        atom = spread(ibm.IBM_SPREAD_ATOMIC)
        for a, b in zip(runs[0], atom):
            assert rel_err(host(a), host(b)) <= 1e-6
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_GATHER, ibm.IBM_SPREAD_ATOMIC, ibm.IBM_SPREAD_ATOMIC_DIRECT])
def test_spread_walls_and_wrap(mode):
    """Markers at the periodic ends and as close to both walls as the wall
    rule allows (support half-width 1.5 hy), in every spreading mode (the
    pre-aggregating CTA's box straddles the periodic ends here, so it falls
    back to direct atomics); no marker is rejected."""
    g = grid(16, 16, 16)
    hy, Ly = g[4], 16 * g[4]
    X = np.array([[0.01, 0.9, 0.02], [2 * math.pi - 0.03, 0.95, 2 * math.pi - 0.01],
                  [1.0, 1.5 * hy + 1e-3, 3.0], [2.0, Ly - 1.5 * hy - 2e-3, 4.0], [3.0, 1.0, 0.0]])
    F = np.random.default_rng(5).standard_normal((5, 3))
    dV = np.full(5, 0.01)
    for prec, dt in ((ibm.IBM_FP64, torch.float64), (ibm.IBM_FP32_REFINED, torch.float32)):
        npdt = np.float64 if dt == torch.float64 else np.float32
        Xc, Fc, dVc = (a.astype(npdt).astype(np.float64) for a in (X, F, dV))
        fref = O.spread(Xc, Fc, dVc, g)
        plan = ibm.ibm_plan_create(16, 16, 16, g[3:], prec, 0 if prec == ibm.IBM_FP64 else 1)
        try:
            ibm.ibm_plan_set_spread(plan, mode)
            f = [torch.zeros((16, 16, 16), dtype=dt, device="cuda") for _ in range(3)]
            ibm.ibm_spread(plan, 5, dev(Xc, dt), dev(Fc, dt), dev(dVc, dt), *f)
            torch.cuda.synchronize()
            tol = TOL_IBM_FP64 if dt == torch.float64 else TOL_IBM_FP32
            for got, ref in zip(f, fref):
                assert rel_err(host(got), ref) <= tol
            ibm.ibm_plan_check(plan)
        finally:
            ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("kernel", [ibm.IBM_DELTA_ROMA3, ibm.IBM_DELTA_PESKIN4])
@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
@pytest.mark.parametrize("mode", [ibm.IBM_SPREAD_GATHER, ibm.IBM_SPREAD_ATOMIC, ibm.IBM_SPREAD_ATOMIC_DIRECT])
def test_markers_within_the_support_of_a_wall_are_rejected(kernel, prec, mode):
    """The wall rule (Eq. 2b, 2d need grid values on the whole support of
    delta_h): a marker closer to a wall than the kernel's half-width (1.5 hy,
    or 2 hy for the 4-point kernel) is neither interpolated (its U is 0) nor
    spread, and ibm_plan_check reports IBM_ERR_ARG with the count of such
    markers; the other markers of the same calls match the oracle, and the
    word is cleared by the check."""
    nx, ny, nz = 24, 20, 16
    g = grid(nx, ny, nz)
    hy, Ly = g[4], ny * g[4]
    half = 1.5 if kernel == ibm.IBM_DELTA_ROMA3 else 2.0
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    tol = TOL_IBM_FP64 if prec == ibm.IBM_FP64 else TOL_IBM_FP32
    r = np.random.default_rng(17)
    n = 300
    X = np.column_stack([r.uniform(0, 2 * math.pi, n), r.uniform(0.3, Ly - 0.3, n), r.uniform(0, 2 * math.pi, n)])
    bad = np.arange(n) % 7 == 3       # 43 markers moved inside the rejection band of one wall or the other
    depth = r.uniform(0.02, 0.95, n) * half * hy
    X[:, 1] = np.where(bad, np.where(np.arange(n) % 2 == 0, depth, Ly - depth), X[:, 1])
    F = r.standard_normal((n, 3))
    dV = np.full(n, 1e-3)
    X, F, dV = (a.astype(npdt).astype(np.float64) for a in (X, F, dV))
    okk = O.clear_of_walls(X, g, kernel)
    assert np.array_equal(okk, ~bad)
    u, vv, w = (r.standard_normal((ny, nz, nx)).astype(npdt).astype(np.float64) for _ in range(3))
    vv[0] = 0.0
    Uref = np.zeros((n, 3))
    Uref[okk] = O.interp(X[okk], u, vv, w, g, kernel)
    fref = O.spread(X[okk], F[okk], dV[okk], g, kernel)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        ibm.ibm_plan_set_delta(plan, kernel)
        ibm.ibm_plan_set_spread(plan, mode)
        U = torch.full((n, 3), float("nan"), dtype=dt, device="cuda")
        ibm.ibm_interp(plan, n, dev(X, dt), dev(u, dt), dev(vv, dt), dev(w, dt), U)
        torch.cuda.synchronize()
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_plan_check(plan)
        assert e.value.code == ibm.IBM_ERR_ARG and ("%d marker" % int(bad.sum())) in str(e.value), str(e.value)
        ibm.ibm_plan_check(plan)  # cleared
        Uh = host(U)
        assert np.all(Uh[bad] == 0.0)
        assert rel_err(Uh, Uref) <= tol
        f = [torch.zeros((ny, nz, nx), dtype=dt, device="cuda") for _ in range(3)]
        ibm.ibm_spread(plan, n, dev(X, dt), dev(F, dt), dev(dV, dt), *f)
        torch.cuda.synchronize()
        with pytest.raises(ibm.IbmError) as e:
            ibm.ibm_plan_check(plan)
        assert e.value.code == ibm.IBM_ERR_ARG and ("%d marker" % int(bad.sum())) in str(e.value), str(e.value)
        for got, ref in zip(f, fref):
            assert rel_err(host(got), ref) <= tol
    finally:
        ibm.ibm_plan_destroy(plan)


@pytest.mark.parametrize("prec", [ibm.IBM_FP64, ibm.IBM_FP32_REFINED])
def test_box_spread_near_walls_and_unordered(prec):
    """Pre-aggregated spreading (IBM_SPREAD_ATOMIC from 40k markers on): a
    compact cluster of markers against each wall, as close as the wall rule
    allows (the CTA boxes reach v's wall face), and a dense sphere's markers
    in random order (most CTA boxes too large: the fallback to direct
    atomics)."""
    nx, ny, nz = 48, 40, 32
    g = grid(nx, ny, nz)
    hy = g[4]
    dt = torch.float64 if prec == ibm.IBM_FP64 else torch.float32
    npdt = np.float64 if prec == ibm.IBM_FP64 else np.float32
    tol = TOL_IBM_FP64 if prec == ibm.IBM_FP64 else TOL_IBM_FP32
    r = np.random.default_rng(7)
    n = 45000
    lo, hi = 1.5 * hy + 1e-4, ny * hy - 1.5 * hy - 0.021
    X = np.column_stack([3.0 + 0.2 * r.random(n), np.where(np.arange(n) < n // 2, lo, hi) + 0.02 * r.random(n),
                         2.0 + 0.2 * r.random(n)])
    F = r.standard_normal((n, 3))
    dV = np.full(n, 1e-3)
    X, F, dV = (a.astype(npdt).astype(np.float64) for a in (X, F, dV))
    fref = O.spread(X, F, dV, g)
    plan = ibm.ibm_plan_create(nx, ny, nz, g[3:], prec, 1)
    try:
        f = [torch.zeros((ny, nz, nx), dtype=dt, device="cuda") for _ in range(3)]
        ibm.ibm_spread(plan, n, dev(X, dt), dev(F, dt), dev(dV, dt), *f)
        torch.cuda.synchronize()
        for got, ref in zip(f, fref):
            assert rel_err(host(got), ref) <= tol
        assert np.all(host(f[1])[0] == 0.0)
    finally:
        ibm.ibm_plan_destroy(plan)
    g = grid(128, 128, 128)
    X, dV, F = _markers(g, 45000, 0.25, wl=61)
    perm = np.random.default_rng(8).permutation(45000)
    X, dV, F = (np.ascontiguousarray(a[perm]).astype(npdt).astype(np.float64) for a in (X, dV, F))
    fref = O.spread(X, F, dV, g)
    plan = ibm.ibm_plan_create(128, 128, 128, g[3:], prec, 1)
    try:
        f = [torch.zeros((128, 128, 128), dtype=dt, device="cuda") for _ in range(3)]
        ibm.ibm_spread(plan, 45000, dev(X, dt), dev(F, dt), dev(dV, dt), *f)
        torch.cuda.synchronize()
        for got, ref in zip(f, fref):
            assert rel_err(host(got), ref) <= tol
    finally:
        ibm.ibm_plan_destroy(plan)
