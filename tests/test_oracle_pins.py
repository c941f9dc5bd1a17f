"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something it does not compute itself:
closed forms (Appendix A modified wavenumbers, the RK amplification
polynomial), dense matrices assembled here entry by entry from Appendix B,
brute-force dense solves on 8^3 grids, and the regularised-delta moment
identities.  A dropped term, a wrong sign, a transposed axis or a wrong index
in the oracle fails at least one of them.
"""

import math

import numpy as np
import pytest

from oracle import ibm_oracle as O
from paper_2406_19920_gb300 import synth


def _grid(nx, ny, nz, Lx=2 * math.pi, Ly=2.0, Lz=2 * math.pi):
    return (nx, ny, nz, Lx / nx, Ly / ny, Lz / nz)


# ---------------------------------------------------------------------------
# dense matrices written from Appendix B (independent of the oracle)
# ---------------------------------------------------------------------------

def _periodic_1d(n, h):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = -2.0 / h ** 2
        A[i, (i + 1) % n] += 1.0 / h ** 2
        A[i, (i - 1) % n] += 1.0 / h ** 2
    return A


def _wall_1d(n, h, bc):
    """Appendix B pencil matrix without the periodic part (kappa' = 0).

    Neumann: corners A3 + A2 (A3 = -2/h^2, A2 = 1/h^2).
    Cell Dirichlet (alpha = 2): corners A11 = A1 - A2.
    Face Dirichlet (alpha = 1): corners A11 = A1, n-1 interior faces.
    """
    A2 = 1.0 / h ** 2
    A1 = -2.0 / h ** 2
    m = n - 1 if bc == O.FACE_DIRICHLET else n
    A = np.zeros((m, m))
    for i in range(m):
        A[i, i] = A1
        if i > 0:
            A[i, i - 1] = A2
        if i < m - 1:
            A[i, i + 1] = A2
    if bc == O.NEUMANN:
        A[0, 0] = A[-1, -1] = A1 + A2
    elif bc == O.CELL_DIRICHLET:
        A[0, 0] = A[-1, -1] = A1 - A2
    return A


def _dense_laplacian(grid, bc):
    """Kronecker sum for the (y, z, x) C-order unknown vector."""
    nx, ny, nz, hx, hy, hz = grid
    Ay = _periodic_1d(ny, hy) if bc == O.PERIODIC else _wall_1d(ny, hy, bc)
    Ax, Az = _periodic_1d(nx, hx), _periodic_1d(nz, hz)
    Iy, Iz, Ix = np.eye(Ay.shape[0]), np.eye(nz), np.eye(nx)
    return (np.kron(np.kron(Ay, Iz), Ix) + np.kron(np.kron(Iy, Az), Ix)
            + np.kron(np.kron(Iy, Iz), Ax))


def _pack(f, bc):
    return (f[1:] if bc == O.FACE_DIRICHLET else f).ravel()


def _unpack(x, grid, bc):
    nx, ny, nz = grid[:3]
    if bc == O.FACE_DIRICHLET:
        out = np.zeros((ny, nz, nx))
        out[1:] = x.reshape(ny - 1, nz, nx)
        return out
    return x.reshape(ny, nz, nx)


GRIDS_8 = [_grid(8, 8, 8), _grid(8, 8, 8, Lx=1.0, Ly=3.0, Lz=0.5), _grid(6, 8, 4, Lx=1.3, Ly=0.7, Lz=2.1)]


# ---------------------------------------------------------------------------
# Appendix A: modified wavenumber
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,h", [(8, 0.3), (32, 2 * math.pi / 32), (48, 0.01)])
def test_modified_wavenumber_is_stencil_eigenvalue(n, h):
    """The 3-point stencil on exp(i kappa x) returns -kappa'^2 of Appendix A."""
    x = np.arange(n) * h
    for m in range(n):
        kappa = 2 * math.pi * m / (n * h)
        f = np.exp(1j * kappa * x)
        d2 = (np.roll(f, -1) - 2 * f + np.roll(f, 1)) / h ** 2
        k2 = O.modified_wavenumber_sq(kappa * h, h)
        assert np.allclose(d2, -k2 * f, rtol=0, atol=1e-9 * (4 / h ** 2))
        # long waves: kappa'^2 -> kappa^2 at second order
    kappa = 2 * math.pi / (n * h)
    assert abs(O.modified_wavenumber_sq(kappa * h, h) - kappa ** 2) <= kappa ** 4 * h ** 2 / 12 * 1.01


@pytest.mark.parametrize("bc", [O.NEUMANN, O.CELL_DIRICHLET, O.FACE_DIRICHLET])
@pytest.mark.parametrize("n", [8, 9, 16])
def test_wall_basis_diagonalises_appendix_b_matrix(bc, n):
    h = 0.37
    A = _wall_1d(n, h, bc)
    Q, th = O.wall_basis(n, bc)
    Qi = Q[1:] if bc == O.FACE_DIRICHLET else Q
    assert np.allclose(Qi.T @ Qi, np.eye(Qi.shape[1]), atol=1e-13)
    lam = O.modified_wavenumber_sq(th, h)
    assert np.allclose(A @ Qi, -Qi * lam[None, :], atol=1e-10 / h ** 2)


@pytest.mark.parametrize("n", [8, 9, 12])
def test_fourier_basis_orthonormal_eigen(n):
    h = 0.2
    Q, th = O.fourier_basis(n)
    assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    A = _periodic_1d(n, h)
    assert np.allclose(A @ Q, -Q * O.modified_wavenumber_sq(th, h)[None, :], atol=1e-10 / h ** 2)


# ---------------------------------------------------------------------------
# Operators and solves against dense matrices (8^3 brute force)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("grid", GRIDS_8)
@pytest.mark.parametrize("bc", [O.NEUMANN, O.CELL_DIRICHLET, O.FACE_DIRICHLET])
def test_laplacian_matches_dense(grid, bc):
    A = _dense_laplacian(grid, bc)
    f = np.random.default_rng(3).standard_normal((grid[1], grid[2], grid[0]))
    got = O.laplacian(f, grid, bc)
    want = _unpack(A @ _pack(f, bc), grid, bc)
    assert np.allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("grid", GRIDS_8)
def test_poisson_matches_dense_gaussian_elimination(grid):
    nx, ny, nz = grid[:3]
    A = _dense_laplacian(grid, O.NEUMANN)
    b = np.random.default_rng(4).standard_normal((ny, nz, nx))
    # singular on constants: append the mean-zero constraint and solve the
    # bordered system [A 1; 1^T 0] (exact for a compatible rhs)
    N = A.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = A
    B[:N, N] = 1.0
    B[N, :N] = 1.0
    rhs = np.concatenate([(b - b.mean()).ravel(), [0.0]])
    x = np.linalg.solve(B, rhs)
    assert abs(x[N]) < 1e-10            # compatible rhs: zero multiplier
    phi, mean_b = O.poisson_solve(b, grid)
    assert abs(mean_b - b.mean()) < 1e-15
    assert O.rel_l2(phi, x[:N].reshape(ny, nz, nx)) < 1e-12


@pytest.mark.parametrize("grid", GRIDS_8)
@pytest.mark.parametrize("bc", [O.NEUMANN, O.CELL_DIRICHLET, O.FACE_DIRICHLET])
@pytest.mark.parametrize("c", [1e-3, 0.25])
def test_helmholtz_matches_dense(grid, bc, c):
    nx, ny, nz = grid[:3]
    A = _dense_laplacian(grid, bc)
    r = np.random.default_rng(5).standard_normal((ny, nz, nx))
    M = np.eye(A.shape[0]) - c * A
    x = np.linalg.solve(M, _pack(r, bc))
    u = O.helmholtz_solve(r, grid, c, bc)
    assert O.rel_l2(u, _unpack(x, grid, bc)) < 1e-12
    if bc == O.FACE_DIRICHLET:
        assert np.all(u[0] == 0.0)


# ---------------------------------------------------------------------------
# triply periodic branch (Sec. 2.3.3, S2): y periodic as well
# ---------------------------------------------------------------------------

GRIDS_3P = [_grid(8, 8, 8), _grid(6, 12, 4, Lx=1.3, Ly=0.7, Lz=2.1)]


@pytest.mark.parametrize("grid", GRIDS_3P)
def test_periodic_laplacian_matches_dense(grid):
    A = _dense_laplacian(grid, O.PERIODIC)
    f = np.random.default_rng(31).standard_normal((grid[1], grid[2], grid[0]))
    want = (A @ f.ravel()).reshape(f.shape)
    got = O.laplacian(f, grid, O.PERIODIC)
    assert np.allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("grid", GRIDS_3P)
def test_periodic_poisson_matches_dense_bordered_solve(grid):
    nx, ny, nz = grid[:3]
    A = _dense_laplacian(grid, O.PERIODIC)
    b = np.random.default_rng(32).standard_normal((ny, nz, nx))
    N = A.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = A
    B[:N, N] = 1.0
    B[N, :N] = 1.0
    x = np.linalg.solve(B, np.concatenate([(b - b.mean()).ravel(), [0.0]]))
    assert abs(x[N]) < 1e-10
    phi, mean_b = O.poisson_solve(b, grid, ybc=O.PERIODIC)
    assert abs(mean_b - b.mean()) < 1e-15
    assert abs(phi.mean()) < 1e-14
    assert O.rel_l2(phi, x[:N].reshape(ny, nz, nx)) < 1e-12
    with pytest.raises(ValueError):
        O.poisson_solve(b, grid, nullspace="pin", ybc=O.PERIODIC)


@pytest.mark.parametrize("grid", GRIDS_3P)
@pytest.mark.parametrize("c", [1e-3, 0.25])
def test_periodic_helmholtz_matches_dense(grid, c):
    nx, ny, nz = grid[:3]
    A = _dense_laplacian(grid, O.PERIODIC)
    r = np.random.default_rng(33).standard_normal((ny, nz, nx))
    x = np.linalg.solve(np.eye(A.shape[0]) - c * A, r.ravel())
    u = O.helmholtz_solve(r, grid, c, O.PERIODIC)
    assert O.rel_l2(u, x.reshape(ny, nz, nx)) < 1e-12


def test_periodic_manufactured_mode_exact():
    """A Fourier mode in all three axes is an exact discrete eigenfunction."""
    g = _grid(24, 16, 32, Ly=3.0)
    nx, ny, nz, hx, hy, hz = g
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    phi = (np.sin(2 * math.pi * 3 * j / ny)[:, None, None]
           * np.cos(2 * math.pi * 5 * k / nz)[None, :, None]
           * np.sin(2 * math.pi * 2 * i / nx)[None, None, :])
    lam = (O.modified_wavenumber_sq(2 * math.pi * 2 / nx, hx) + O.modified_wavenumber_sq(2 * math.pi * 3 / ny, hy)
           + O.modified_wavenumber_sq(2 * math.pi * 5 / nz, hz))
    assert np.abs(O.laplacian(phi, g, O.PERIODIC) + lam * phi).max() < 1e-11 * lam
    got, _ = O.poisson_solve(-lam * phi, g, ybc=O.PERIODIC)
    assert O.rel_l2(got, phi) < 1e-13


def test_manufactured_eigenfunction_exact():
    """Discrete eigenfunction rhs: the solve is exact to round-off."""
    g = _grid(32, 32, 32)
    nx, ny, nz, hx, hy, hz = g
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    mx, my, mz = 3, 5, 2
    phi = (np.cos(math.pi * my * (j + 0.5) / ny)[:, None, None]
           * np.sin(2 * math.pi * mz * k / nz)[None, :, None]
           * np.cos(2 * math.pi * mx * i / nx)[None, None, :])
    lam = (O.modified_wavenumber_sq(2 * math.pi * mx / nx, hx)
           + O.modified_wavenumber_sq(math.pi * my / ny, hy)
           + O.modified_wavenumber_sq(2 * math.pi * mz / nz, hz))
    b = -lam * phi
    got, _ = O.poisson_solve(b, g)
    assert O.rel_l2(got, phi) < 1e-13
    assert np.abs(O.laplacian(phi, g, O.NEUMANN) - b).max() < 1e-12 * lam
    # Helmholtz on a cell-Dirichlet mode
    ud = (np.sin(math.pi * 3 * (j + 0.5) / ny)[:, None, None]
          * np.cos(2 * math.pi * 1 * k / nz)[None, :, None]
          * np.sin(2 * math.pi * 4 * i / nx)[None, None, :])
    lam_d = (O.modified_wavenumber_sq(2 * math.pi * 4 / nx, hx)
             + O.modified_wavenumber_sq(math.pi * 3 / ny, hy)
             + O.modified_wavenumber_sq(2 * math.pi * 1 / nz, hz))
    c = 0.01
    got = O.helmholtz_solve((1 + c * lam_d) * ud, g, c, O.CELL_DIRICHLET)
    assert O.rel_l2(got, ud) < 1e-13


def test_residual_and_symmetry_32():
    g = _grid(32, 32, 32)
    b, _ = synth.rhs_eigen_sum(32, 32, 32, workload=0)
    phi, _ = O.poisson_solve(b, g)
    assert O.normalised_residual(phi, b, g) <= 1e-12
    r = np.random.default_rng(6)
    for bc in (O.NEUMANN, O.CELL_DIRICHLET, O.FACE_DIRICHLET):
        x, y = r.standard_normal((2, 32, 32, 32))
        if bc == O.FACE_DIRICHLET:
            x[0] = y[0] = 0
        lhs = np.vdot(O.laplacian(x, g, bc), y)
        rhs = np.vdot(x, O.laplacian(y, g, bc))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs) + 1e-9


def test_pin_and_mean_differ_by_constant():
    g = _grid(16, 16, 16)
    b = np.random.default_rng(7).standard_normal((16, 16, 16))
    pm, _ = O.poisson_solve(b, g, "mean")
    pp, _ = O.poisson_solve(b, g, "pin")
    d = pp - pm
    assert np.ptp(d) < 1e-12
    assert abs(pp[0].mean()) < 1e-13
    assert abs(pm.mean()) < 1e-13


# ---------------------------------------------------------------------------
# Divergence, gradient, projection, advection
# ---------------------------------------------------------------------------

def test_div_grad_is_neumann_laplacian():
    g = _grid(12, 10, 8, Lx=1.0, Ly=2.0, Lz=3.0)
    phi = np.random.default_rng(8).standard_normal((10, 8, 12))
    assert np.allclose(O.divergence(*O.gradient(phi, g), g), O.laplacian(phi, g, O.NEUMANN), atol=1e-9)


def test_projection_makes_divergence_free():
    g = _grid(16, 16, 16)
    r = np.random.default_rng(9)
    u, v, w = r.standard_normal((3, 16, 16, 16))
    v[0] = 0
    k = 0.37
    d = O.divergence(u, v, w, g)
    phi, _ = O.poisson_solve(d / k, g)
    G = O.gradient(phi, g)
    un, vn, wn = u - k * G[0], v - k * G[1], w - k * G[2]
    dn = O.divergence(un, vn, wn, g)
    assert np.abs(dn).max() <= 1e-12 * np.abs(d).max()
    assert np.all(vn[0] == 0)


def test_synthetic_velocity_is_discretely_divergence_free():
    g = _grid(24, 16, 20)
    u, v, w = synth.div_free_velocity(g, workload=1, kmax=6)
    d = O.divergence(u, v, w, g)
    assert np.abs(d).max() < 1e-10 * (np.abs(u).max() / g[3])


def test_advection_conserves_momentum_and_energy():
    """Divergence-form MAC advection: x/z momentum fluxes telescope and, for a
    discretely divergence-free field with v = 0 on the walls, the kinetic
    energy production sum u.N vanishes (Morinishi et al. 1998)."""
    g = _grid(16, 12, 8, Lx=1.0, Ly=1.5, Lz=0.8)
    u, v, w = synth.div_free_velocity(g, workload=2, kmax=5)
    Nu, Nv, Nw = O.advection(u, v, w, g)
    scale = np.abs(Nu).max()
    assert abs(Nu.sum()) < 1e-11 * scale * Nu.size
    assert abs(Nw.sum()) < 1e-11 * scale * Nw.size
    e = np.vdot(u, Nu) + np.vdot(v[1:], Nv[1:]) + np.vdot(w, Nw)
    assert abs(e) < 1e-11 * scale * np.abs(u).sum()
    # a non-solenoidal field does produce energy (the test can fail)
    r = np.random.default_rng(1)
    a, b, c = r.standard_normal((3,) + u.shape)
    b[0] = 0
    Na = O.advection(a, b, c, g)
    assert abs(np.vdot(a, Na[0]) + np.vdot(b[1:], Na[1][1:]) + np.vdot(c, Na[2])) > 1e-3


def test_advection_of_uniform_shear_is_zero():
    """u = U(y, z) with v = w = 0 is a steady Euler solution: N = 0."""
    g = _grid(8, 8, 8)
    u = np.random.default_rng(2).standard_normal((8, 8, 1)) * np.ones((8, 8, 8))
    z = np.zeros_like(u)
    for comp in O.advection(u, z, z, g):
        assert np.abs(comp).max() < 1e-13


# ---------------------------------------------------------------------------
# Regularised delta kernels (Eq. 2b, 2d; Roma et al. 1999, Peskin 2002)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel,sum_sq,support", [(O.ROMA3, 0.5, 1.5), (O.PESKIN4, 3.0 / 8.0, 2.0)])
def test_delta_moments(kernel, sum_sq, support):
    r = np.random.default_rng(10).uniform(-0.5, 0.5, 2000)
    j = np.arange(-3, 4)
    phi = O.delta_1d(r[:, None] - j[None, :], kernel)
    assert np.allclose(phi.sum(1), 1.0, atol=1e-14)                      # partition of unity
    assert np.allclose(((r[:, None] - j[None, :]) * phi).sum(1), 0, atol=1e-14)   # first moment
    assert np.allclose((phi ** 2).sum(1), sum_sq, atol=1e-14)            # sum of squares
    assert np.all(O.delta_1d(np.array([support + 1e-9, -support - 1e-9, 3.0]), kernel) == 0)
    assert np.all(phi >= 0)


def _sphere(g, n, workload=0):
    nx, ny, nz, hx, hy, hz = g
    Lx, Ly, Lz = nx * hx, ny * hy, nz * hz
    X, dV = synth.fibonacci_sphere(n, 0.25 * Ly / 2 * 2, (Lx / 2, Ly / 2, Lz / 2), hx)
    return X, dV


@pytest.mark.parametrize("kernel", [O.ROMA3, O.PESKIN4])
def test_interp_exact_for_linear_fields(kernel):
    g = _grid(32, 32, 32)
    nx, ny, nz, hx, hy, hz = g
    X, _ = _sphere(g, 300)
    j, k, i = np.meshgrid(np.arange(ny), np.arange(nz), np.arange(nx), indexing="ij")
    a, bx, by, bz = 0.7, 0.3, -1.1, 0.45
    origins = {0: (0.0, 0.5, 0.5), 1: (0.5, 0.0, 0.5), 2: (0.5, 0.5, 0.0)}
    fields = []
    for c in range(3):
        ox, oy, oz = origins[c]
        fields.append(a + bx * (i + ox) * hx + by * (j + oy) * hy + bz * (k + oz) * hz)
    fields[1][0] = 0.0
    U = O.interp(X, *fields, g, kernel)
    exact = a + bx * X[:, 0] + by * X[:, 1] + bz * X[:, 2]
    for c in range(3):
        assert np.allclose(U[:, c], exact, atol=1e-12)


@pytest.mark.parametrize("kernel", [O.ROMA3, O.PESKIN4])
def test_spread_conserves_force_and_moment_and_is_adjoint(kernel):
    g = _grid(32, 32, 32)
    nx, ny, nz, hx, hy, hz = g
    X, dV = _sphere(g, 500)
    F = synth.marker_forces(500, workload=0)
    fu, fv, fw = O.spread(X, F, dV, g, kernel)
    h3 = hx * hy * hz
    origins = {0: (0.0, 0.5, 0.5), 1: (0.5, 0.0, 0.5), 2: (0.5, 0.5, 0.0)}
    j, k, i = np.meshgrid(np.arange(ny), np.arange(nz), np.arange(nx), indexing="ij")
    for c, f in enumerate((fu, fv, fw)):
        assert abs(f.sum() * h3 - (F[:, c] * dV).sum()) < 1e-12 * np.abs(F[:, c] * dV).sum()
        ox, oy, oz = origins[c]
        xs = (i + ox) * hx
        assert abs((xs * f).sum() * h3 - (X[:, 0] * F[:, c] * dV).sum()) < 1e-11
    r = np.random.default_rng(11)
    u, v, w = r.standard_normal((3, ny, nz, nx))
    v[0] = 0.0
    U = O.interp(X, u, v, w, g, kernel)
    lhs = (dV[:, None] * U * F).sum()
    rhs = h3 * (np.vdot(u, fu) + np.vdot(v, fv) + np.vdot(w, fw))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12


@pytest.mark.parametrize("kernel", [O.ROMA3, O.PESKIN4])
def test_wall_rule_is_the_support_of_the_delta_kernel(kernel):
    """The markers clear_of_walls accepts are exactly those whose stencil,
    enumerated point by point with the delta kernel's own weights, puts
    non-zero weight only on stored unknowns of every component (cell rows
    0..ny-1, v faces 1..ny-1): the one-dimensional support of phi has
    half-width 1.5 (ROMA3) or 2 (PESKIN4) cells, and v's wall face sits on
    the wall.  Brute force over Y sweeping both wall regions."""
    g = _grid(8, 12, 8, Ly=1.2)
    nx, ny, nz, hx, hy, hz = g
    S = 3 if kernel == O.ROMA3 else 4
    Y = np.concatenate([np.linspace(0.0, 3.0 * hy, 601), np.linspace(g[4] * ny - 3.0 * hy, g[4] * ny, 601)])
    Y = Y[np.abs(Y / hy - round(S / 2)) > 1e-9]          # off the exact boundary
    Y = Y[np.abs((ny * hy - Y) / hy - round(S / 2)) > 1e-9]
    X = np.column_stack([np.full_like(Y, 0.37), Y, np.full_like(Y, 1.1)])
    ok = O.clear_of_walls(X, g, kernel)
    s = np.arange(-S, S + 1)
    for i, y in enumerate(Y):
        needs_outside = False
        for lo, origin in ((0, 0.5), (0, 0.5), (1, 0.0)):  # u, w (cell rows), v (faces)
            j = np.floor(y / hy - origin) + s            # candidate rows around the marker
            wgt = O.delta_1d(y / hy - origin - j, kernel)
            hit = j[wgt > 0]
            needs_outside |= bool(np.any((hit < lo) | (hit > ny - 1)))
        assert ok[i] == (not needs_outside), (y / hy, ok[i])
    assert ok.any() and (~ok).any()
    with pytest.raises(ValueError):
        O.interp(X, *np.zeros((3, ny, nz, nx)), g, kernel)
    with pytest.raises(ValueError):
        O.spread(X, np.ones_like(X), np.ones(len(X)), g, kernel)


def test_interp_spread_periodic_wrap():
    """A marker at x = 0 sees the same neighbourhood as one at x = Lx."""
    g = _grid(16, 16, 16)
    nx, ny, nz, hx, hy, hz = g
    r = np.random.default_rng(12)
    u, v, w = r.standard_normal((3, ny, nz, nx))
    v[0] = 0
    X1 = np.array([[0.01, 1.0, 0.02]])
    X2 = X1 + np.array([[nx * hx, 0.0, nz * hz]])
    assert np.allclose(O.interp(X1, u, v, w, g), O.interp(X2, u, v, w, g), atol=1e-12)


# ---------------------------------------------------------------------------
# RK coefficients (Rai & Moin) and one RK stage (Eq. 2a-2h)
# ---------------------------------------------------------------------------

def test_rk_coefficients_third_order_explicit_and_consistent():
    a, b, gm, zt = map(np.array, (O.RK_ALPHA, O.RK_BETA, O.RK_GAMMA, O.RK_ZETA))
    assert np.allclose(gm + zt, a + b)
    assert abs((a + b).sum() - 1.0) < 1e-15
    # explicit part on y' = lam y: stability polynomial 1 + z + z^2/2 + z^3/6
    for z in (0.1, -0.3, 0.05 + 0.2j):
        y, Nprev = 1.0 + 0j, 0.0
        for n in range(3):
            N = -z * y              # advection-like term with du/dt = -N
            y = y + (-gm[n] * N - zt[n] * Nprev)
            Nprev = N
        assert abs(y - (1 + z + z ** 2 / 2 + z ** 3 / 6)) < 1e-14
    # implicit part: second order, prod (1 + a z)/(1 - b z) = e^z + O(z^3)
    for z in (1e-2, -2e-2):
        R = np.prod((1 + a * z) / (1 - b * z))
        assert abs(R - math.exp(z)) < 0.2 * abs(z) ** 3


@pytest.mark.parametrize("stage", [1, 2, 3])
def test_rk_stage_viscous_mode_closed_form(stage):
    """u = sin(pi m (j+1/2)/ny) cos(2 pi q k / nz), v = w = 0, p = 0, no
    markers: N = 0, div u = 0, so Eq. 2a-2h reduce to
    u^n = u (1 - alpha nu dt lam) / (1 + beta nu dt lam) and phi = p^n = 0."""
    g = _grid(16, 16, 16)
    nx, ny, nz, hx, hy, hz = g
    j, k = np.arange(ny), np.arange(nz)
    m, q = 2, 3
    u = (np.sin(math.pi * m * (j + 0.5) / ny)[:, None, None]
         * np.cos(2 * math.pi * q * k / nz)[None, :, None]) * np.ones((1, 1, nx))
    z = np.zeros_like(u)
    lam = O.modified_wavenumber_sq(math.pi * m / ny, hy) + O.modified_wavenumber_sq(2 * math.pi * q / nz, hz)
    dt, nu = 1e-2, 0.3
    st = dict(u=u, v=z.copy(), w=z.copy(), p=z.copy(), N_prev=(z, z, z), t=0.0)
    mk = dict(X0=np.zeros((0, 3)), dV=np.zeros(0), kind=O.MOTION_STATIC, params=())
    new, info = O.rk_stage(st, mk, stage, dt, nu, g)
    a, b = O.RK_ALPHA[stage - 1], O.RK_BETA[stage - 1]
    want = u * (1 - a * nu * dt * lam) / (1 + b * nu * dt * lam)
    assert O.rel_l2(new["u"], want) < 1e-13
    assert np.abs(new["v"]).max() < 1e-13 and np.abs(new["w"]).max() < 1e-13
    assert np.abs(new["p"]).max() < 1e-10
    assert abs(new["t"] - (a + b) * dt) < 1e-16


def test_rk_stage_projection_and_forcing_invariants():
    g = _grid(16, 16, 16)
    nx, ny, nz, hx, hy, hz = g
    u, v, w = synth.div_free_velocity(g, workload=3, kmax=4)
    z = np.zeros_like(u)
    X0, dV = synth.fibonacci_sphere(200, 0.25, (math.pi, 1.0, math.pi), hx)
    st = dict(u=u, v=v, w=w, p=z.copy(), N_prev=(z, z, z), t=0.0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_TRANSLATE, params=(0.1, 0.0, 0.0))
    new, info = O.rk_stage(st, mk, 1, 1e-3, 1e-2, g)
    d = O.divergence(new["u"], new["v"], new["w"], g)
    d0 = O.divergence(*info["ustar"], g)
    assert np.abs(d).max() <= 1e-11 * max(1.0, np.abs(d0).max())
    # Eq. 2c: F = (U^d - U^e)/dt
    assert np.allclose(info["F"], (np.array([0.1, 0, 0])[None, :] - info["Ue"]) / 1e-3)


def _no_markers():
    return dict(X0=np.zeros((0, 3)), dV=np.zeros(0), kind=O.MOTION_STATIC, params=())


@pytest.mark.parametrize("stage", [2, 3])
@pytest.mark.parametrize("comp", [0, 2])
def test_rk_stage_history_term_closed_form(stage, comp):
    """The -zeta N^{n-2} term of Eq. 2a on its own.  With u = v = w = p = 0
    and N_prev a single mode that is an eigenfunction of its component's
    Helmholtz operator and carries no divergence (the u component varies in
    y and z only, the w component in y and x only), Eq. 2a gives
    u^e = -zeta dt N_prev, Eq. 2e divides by 1 + beta nu dt lam, the
    divergence and hence phi vanish, so u^n = -zeta dt N_prev / (1 + beta nu
    dt lam) and p^n = 0.  A wrong sign or factor on zeta, or the history
    term landing on another component, fails this."""
    g = _grid(16, 12, 8, Lx=1.7, Ly=1.1, Lz=0.9)
    nx, ny, nz, hx, hy, hz = g
    m, q = 3, 2
    j = np.arange(ny)
    ymode = np.sin(math.pi * m * (j + 0.5) / ny)
    if comp == 0:   # u on x-faces: vary along z (k hz + hz/2 is a shift; the cos mode stays an eigenvector)
        f = ymode[:, None, None] * np.cos(2 * math.pi * q * np.arange(nz) / nz)[None, :, None] * np.ones((1, 1, nx))
        lam = O.modified_wavenumber_sq(math.pi * m / ny, hy) + O.modified_wavenumber_sq(2 * math.pi * q / nz, hz)
    else:           # w on z-faces: vary along x
        f = ymode[:, None, None] * np.ones((1, nz, 1)) * np.cos(2 * math.pi * q * np.arange(nx) / nx)[None, None, :]
        lam = O.modified_wavenumber_sq(math.pi * m / ny, hy) + O.modified_wavenumber_sq(2 * math.pi * q / nx, hx)
    z = np.zeros_like(f)
    Np = [z, z, z]
    Np[comp] = f
    dt, nu, stage_i = 3e-3, 0.2, stage - 1
    st = dict(u=z.copy(), v=z.copy(), w=z.copy(), p=z.copy(), N_prev=tuple(Np), t=0.0)
    new, info = O.rk_stage(st, _no_markers(), stage, dt, nu, g)
    zeta, beta = O.RK_ZETA[stage_i], O.RK_BETA[stage_i]
    want = -zeta * dt * f / (1.0 + beta * nu * dt * lam)
    names = ("u", "v", "w")
    assert O.rel_l2(new[names[comp]], want) < 1e-13
    for c in range(3):
        if c != comp:
            assert np.abs(new[names[c]]).max() < 1e-14
    assert np.abs(new["p"]).max() < 1e-12 * np.abs(want).max()
    assert np.abs(info["phi"]).max() < 1e-12 * np.abs(want).max()
    for c in range(3):                      # N(0) = 0 is the next stage's history
        assert np.abs(new["N_prev"][c]).max() == 0.0


@pytest.mark.parametrize("stage", [1, 2, 3])
def test_rk_stage_pressure_gradient_projection_and_update_cancel(stage):
    """The -(alpha+beta) G p term of Eq. 2a, the projection (Eq. 2g) and the
    pressure update (Eq. 2h) together.  u = v = w = 0 and p a y-only
    Neumann mode cos(pi m (j+1/2)/ny): u^e = -(a+b) dt G p is a single
    face-Dirichlet mode of v (the discrete gradient of the cosine is the
    sine on faces), Eq. 2e divides it by 1 + c lam (c = beta dt nu), its
    divergence over (a+b) dt is lam p / (1 + c lam), so Eq. 2f gives
    phi = -p / (1 + c lam).  The projection then returns u^n = 0 exactly and
    Eq. 2h p^n = p + phi - c L phi = 0.  A wrong coefficient on G p, a sign
    slip in the projection, or a wrong sign or factor in the pressure update
    leaves a non-zero u^n or p^n."""
    g = _grid(8, 16, 6, Lx=1.0, Ly=1.3, Lz=0.8)
    nx, ny, nz, hx, hy, hz = g
    m = 2
    p = np.cos(math.pi * m * (np.arange(ny) + 0.5) / ny)[:, None, None] * np.ones((1, nz, nx))
    lam = O.modified_wavenumber_sq(math.pi * m / ny, hy)
    dt, nu = 2e-3, 0.7
    z = np.zeros_like(p)
    st = dict(u=z.copy(), v=z.copy(), w=z.copy(), p=p, N_prev=(z, z, z), t=0.0)
    new, info = O.rk_stage(st, _no_markers(), stage, dt, nu, g)
    cH = O.RK_BETA[stage - 1] * dt * nu
    assert O.rel_l2(info["phi"], -p / (1.0 + cH * lam)) < 1e-12
    # v* carries the whole pressure-gradient step before the projection
    ab = O.RK_ALPHA[stage - 1] + O.RK_BETA[stage - 1]
    gv = np.zeros_like(p)
    gv[1:] = (p[1:] - p[:-1]) / hy
    assert O.rel_l2(info["ustar"][1], -ab * dt * gv / (1.0 + cH * lam)) < 1e-12
    vmax = ab * dt * np.abs(gv).max()
    for name in ("u", "v", "w"):
        assert np.abs(new[name]).max() < 1e-12 * vmax
    assert np.abs(new["p"]).max() < 1e-12


@pytest.mark.parametrize("stage", [2, 3])
def test_rk_stage_advection_term_by_superposition(stage):
    """The -gamma N(u) term of Eq. 2a, pinned against the history term.

    With p = 0 and no markers every output of the stage is an affine map of
    the explicit estimate u^e, and u^e = lin(u) - dt (gamma N(u) + zeta
    N_prev) with lin linear in u and N quadratic.  Hence
      out(u) + out(-u) = 2 S(-gamma dt N(u))            (the linear parts cancel)
      out(u; N_prev = N(u)) - out(u; 0) = S(-zeta dt N(u)),
    S the linear solve-and-project map, so the second difference equals
    zeta / gamma times half the first.  The history term is pinned on its
    own above, so this fixes gamma's sign and size, and that the advection
    enters every component."""
    g = _grid(16, 12, 8, Lx=1.0, Ly=1.5, Lz=0.8)
    u, v, w = synth.div_free_velocity(g, workload=5, kmax=4)
    z = np.zeros_like(u)
    dt, nu = 4e-3, 0.05
    names = ("u", "v", "w", "p")

    def run(sign, Np):
        st = dict(u=sign * u, v=sign * v, w=sign * w, p=z.copy(), N_prev=Np, t=0.0)
        return O.rk_stage(st, _no_markers(), stage, dt, nu, g)[0]

    N = O.advection(u, v, w, g)
    plus, minus, hist = run(1.0, (z, z, z)), run(-1.0, (z, z, z)), run(1.0, N)
    ratio = O.RK_ZETA[stage - 1] / O.RK_GAMMA[stage - 1]
    for name in names:
        sym = 0.5 * (plus[name] + minus[name])          # S(-gamma dt N(u))
        assert np.abs(sym).max() > 1e-6                 # the advection term is present
        d = hist[name] - plus[name]                     # S(-zeta dt N(u))
        assert np.abs(d - ratio * sym).max() <= 1e-10 * np.abs(sym).max(), name


def test_heave_motion_closed_form_values():
    """HEAVE (L2): at t = 0, T/4, T/2, 3T/4 the plate sits at y0, y0 + A, y0,
    y0 - A with vertical velocity 2 pi A / T, 0, -2 pi A / T, 0; x and z
    never move; the motion has period T; U^d is the time derivative of X
    (central difference)."""
    X0 = np.array([[0.3, 1.1, 2.0], [1.0, 0.9, 0.1]])
    A, T = 0.5, 1.7
    w = 2 * math.pi * A / T
    for t, dy, vy in ((0.0, 0.0, w), (T / 4, A, 0.0), (T / 2, 0.0, -w), (3 * T / 4, -A, 0.0)):
        X, Ud = O.marker_motion(X0, t, O.MOTION_HEAVE, (A, T))
        assert np.allclose(X[:, 1] - X0[:, 1], dy, atol=1e-14)
        assert np.allclose(Ud[:, 1], vy, atol=1e-14)
        assert np.array_equal(X[:, [0, 2]], X0[:, [0, 2]])
        assert np.array_equal(Ud[:, [0, 2]], np.zeros((2, 2)))
    for t in (0.137, 0.9, 2.3):
        X, Ud = O.marker_motion(X0, t, O.MOTION_HEAVE, (A, T))
        Xp = O.marker_motion(X0, t + T, O.MOTION_HEAVE, (A, T))[0]
        assert np.allclose(X, Xp, atol=1e-13)
        e = 1e-5
        d = (O.marker_motion(X0, t + e, O.MOTION_HEAVE, (A, T))[0]
             - O.marker_motion(X0, t - e, O.MOTION_HEAVE, (A, T))[0]) / (2 * e)
        assert np.allclose(d, Ud, atol=1e-8)


def test_rk_stage_forces_markers_at_the_stage_start_time():
    """With every field zero the interpolated velocity is zero, so Eq. 2c
    gives F = U^d / dt with U^d the heave velocity at the stage's start
    time t (not t + dt or the end of the stage)."""
    g = _grid(16, 16, 16)
    X0, dV = synth.fibonacci_sphere(50, 0.25, (math.pi, 1.0, math.pi), g[3])
    z = np.zeros((16, 16, 16))
    A, T, t0, dt = 0.1, 0.8, 0.13, 1e-3
    st = dict(u=z.copy(), v=z.copy(), w=z.copy(), p=z.copy(), N_prev=(z, z, z), t=t0)
    mk = dict(X0=X0, dV=dV, kind=O.MOTION_HEAVE, params=(A, T))
    new, info = O.rk_stage(st, mk, 1, dt, 1e-2, g)
    vy = 2 * math.pi * A / T * math.cos(2 * math.pi * t0 / T)
    assert np.allclose(info["F"][:, 1], vy / dt, rtol=1e-13)
    assert np.abs(info["F"][:, [0, 2]]).max() == 0.0
    assert abs(new["t"] - (t0 + (O.RK_ALPHA[0] + O.RK_BETA[0]) * dt)) < 1e-16


# ---------------------------------------------------------------------------
# Inhomogeneous wall data (Appendix B: boundary values on the first and last
# pencil rows' right-hand sides)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [O.NEUMANN, O.CELL_DIRICHLET, O.FACE_DIRICHLET])
def test_wall_data_ghosts_exact_on_linear_fields(bc):
    """The ghost rules with wall data reproduce a field linear in y exactly:
    a Neumann ghost from the slope, a cell-Dirichlet ghost by reflection
    through the wall value, a face-Dirichlet wall face at its value.  The
    7-point Laplacian of such a field vanishes on every row, wall rows
    included."""
    grid = _grid(8, 10, 6, Ly=1.7)
    nx, ny, nz, hx, hy, hz = grid
    a, bslope = 0.7, -2.3
    ones = np.ones((nz, nx))
    if bc == O.FACE_DIRICHLET:
        y = np.arange(ny) * hy                 # faces j = 0 .. ny-1
        g_lo, g_hi = a * ones, (a + bslope * ny * hy) * ones
    else:
        y = (np.arange(ny) + 0.5) * hy         # cell centres
        if bc == O.NEUMANN:
            g_lo = g_hi = bslope * ones
        else:
            g_lo, g_hi = a * ones, (a + bslope * ny * hy) * ones
    f = (a + bslope * y)[:, None, None] * np.ones((ny, nz, nx))
    L = O.laplacian(f, grid, bc, g_lo, g_hi)
    assert np.max(np.abs(L)) <= 1e-9 / hy ** 2
    # and the homogeneous rule does not (the data matter)
    assert np.max(np.abs(O.laplacian(f, grid, bc))) > 1e-3


@pytest.mark.parametrize("bc", [O.NEUMANN, O.CELL_DIRICHLET, O.FACE_DIRICHLET])
def test_helmholtz_with_wall_data_manufactured(bc):
    """(I - c L_h) u = r with the ghosts of the wall data: the solve with that
    data returns u (face fields: plane 0 is the wall value)."""
    grid = _grid(8, 12, 6, Ly=1.3)
    nx, ny, nz = grid[:3]
    rng = np.random.default_rng(61 + bc)
    u = rng.standard_normal((ny, nz, nx))
    g_lo, g_hi = rng.standard_normal((2, nz, nx))
    if bc == O.FACE_DIRICHLET:
        u[0] = g_lo
    c = 0.03
    r = u - c * O.laplacian(u, grid, bc, g_lo, g_hi)
    got = O.helmholtz_solve(r, grid, c, bc, g_lo, g_hi)
    assert np.max(np.abs(got - u)) <= 1e-11 * np.max(np.abs(u))


def test_poisson_with_flux_manufactured():
    """L_h phi = b with the Neumann ghosts of dphi/dy = q at the walls: the
    solve returns phi up to its mean, and the data-corrected right-hand side
    is compatible (discrete divergence theorem: nothing to remove)."""
    grid = _grid(8, 10, 6, Ly=1.1)
    nx, ny, nz = grid[:3]
    rng = np.random.default_rng(7)
    phi = rng.standard_normal((ny, nz, nx))
    phi -= phi.mean()
    q_lo, q_hi = rng.standard_normal((2, nz, nx))
    b = O.laplacian(phi, grid, O.NEUMANN, q_lo, q_hi)
    got, removed = O.poisson_solve(b, grid, q_lo=q_lo, q_hi=q_hi)
    assert abs(removed) <= 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(got - phi)) <= 1e-11 * np.max(np.abs(phi))


# ---------------------------------------------------------------------------
# Inflow-outflow RK stage (Sec. 3's inflow-outflow configuration)
# ---------------------------------------------------------------------------

def _io_state(g, wl):
    nx, ny, nz = g[:3]
    u, v, w = synth.div_free_velocity(g, workload=wl, kmax=4)
    r = np.random.default_rng(wl)
    p = 0.1 * r.standard_normal((ny, nz, nx))
    Np = [0.5 * r.standard_normal((ny, nz, nx)) for _ in range(3)]
    Np[1][0] = 0.0
    return dict(u=u, v=v, w=w, p=p, N_prev=tuple(Np), t=0.0)


_NO_MARKERS = dict(X0=np.zeros((0, 3)), dV=np.zeros(0), kind=O.MOTION_STATIC, params=(0, 0, 0))


def test_advection_with_zero_wall_data_is_the_no_slip_form():
    g = _grid(16, 12, 8, Lx=1.0, Ly=1.5, Lz=0.8)
    nx, ny, nz = g[:3]
    u, v, w = synth.div_free_velocity(g, workload=5, kmax=5)
    z = np.zeros((nz, nx))
    ref = O.advection(u, v, w, g)
    got = O.advection(u, v, w, g, (0.0, z, z, z))
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))


def test_inout_stage_with_zero_data_is_the_no_slip_stage():
    """No inflow, a resting outlet (C = 0, zero outlet values): the
    inflow-outflow stage is the no-slip stage."""
    g = _grid(16, 12, 8, Lx=2 * math.pi, Ly=2.0, Lz=2 * math.pi)
    nx, ny, nz = g[:3]
    st = _io_state(g, 3)
    z = np.zeros((nz, nx))
    io = dict(v_in=0.0, c_out=0.0, u_out=z, v_out=z, w_out=z)
    ref, _ = O.rk_stage(st, _NO_MARKERS, 2, 1e-3, 1e-2, g)
    got, _ = O.rk_stage(st, _NO_MARKERS, 2, 1e-3, 1e-2, g, inout=io)
    for k in ("u", "v", "w", "p"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-12 * np.max(np.abs(ref[k])), k


def test_inout_stage_keeps_uniform_through_flow():
    """v = U everywhere (inlet, interior faces and outlet), u = w = 0, uniform
    pressure, C = U: a steady state of the stage, kept to rounding."""
    g = _grid(12, 10, 8, Lx=1.3, Ly=1.7, Lz=0.9)
    nx, ny, nz = g[:3]
    U = 0.8
    zf = np.zeros((ny, nz, nx))
    st = dict(u=zf.copy(), v=np.full((ny, nz, nx), U), w=zf.copy(), p=np.full((ny, nz, nx), 0.3),
              N_prev=(zf, zf, zf), t=0.0)
    z = np.zeros((nz, nx))
    io = dict(v_in=U, c_out=U, u_out=z, v_out=np.full((nz, nx), U), w_out=z)
    for stage in (1, 2, 3):
        new, info = O.rk_stage(st, _NO_MARKERS, stage, 2e-3, 1e-2, g, inout=io)
        assert np.max(np.abs(new["u"])) <= 1e-12 and np.max(np.abs(new["w"])) <= 1e-12
        assert np.max(np.abs(new["v"] - U)) <= 1e-12
        assert np.max(np.abs(new["p"] - 0.3)) <= 1e-12
        assert np.max(np.abs(new["inout"]["v_out"] - U)) <= 1e-12
        st, io = new, new["inout"]


def test_inout_stage_projects_onto_the_through_flow():
    """With inflow and an advected outlet the projected field is discretely
    divergence-free with the stage's wall faces, and the outlet carries out
    what the inlet brings in."""
    g = _grid(16, 12, 8, Lx=2 * math.pi, Ly=2.0, Lz=2 * math.pi)
    nx, ny, nz = g[:3]
    st = _io_state(g, 4)
    r = np.random.default_rng(4)
    io = dict(v_in=0.5, c_out=0.5, u_out=0.1 * r.standard_normal((nz, nx)),
              v_out=0.5 + 0.1 * r.standard_normal((nz, nx)), w_out=0.1 * r.standard_normal((nz, nx)))
    new, _ = O.rk_stage(st, _NO_MARKERS, 1, 1e-3, 1e-2, g, inout=io)
    vo = new["inout"]["v_out"]
    assert abs(vo.mean() - 0.5) <= 1e-14
    d = O.divergence(new["u"], new["v"], new["w"], g, 0.5, vo)
    assert np.max(np.abs(d)) <= 1e-10 * np.max(np.abs(new["v"])) / g[4]
    assert np.all(new["v"][0] == 0.5)


def test_outflow_update_closed_forms():
    """The outlet's first-order upwind step (Sec. 3's advective condition):
    with C = 0 the planes stay (up to the mass shift, here zero); with a
    Courant number of one over the distance to the last interior value
    (step C = hy/2 for u and w at the wall, step C = hy for v's face) the
    outlet takes exactly that value; the v shift restores mean = v_in."""
    g = _grid(8, 6, 4, Lx=1.0, Ly=1.2, Lz=0.8)
    nx, ny, nz, hx, hy, hz = g
    r = np.random.default_rng(11)
    u, v, w = (r.standard_normal((ny, nz, nx)) for _ in range(3))
    vo0 = r.standard_normal((nz, nx))
    vo0 += 0.3 - vo0.mean()
    io = dict(v_in=0.3, c_out=0.0, u_out=r.standard_normal((nz, nx)), v_out=vo0, w_out=r.standard_normal((nz, nx)))
    uo, vo, wo = O.outflow_update(io, u, v, w, g, 0.01)
    assert np.array_equal(uo, io["u_out"]) and np.array_equal(wo, io["w_out"])
    assert np.max(np.abs(vo - io["v_out"])) <= 1e-15
    io1 = dict(io, c_out=1.0)
    uo, _, wo = O.outflow_update(io1, u, v, w, g, 0.5 * hy)
    assert np.max(np.abs(uo - u[-1])) <= 1e-15 and np.max(np.abs(wo - w[-1])) <= 1e-15
    _, vo, _ = O.outflow_update(io1, u, v, w, g, hy)
    assert np.max(np.abs(vo - (v[-1] + (0.3 - v[-1].mean())))) <= 1e-14
    assert abs(vo.mean() - 0.3) <= 1e-15


def test_advection_with_wall_data_telescopes_to_the_wall_fluxes():
    """Conservative form: the x and z fluxes telescope over the periodic
    axes, the y fluxes to the two walls.  With inflow v_lo (u = w = 0 on
    that wall) and outlet values (u_hi, v_hi, w_hi), the grid sum of each
    component equals its net wall flux over hy: u and w carry
    avg(v_hi) * g through the outlet and nothing through the inflow wall; v
    carries (v on the cell centre)^2 from the first to the last cell row."""
    g = _grid(12, 10, 8, Lx=1.1, Ly=1.4, Lz=0.9)
    nx, ny, nz, hx, hy, hz = g
    r = np.random.default_rng(21)
    u, v, w = (r.standard_normal((ny, nz, nx)) for _ in range(3))
    v_lo = 0.4
    u_hi, v_hi, w_hi = (r.standard_normal((nz, nx)) for _ in range(3))
    Nu, Nv, Nw = O.advection(u, v, w, g, (v_lo, u_hi, v_hi, w_hi))
    vx = 0.5 * (v_hi + np.roll(v_hi, 1, 1))   # outlet v at the u points (x-faces)
    vz = 0.5 * (v_hi + np.roll(v_hi, 1, 0))   # ... at the w points (z-faces)
    assert abs(Nu.sum() - (vx * u_hi).sum() / hy) <= 1e-11 * np.abs(Nu).sum()
    assert abs(Nw.sum() - (vz * w_hi).sum() / hy) <= 1e-11 * np.abs(Nw).sum()
    vc_top = 0.5 * (v[ny - 1] + v_hi)
    vc_bot = 0.5 * (v_lo + v[1])
    assert abs(Nv.sum() - ((vc_top ** 2).sum() - (vc_bot ** 2).sum()) / hy) <= 1e-11 * np.abs(Nv).sum()
