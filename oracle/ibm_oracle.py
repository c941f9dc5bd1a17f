"""Plain FP64 CPU oracle for the immersed-boundary fractional-step hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only the tests, the smoke check and the benchmark's CPU-baseline leg may call
it.  It shares no code with the CUDA library (no FFT, no Thomas sweep, no
tables); it writes out the plain definition of each result in numpy FP64.

Paper: "A Python-based flow solver for numerical simulations using an
immersed boundary method on single GPUs" (arXiv 2406.19920).  Equation names
below follow the paper: Eq. 2a-2h is the RK-stage system of Sec. 2.1
(explicit estimate, interpolation, Lagrangian force, spreading, Helmholtz,
Poisson, projection, pressure update); Appendix A is the modified-wavenumber
derivation; Appendix B gives the pencil matrices with their boundary rows.

Grid and layout (shared convention with the library, restated here):
  * domain periodic in x and z, bounded by walls in y; spacings hx, hy, hz;
  * every field is an array of shape (ny, nz, nx) -- axis 0 is y, axis 1 is
    z, axis 2 is x (x fastest in memory);
  * p, phi and the Poisson right-hand side sit at cell centres
    ((i+1/2)hx, (j+1/2)hy, (k+1/2)hz);
  * u sits on x-faces (i hx, (j+1/2)hy, (k+1/2)hz), w on z-faces
    ((i+1/2)hx, (j+1/2)hy, k hz), v on y-faces ((i+1/2)hx, j hy, (k+1/2)hz);
    v plane j is face j; plane 0 is the bottom wall and the top wall face
    j = ny is not stored -- both wall faces carry v = 0 and the stored plane
    0 is ignored on input and written as 0 on output (no-slip walls; the
    inflow-outflow stage of rk_stage carries v_in and the outlet plane
    there instead).

Pins (tests/test_oracle_pins.py) tie every function to results fixed by the
mathematics: closed forms, dense brute-force solves, invariants and special
cases.  The paper prints no stage values, so the RK stage (rk_stage) is
pinned term by term, each by a case in which that term alone has a
closed-form effect on the stage's output:
  * a viscous eigenmode carried through a full stage (the alpha / beta
    split of Eq. 2a and 2e);
  * the history term -zeta N_prev on a divergence-free Helmholtz eigenmode;
  * the advection term -gamma N(u), by superposition against the history
    term (out(u) + out(-u) isolates it);
  * -(alpha+beta) G p with the projection and the pressure update of Eq.
    2g-2h, which cancel exactly for a y-only pressure mode;
  * the scheme's stability polynomial, projection to round-off, the
    Lagrangian force at the stage start time;
  * the inflow-outflow reductions.
marker_motion is pinned by the heave's values at quarter periods, its
period and its velocity as the derivative of its position.

Boundary kinds of a field along y ("field_bc"):
  NEUMANN         cell-centred, ghost x_{-1} = x_0 (Appendix B, Neumann rows
                  with A3 + A2 corners and homogeneous BC)
  CELL_DIRICHLET  cell-centred, ghost x_{-1} = -x_0 (Appendix B, alpha = 2,
                  A11 = A1 - A2): tangential velocity at a no-slip wall
  FACE_DIRICHLET  face-centred, unknowns on faces 1..ny-1, walls = 0
                  (Appendix B, alpha = 1): wall-normal velocity
"""

from __future__ import annotations

import numpy as np

NEUMANN = 0
CELL_DIRICHLET = 1
FACE_DIRICHLET = 2
PERIODIC = 3  # the triply periodic branch (Sec. 2.3.3, S2: y periodic as well)

ROMA3 = 0
PESKIN4 = 1

# Low-storage semi-implicit RK3 of Rai & Moin (1991), cited by the paper in
# Sec. 2.1 for alpha_n, beta_n, gamma_n, zeta_n (the paper does not print
# them).  alpha = beta splits the viscous term Crank-Nicolson style.
RK_ALPHA = (4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0)
RK_BETA = (4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0)
RK_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
RK_ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)


# ---------------------------------------------------------------------------
# Modified wavenumbers and eigen-bases (Appendix A, Appendix B)
# ---------------------------------------------------------------------------

def modified_wavenumber_sq(theta, h):
    """kappa'^2 = (2/h^2)(1 - cos(kappa h)) with theta = kappa h (Appendix A).

    This is the eigenvalue (with sign flipped) of the 3-point second
    difference on a Fourier mode; the same expression is the eigenvalue of
    the wall-bounded pencil matrices of Appendix B on their sine/cosine
    eigenvectors, with theta = pi m / n.
    """
    return (2.0 / (h * h)) * (1.0 - np.cos(theta))


def fourier_basis(n):
    """Orthonormal real Fourier basis of R^n and the angle of each column.

    Columns: constant, cos(2 pi m i/n) and sin(2 pi m i/n) for 0 < m < n/2,
    and the alternating vector when n is even.  Each column is an
    eigenvector of the periodic second difference with eigenvalue
    -(2/h^2)(1 - cos(2 pi m / n)) (Appendix A).
    """
    i = np.arange(n, dtype=np.float64)
    cols, thetas = [np.full(n, 1.0 / np.sqrt(n))], [0.0]
    for m in range(1, (n + 1) // 2):
        th = 2.0 * np.pi * m / n
        cols.append(np.sqrt(2.0 / n) * np.cos(th * i))
        thetas.append(th)
        cols.append(np.sqrt(2.0 / n) * np.sin(th * i))
        thetas.append(th)
    if n % 2 == 0:
        cols.append(np.cos(np.pi * i) / np.sqrt(n))
        thetas.append(np.pi)
    return np.stack(cols, axis=1), np.array(thetas)


def wall_basis(n, field_bc):
    """Orthonormal eigenvectors of the wall-normal pencil matrix (Appendix B).

    NEUMANN: cos(pi m (j+1/2)/n), m = 0..n-1  (A3 + A2 corner rows)
    CELL_DIRICHLET: sin(pi m (j+1/2)/n), m = 1..n  (A11 = A1 - A2, alpha=2)
    FACE_DIRICHLET: sin(pi m j/n) on faces j = 1..n-1, m = 1..n-1 (alpha=1)
    Angle theta = pi m / n in every case.  Returns (Q, theta) where Q has one
    row per stored plane (n rows; for FACE_DIRICHLET row 0 is the wall face
    and is identically zero, with n-1 columns).
    PERIODIC (no walls, the triply periodic branch): the Fourier basis.
    """
    if field_bc == PERIODIC:
        return fourier_basis(n)
    j = np.arange(n, dtype=np.float64)
    if field_bc == NEUMANN:
        m = np.arange(n, dtype=np.float64)
        Q = np.cos(np.pi * np.outer(j + 0.5, m) / n)
    elif field_bc == CELL_DIRICHLET:
        m = np.arange(1, n + 1, dtype=np.float64)
        Q = np.sin(np.pi * np.outer(j + 0.5, m) / n)
    elif field_bc == FACE_DIRICHLET:
        m = np.arange(1, n, dtype=np.float64)
        Q = np.sin(np.pi * np.outer(j, m) / n)
    else:
        raise ValueError("unknown field_bc")
    Q = Q / np.linalg.norm(Q, axis=0, keepdims=True)
    return Q, np.pi * m / n


def _to_modes(f, Qy, Qz, Qx):
    """Coefficients of f (ny, nz, nx) in the separable basis Qy x Qz x Qx."""
    ny, nz, nx = f.shape
    t = f @ Qx                                              # x-modes
    t = np.swapaxes(np.swapaxes(t, 1, 2) @ Qz, 1, 2)        # z-modes
    return (Qy.T @ t.reshape(ny, -1)).reshape(Qy.shape[1], nz, nx)


def _from_modes(c, Qy, Qz, Qx):
    """Inverse of _to_modes (the bases are orthonormal)."""
    nm, nz, nx = c.shape
    t = (Qy @ c.reshape(nm, -1)).reshape(Qy.shape[0], nz, nx)
    t = np.swapaxes(np.swapaxes(t, 1, 2) @ Qz.T, 1, 2)
    return t @ Qx.T


def _eigen_sum(grid, field_bc):
    """lambda_x + lambda_y + lambda_z >= 0 for every separable mode."""
    nx, ny, nz, hx, hy, hz = grid
    Qx, tx = fourier_basis(nx)
    Qz, tz = fourier_basis(nz)
    Qy, ty = wall_basis(ny, field_bc)
    lam = (modified_wavenumber_sq(ty, hy)[:, None, None]
           + modified_wavenumber_sq(tz, hz)[None, :, None]
           + modified_wavenumber_sq(tx, hx)[None, None, :])
    return (Qy, Qz, Qx), lam


# ---------------------------------------------------------------------------
# Linear solves: Eq. 2e (Helmholtz) and Eq. 2f (Poisson), Sec. 2.3.3
# ---------------------------------------------------------------------------

def poisson_solve(b, grid, nullspace="mean", ybc=NEUMANN, q_lo=None, q_hi=None):
    """Solve L_h phi = b - mean(b) on the staggered grid (Eq. 2f, S2 / S2.1).

    L_h is the 7-point Laplacian (second-order central differences, Sec. 2.1)
    with periodic x, z and homogeneous Neumann y (Appendix B).  The system is
    singular on constants; the right-hand side is made compatible by
    removing its mean (the paper does not say how; this is the reading used
    throughout) and the free constant is fixed by
      nullspace="mean": mean(phi) = 0 (the triply periodic branch's rule,
                         Sec. 2.3.3, S2), or
      nullspace="pin":  the x-z mean of phi on the first interior plane is 0
                         (Sec. 2.3.3, S2.1: phi_hat(x_b + h/2, 0, 0) = 0).
    Method: exact eigen-decomposition with dense orthonormal bases.
    ybc=PERIODIC is the triply periodic branch (Sec. 2.3.3, S2: Fourier
    along all three axes, the divide diagonal, mean(phi) = 0).
    q_lo, q_hi ([nz][nx] or None): inhomogeneous Neumann data dphi/dy at the
    walls (Appendix B, the right-hand sides of the first and last pencil
    rows): L_h phi with those ghosts equals b, i.e. the homogeneous system
    with b minus the data's share of the operator.
    Returns (phi, removed_mean).
    """
    b = np.asarray(b, dtype=np.float64)
    if q_lo is not None or q_hi is not None:
        if ybc != NEUMANN:
            raise ValueError("wall data needs the wall-bounded branch")
        b = b - laplacian(np.zeros_like(b), grid, NEUMANN, q_lo, q_hi)
    mean_b = b.mean()
    rhs = b - mean_b
    if ybc not in (NEUMANN, PERIODIC):
        raise ValueError("ybc must be NEUMANN or PERIODIC")
    if ybc == PERIODIC and nullspace != "mean":
        raise ValueError("the triply periodic branch fixes mean(phi) = 0")
    Q, lam = _eigen_sum(grid, ybc)
    c = _to_modes(rhs, *Q)
    lam = lam.copy()
    lam[0, 0, 0] = 1.0
    c = -c / lam
    c[0, 0, 0] = 0.0
    phi = _from_modes(c, *Q)
    if nullspace == "pin":
        phi = phi - phi[0].mean()
    elif nullspace != "mean":
        raise ValueError("nullspace must be 'mean' or 'pin'")
    return phi, mean_b


def helmholtz_solve(r, grid, c, field_bc, g_lo=None, g_hi=None):
    """Solve (I - c L_h) u = r (Eq. 2e, S1 / S1.1).

    Eq. 2e reads  lap u* - (Re / (beta dt)) u* = -(Re / (beta dt)) RHS, which
    is (I - c L_h) u* = RHS with c = beta dt / Re.  field_bc selects the
    wall rows of Appendix B (PERIODIC: no walls).  For FACE_DIRICHLET plane 0
    (the wall face) of the input is ignored and of the output is 0, or g_lo.
    g_lo, g_hi ([nz][nx] or None): inhomogeneous wall data (the wall value
    for the Dirichlet kinds, du/dy at the wall for NEUMANN); L_h then uses
    the ghosts of laplacian(..., g_lo, g_hi), which is the homogeneous system
    with r plus c times the data's share of the operator.
    """
    r = np.asarray(r, dtype=np.float64)
    wall = g_lo is not None or g_hi is not None
    if wall:
        if field_bc == PERIODIC:
            raise ValueError("wall data needs the wall-bounded branch")
        r = r + c * laplacian(np.zeros_like(r), grid, field_bc, g_lo, g_hi)
    Q, lam = _eigen_sum(grid, field_bc)
    coeff = _to_modes(r, *Q) / (1.0 + c * lam)
    u = _from_modes(coeff, *Q)
    if wall and field_bc == FACE_DIRICHLET and g_lo is not None:
        u[0] = g_lo
    return u


# ---------------------------------------------------------------------------
# Finite-difference operators (Sec. 2.1: second-order central, ghost points)
# ---------------------------------------------------------------------------

def _ypad(f, field_bc, hy=1.0, g_lo=None, g_hi=None):
    """f with one ghost plane below and above along y.

    Wall data (Appendix B; 0 where None): NEUMANN g = df/dy at the wall,
    ghost f_{-1} = f_0 - hy g_lo, f_ny = f_{ny-1} + hy g_hi;
    CELL_DIRICHLET g = the wall value, ghost 2 g - f (the wall halfway);
    FACE_DIRICHLET g = the wall-face values (face 0 is the stored plane 0,
    face ny the ghost above)."""
    ny = f.shape[0]
    zero = np.zeros(f.shape[1:])
    gl = zero if g_lo is None else np.asarray(g_lo, dtype=np.float64)
    gh = zero if g_hi is None else np.asarray(g_hi, dtype=np.float64)
    out = np.empty((ny + 2,) + f.shape[1:])
    out[1:-1] = f
    if field_bc == NEUMANN:
        out[0], out[-1] = f[0] - hy * gl, f[-1] + hy * gh
    elif field_bc == CELL_DIRICHLET:
        out[0], out[-1] = 2.0 * gl - f[0], 2.0 * gh - f[-1]
    elif field_bc == FACE_DIRICHLET:
        out[1] = gl           # stored bottom wall face
        out[0] = 0.0          # never used by interior faces
        out[-1] = gh          # top wall face j = ny
    elif field_bc == PERIODIC:
        out[0], out[-1] = f[-1], f[0]
    else:
        raise ValueError("unknown field_bc")
    return out


def laplacian(f, grid, field_bc, g_lo=None, g_hi=None):
    """7-point L_h f: sum over axes of (f_{+1} - 2 f + f_{-1}) / h^2.

    Periodic in x and z; y uses the ghost rule of field_bc with the wall
    data g_lo, g_hi (see _ypad; None is 0).  For FACE_DIRICHLET the wall
    plane of f is the face value g_lo and that of the result is 0.
    """
    nx, ny, nz, hx, hy, hz = grid
    f = np.asarray(f, dtype=np.float64)
    if field_bc == FACE_DIRICHLET:
        f = f.copy()
        f[0] = 0.0 if g_lo is None else g_lo
    g = _ypad(f, field_bc, hy, g_lo, g_hi)
    out = (np.roll(f, -1, 2) - 2.0 * f + np.roll(f, 1, 2)) / (hx * hx)
    out += (np.roll(f, -1, 1) - 2.0 * f + np.roll(f, 1, 1)) / (hz * hz)
    out += (g[2:] - 2.0 * f + g[:-2]) / (hy * hy)
    if field_bc == FACE_DIRICHLET:
        out[0] = 0.0
    return out


def divergence(u, v, w, grid, v_lo=0.0, v_hi=None):
    """Cell-centred D(u, v, w) (E2, Sec. 2.3.1).  The wall faces carry v_lo
    (bottom, a scalar) and v_hi (top, a [nz][nx] plane or None for 0):
    0 on both for no-slip walls."""
    nx, ny, nz, hx, hy, hz = grid
    top = np.zeros((1, nz, nx)) if v_hi is None else np.asarray(v_hi, dtype=np.float64)[None]
    vv = np.concatenate([np.full((1, nz, nx), float(v_lo)), v[1:], top])
    return ((np.roll(u, -1, 2) - u) / hx
            + (vv[1:] - vv[:-1]) / hy
            + (np.roll(w, -1, 1) - w) / hz)


def gradient(phi, grid):
    """Face-centred G phi; the v-component is 0 on the wall face (plane 0)."""
    nx, ny, nz, hx, hy, hz = grid
    gu = (phi - np.roll(phi, 1, 2)) / hx
    gw = (phi - np.roll(phi, 1, 1)) / hz
    gv = np.zeros_like(phi)
    gv[1:] = (phi[1:] - phi[:-1]) / hy
    return gu, gv, gw


def advection(u, v, w, grid, wall=None):
    """Divergence-form MAC advection N = div(u u) on the staggered grid.

    The paper discretises (u . grad) u with second-order central differences
    (Sec. 2.1) without printing the staggered formula; this is the standard
    conservative form with two-point averages, which equals the advective
    form to O(h^2) for a discretely divergence-free field and conserves
    momentum and kinetic energy.  No-slip walls carry v = 0, so fluxes
    through them vanish.  wall = (v_lo, u_hi, v_hi, w_hi) gives an inflow
    face (v = v_lo, u = w = 0) at y = 0 and outlet values at y = Ly (u, w at
    the wall, v on the face): the wall values of u and w enter the y-fluxes
    through their ghosts 2 g - u.  Returns (Nu, Nv, Nw) on the u, v, w
    positions.
    """
    nx, ny, nz, hx, hy, hz = grid
    if wall is not None:
        return _advection_wall(u, v, w, grid, wall)
    xm = lambda f: np.roll(f, 1, 2)     # f[..., i-1]
    xp = lambda f: np.roll(f, -1, 2)    # f[..., i+1]
    zm = lambda f: np.roll(f, 1, 1)
    zp = lambda f: np.roll(f, -1, 1)
    zero = np.zeros((1, nz, nx))
    # v with both wall faces explicit: vf[j] = face j, j = 0..ny
    vf = np.concatenate([zero, v[1:], zero])

    # --- x-momentum at x-face (i, j, k) ---
    uc = 0.5 * (u + xp(u))                            # u at cell centres
    tx = (uc * uc - xm(uc) * xm(uc)) / hx
    # edge (x-face i, y-face j'), j' = 0..ny
    v_e = 0.5 * (vf + xm(vf))
    u_pad = np.concatenate([zero, u, zero])          # values irrelevant at walls
    u_e = 0.5 * (u_pad[:-1] + u_pad[1:])
    fy = v_e * u_e
    ty = (fy[1:] - fy[:-1]) / hy
    # edge (x-face i, z-face k)
    w_e = 0.5 * (w + xm(w))
    u_ez = 0.5 * (u + zm(u))
    fz = w_e * u_ez
    tz = (zp(fz) - fz) / hz
    Nu = tx + ty + tz

    # --- y-momentum at y-face (i, j, k), j = 1..ny-1 ---
    vc = 0.5 * (vf[:-1] + vf[1:])                    # v at cell centres
    ty_v = np.zeros((ny, nz, nx))
    ty_v[1:] = (vc[1:] * vc[1:] - vc[:-1] * vc[:-1]) / hy
    # edge (x-face i', y-face j)
    u_ey = np.zeros((ny, nz, nx))
    u_ey[1:] = 0.5 * (u[1:] + u[:-1])
    v_ex = 0.5 * (vf[:-1] + xm(vf[:-1]))
    fx = u_ey * v_ex
    tx_v = (xp(fx) - fx) / hx
    # edge (z-face k', y-face j)
    w_ey = np.zeros((ny, nz, nx))
    w_ey[1:] = 0.5 * (w[1:] + w[:-1])
    v_ez = 0.5 * (vf[:-1] + zm(vf[:-1]))
    fz_v = w_ey * v_ez
    tz_v = (zp(fz_v) - fz_v) / hz
    Nv = tx_v + ty_v + tz_v
    Nv[0] = 0.0

    # --- z-momentum at z-face (i, j, k) ---
    wc = 0.5 * (w + zp(w))
    tz_w = (wc * wc - zm(wc) * zm(wc)) / hz
    u_ez2 = 0.5 * (u + zm(u))                        # u at z-face k, x-face i'
    w_ex = 0.5 * (w + xm(w))
    fx_w = u_ez2 * w_ex
    tx_w = (xp(fx_w) - fx_w) / hx
    v_ez2 = 0.5 * (vf + zm(vf))                      # v at y-face j', z-face k
    w_pad = np.concatenate([zero, w, zero])
    w_ey2 = 0.5 * (w_pad[:-1] + w_pad[1:])
    fy_w = v_ez2 * w_ey2
    ty_w = (fy_w[1:] - fy_w[:-1]) / hy
    Nw = tx_w + ty_w + tz_w
    return Nu, Nv, Nw


def _advection_wall(u, v, w, grid, wall):
    """advection() with the inflow / outlet wall data (see there)."""
    nx, ny, nz, hx, hy, hz = grid
    v_lo, u_hi, v_hi, w_hi = wall
    xm = lambda f: np.roll(f, 1, 2)
    xp = lambda f: np.roll(f, -1, 2)
    zm = lambda f: np.roll(f, 1, 1)
    zp = lambda f: np.roll(f, -1, 1)
    vf = np.concatenate([np.full((1, nz, nx), float(v_lo)), v[1:], np.asarray(v_hi, dtype=np.float64)[None]])
    # u, w with their ghost planes (wall values 0 at the inlet, u_hi / w_hi at the outlet)
    u_pad = np.concatenate([-u[:1], u, 2.0 * np.asarray(u_hi)[None] - u[-1:]])
    w_pad = np.concatenate([-w[:1], w, 2.0 * np.asarray(w_hi)[None] - w[-1:]])

    uc = 0.5 * (u + xp(u))
    tx = (uc * uc - xm(uc) * xm(uc)) / hx
    v_e = 0.5 * (vf + xm(vf))
    u_e = 0.5 * (u_pad[:-1] + u_pad[1:])             # u at the y-faces 0 .. ny (walls: the wall value)
    fy = v_e * u_e
    ty = (fy[1:] - fy[:-1]) / hy
    w_e = 0.5 * (w + xm(w))
    u_ez = 0.5 * (u + zm(u))
    fz = w_e * u_ez
    tz = (zp(fz) - fz) / hz
    Nu = tx + ty + tz

    vc = 0.5 * (vf[:-1] + vf[1:])
    ty_v = np.zeros((ny, nz, nx))
    ty_v[1:] = (vc[1:] * vc[1:] - vc[:-1] * vc[:-1]) / hy
    u_ey = np.zeros((ny, nz, nx))
    u_ey[1:] = 0.5 * (u[1:] + u[:-1])
    v_ex = 0.5 * (vf[:-1] + xm(vf[:-1]))
    fx = u_ey * v_ex
    tx_v = (xp(fx) - fx) / hx
    w_ey = np.zeros((ny, nz, nx))
    w_ey[1:] = 0.5 * (w[1:] + w[:-1])
    v_ez = 0.5 * (vf[:-1] + zm(vf[:-1]))
    fz_v = w_ey * v_ez
    tz_v = (zp(fz_v) - fz_v) / hz
    Nv = tx_v + ty_v + tz_v
    Nv[0] = 0.0

    wc = 0.5 * (w + zp(w))
    tz_w = (wc * wc - zm(wc) * zm(wc)) / hz
    u_ez2 = 0.5 * (u + zm(u))
    w_ex = 0.5 * (w + xm(w))
    fx_w = u_ez2 * w_ex
    tx_w = (xp(fx_w) - fx_w) / hx
    v_ez2 = 0.5 * (vf + zm(vf))
    w_e2 = 0.5 * (w_pad[:-1] + w_pad[1:])
    fy_w = v_ez2 * w_e2
    ty_w = (fy_w[1:] - fy_w[:-1]) / hy
    Nw = tz_w + tx_w + ty_w
    return Nu, Nv, Nw


# ---------------------------------------------------------------------------
# Regularised delta kernels and the Lagrangian operations (Eq. 2b-2d, L1)
# ---------------------------------------------------------------------------

def delta_1d(r, kernel=ROMA3):
    """One-dimensional regularised delta phi(r), r in grid units.

    The paper cites Peskin and Roma et al. (Sec. 2.1) without writing the
    kernel out.  ROMA3 is the three-point kernel of Roma, Peskin & Berger
    (1999) used by Uhlmann's method; PESKIN4 is Peskin's (2002) four-point
    cosine-free kernel.
    """
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    if kernel == ROMA3:
        m1 = a <= 0.5
        m2 = (a > 0.5) & (a <= 1.5)
        out[m1] = (1.0 + np.sqrt(1.0 - 3.0 * a[m1] ** 2)) / 3.0
        t = 1.0 - a[m2]
        out[m2] = (5.0 - 3.0 * a[m2] - np.sqrt(np.maximum(0.0, 1.0 - 3.0 * t * t))) / 6.0
    elif kernel == PESKIN4:
        m1 = a <= 1.0
        m2 = (a > 1.0) & (a <= 2.0)
        out[m1] = (3.0 - 2.0 * a[m1] + np.sqrt(1.0 + 4.0 * a[m1] - 4.0 * a[m1] ** 2)) / 8.0
        out[m2] = (5.0 - 2.0 * a[m2] - np.sqrt(np.maximum(0.0, -7.0 + 12.0 * a[m2] - 4.0 * a[m2] ** 2))) / 8.0
    else:
        raise ValueError("unknown kernel")
    return out


# staggered origin of each velocity component, in grid units (x, y, z)
_ORIGIN = {0: (0.0, 0.5, 0.5), 1: (0.5, 0.0, 0.5), 2: (0.5, 0.5, 0.0)}


def _stencil(X, grid, comp, kernel):
    """Support indices and weights of every marker for one component.

    Returns (jy, kz, ix, wgt, valid): arrays of shape (N, S, S, S), S = 3
    (ROMA3) or 4 (PESKIN4).  Periodic wrap in x and z; along y the support
    points outside the stored unknowns (below plane 0 / above plane ny-1,
    and the wall face 0 of v) are marked invalid and dropped.
    """
    nx, ny, nz, hx, hy, hz = grid
    ox, oy, oz = _ORIGIN[comp]
    X = np.asarray(X, dtype=np.float64)
    s = np.stack([X[:, 0] / hx - ox, X[:, 1] / hy - oy, X[:, 2] / hz - oz], axis=1)
    if kernel == ROMA3:
        base = np.floor(s + 0.5) - 1.0
        S = 3
    else:
        base = np.floor(s) - 1.0
        S = 4
    off = np.arange(S, dtype=np.float64)
    idx = base[:, :, None] + off[None, None, :]            # (N, 3, S)
    w1 = delta_1d(s[:, :, None] - idx, kernel)             # (N, 3, S)
    ix = np.mod(idx[:, 0].astype(np.int64), nx)
    jy = idx[:, 1].astype(np.int64)
    kz = np.mod(idx[:, 2].astype(np.int64), nz)
    wgt = (w1[:, 1][:, :, None, None] * w1[:, 2][:, None, :, None]
           * w1[:, 0][:, None, None, :])                    # (N, Sy, Sz, Sx)
    lo = 1 if comp == 1 else 0
    vy = (jy >= lo) & (jy <= ny - 1)
    JY = np.broadcast_to(jy[:, :, None, None], wgt.shape)
    KZ = np.broadcast_to(kz[:, None, :, None], wgt.shape)
    IX = np.broadcast_to(ix[:, None, None, :], wgt.shape)
    valid = np.broadcast_to(vy[:, :, None, None], wgt.shape)
    return JY, KZ, IX, wgt, valid


def clear_of_walls(X, grid, kernel=ROMA3):
    """The wall rule for markers: True where the support of delta_h along y,
    |y - Y| < (S/2) hy (S = 3 for ROMA3, 4 for PESKIN4), stays between the
    walls, i.e. (S/2) hy <= Y <= Ly - (S/2) hy.  Such a marker's stencil
    touches stored unknowns only (v's wall face gets zero weight).  The
    paper states no rule for markers nearer a wall; a closer marker would
    need values beyond the wall, and it is treated as invalid input."""
    nx, ny, nz, hx, hy, hz = grid
    r = 1.5 if kernel == ROMA3 else 2.0
    s = np.asarray(X, dtype=np.float64).reshape(-1, 3)[:, 1] / hy
    return (s >= r) & (s <= ny - r)


def _require_clear(X, grid, kernel):
    ok = clear_of_walls(X, grid, kernel)
    if not np.all(ok):
        raise ValueError("%d marker(s) within the delta kernel's support of a wall" % int((~ok).sum()))


def interp(X, u, v, w, grid, kernel=ROMA3):
    """U(X_eta) = sum_xi u(x_xi) delta_h(x_xi - X_eta) h^3  (Eq. 2b).

    delta_h is the tensor product of phi((x - X)/h) / h per axis, so the h^3
    cancels and U is a weighted sum with weights phi phi phi.
    Returns U of shape (N, 3).  Markers must be clear of the walls
    (clear_of_walls); otherwise ValueError.
    """
    _require_clear(X, grid, kernel)
    out = np.zeros((len(X), 3))
    for comp, f in enumerate((u, v, w)):
        JY, KZ, IX, wgt, valid = _stencil(X, grid, comp, kernel)
        vals = np.where(valid, f[np.where(valid, JY, 0), KZ, IX], 0.0)
        out[:, comp] = (vals * wgt).sum(axis=(1, 2, 3))
    return out


def spread(X, F, dV, grid, kernel=ROMA3):
    """f(x_xi) = sum_eta F(X_eta) delta_h(x_xi - X_eta) dV_eta  (Eq. 2d).

    delta_h = phi phi phi / (hx hy hz).  Accumulation runs in marker order in
    FP64 (deterministic).  Returns (fu, fv, fw).  Markers must be clear of
    the walls (clear_of_walls); otherwise ValueError.
    """
    nx, ny, nz, hx, hy, hz = grid
    _require_clear(X, grid, kernel)
    X = np.asarray(X, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    dV = np.asarray(dV, dtype=np.float64)
    outs = []
    for comp in range(3):
        f = np.zeros((ny, nz, nx))
        JY, KZ, IX, wgt, valid = _stencil(X, grid, comp, kernel)
        amp = (F[:, comp] * dV / (hx * hy * hz))[:, None, None, None] * wgt
        m = valid.reshape(-1)
        np.add.at(f, (JY.reshape(-1)[m], KZ.reshape(-1)[m], IX.reshape(-1)[m]),
                  amp.reshape(-1)[m])
        outs.append(f)
    return tuple(outs)


# ---------------------------------------------------------------------------
# Prescribed marker motion (L2) and one RK stage (Eq. 2a-2h)
# ---------------------------------------------------------------------------

MOTION_STATIC = 0
MOTION_TRANSLATE = 1
MOTION_HEAVE = 2


def marker_motion(X0, t, kind, params):
    """Positions and surface velocity of markers under prescribed motion (L2).

    STATIC:     X = X0, U^d = 0
    TRANSLATE:  X = X0 + U t, U^d = U         params = (Ux, Uy, Uz)
    HEAVE:      X = X0 + (0, A sin(2 pi t / T), 0),
                U^d = (0, A (2 pi / T) cos(2 pi t / T), 0)   params = (A, T)
    """
    X0 = np.asarray(X0, dtype=np.float64)
    X = X0.copy()
    Ud = np.zeros_like(X0)
    if kind == MOTION_TRANSLATE:
        U = np.asarray(params[:3], dtype=np.float64)
        X = X0 + U[None, :] * t
        Ud[:] = U[None, :]
    elif kind == MOTION_HEAVE:
        A, T = params[0], params[1]
        X[:, 1] = X0[:, 1] + A * np.sin(2.0 * np.pi * t / T)
        Ud[:, 1] = A * (2.0 * np.pi / T) * np.cos(2.0 * np.pi * t / T)
    elif kind != MOTION_STATIC:
        raise ValueError("unknown motion kind")
    return X, Ud


def outflow_update(inout, u, v, w, grid, step):
    """The outlet condition d phi/dt + C d phi/dy = 0 (Sec. 3, inflow-outflow
    configuration) advanced over one stage step (alpha + beta) dt by
    first-order upwinding from the last interior value (the distance to it
    is hy/2 for u, w at the wall, hy for v's outlet face).  The paper leaves
    the discretisation to a reference; this is the reading used here.  The
    outlet v is then shifted by a constant so that the outflow through the
    top face equals the inflow through the bottom one (global mass balance,
    which keeps the Poisson right-hand side compatible).  Returns new
    (u_out, v_out, w_out)."""
    nx, ny, nz, hx, hy, hz = grid
    C = inout["c_out"]
    uo = inout["u_out"] - step * C * (inout["u_out"] - u[-1]) / (0.5 * hy)
    wo = inout["w_out"] - step * C * (inout["w_out"] - w[-1]) / (0.5 * hy)
    vo = inout["v_out"] - step * C * (inout["v_out"] - v[-1]) / hy
    vo = vo + (inout["v_in"] - vo.mean())
    return uo, vo, wo


def rk_stage(state, markers, stage, dt, nu, grid, kernel=ROMA3, inout=None):
    """One stage n = stage (1, 2, 3) of the RK system, Eq. 2a-2h.

    state: dict with u, v, w, p (ny, nz, nx) and N_prev = (Nu, Nv, Nw), the
           advection term of the previous stage ([(u.grad)u]^{n-2}), and t,
           the time at the start of this stage.
    markers: dict with X0 (N,3), dV (N,), motion kind and params; the stage
           forces with X, U^d evaluated at the stage start time.
    inout: None for no-slip walls; else the inflow-outflow configuration
           (Sec. 3): dict with v_in (the wall-normal inflow through y = 0,
           where u = w = 0), c_out (outlet advection speed) and the outlet
           values u_out, v_out, w_out ([nz][nx]; u, w at the wall y = Ly, v
           on its face).  The outlet values are advanced first
           (outflow_update) and, with the inflow, are the wall data of the
           whole stage: the explicit terms, the Helmholtz solves (Appendix B
           boundary rows), the divergence and the projection all see them.
           The new values are returned in new_state["inout"].
    Re^{-1} = nu.  Returns (new_state, info) where info holds U^e, F, phi.
    """
    n = stage - 1
    a, b, g, z = RK_ALPHA[n], RK_BETA[n], RK_GAMMA[n], RK_ZETA[n]
    ab = a + b
    u, v, w, p = state["u"], state["v"], state["w"], state["p"]
    bcs = (CELL_DIRICHLET, FACE_DIRICHLET, CELL_DIRICHLET)
    if inout is None:
        glo, ghi, v_lo, v_hi, wall = (None,) * 3, (None,) * 3, 0.0, None, None
    else:
        nxg, nyg, nzg = grid[:3]
        uo, vo, wo = outflow_update(inout, u, v, w, grid, ab * dt)
        zero = np.zeros((nzg, nxg))
        glo = (zero, np.full((nzg, nxg), float(inout["v_in"])), zero)
        ghi = (uo, vo, wo)
        v_lo, v_hi, wall = inout["v_in"], vo, (inout["v_in"], uo, vo, wo)
        v = v.copy()
        v[0] = inout["v_in"]
    vel = (u, v, w)
    N = advection(u, v, w, grid, wall)
    Np = state["N_prev"]
    G = gradient(p, grid)
    # Eq. 2a: explicit estimate
    ue = []
    for c in range(3):
        e = vel[c] + dt * (ab * nu * laplacian(vel[c], grid, bcs[c], glo[c], ghi[c])
                           - ab * G[c] - g * N[c] - z * Np[c])
        if c == 1:
            e[0] = v_lo
        ue.append(e)
    # Eq. 2b-2d: interpolation, Lagrangian force, spreading
    X, Ud = marker_motion(markers["X0"], state["t"], markers["kind"], markers["params"])
    Ue = interp(X, *ue, grid, kernel)
    F = (Ud - Ue) / dt
    f = spread(X, F, markers["dV"], grid, kernel)
    # Eq. 2e: implicit viscous Helmholtz, (I - c L) u* = RHS, c = beta dt nu
    cH = b * dt * nu
    us = []
    for c in range(3):
        rhs = ue[c] - cH * laplacian(vel[c], grid, bcs[c], glo[c], ghi[c]) + dt * f[c]
        if inout is None:
            us.append(helmholtz_solve(rhs, grid, cH, bcs[c]))
        else:
            us.append(helmholtz_solve(rhs, grid, cH, bcs[c], glo[c], ghi[c]))
    # Eq. 2f: Poisson for the pseudo-pressure
    rhs_phi = divergence(*us, grid, v_lo, v_hi) / (ab * dt)
    phi, _ = poisson_solve(rhs_phi, grid)
    # Eq. 2g: projection
    Gphi = gradient(phi, grid)
    un = [us[c] - ab * dt * Gphi[c] for c in range(3)]
    un[1][0] = v_lo
    # Eq. 2h: pressure update
    pn = p + phi - cH * laplacian(phi, grid, NEUMANN)
    new = dict(u=un[0], v=un[1], w=un[2], p=pn, N_prev=N, t=state["t"] + ab * dt)
    if inout is not None:
        new["inout"] = dict(inout, u_out=uo, v_out=vo, w_out=wo)
    return new, dict(Ue=Ue, F=F, phi=phi, rhs_phi=rhs_phi, ustar=us)


# ---------------------------------------------------------------------------
# Error metrics
# ---------------------------------------------------------------------------

def rel_l2(x, ref):
    """||x - ref||_2 / ||ref||_2 in FP64."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def normalised_residual(phi, b, grid):
    """||b - L phi||_inf / (||L||_inf ||phi||_inf + ||b||_inf), b mean-free."""
    nx, ny, nz, hx, hy, hz = grid
    b0 = b - b.mean()
    r = b0 - laplacian(phi, grid, NEUMANN)
    normL = 4.0 / hx ** 2 + 4.0 / hy ** 2 + 4.0 / hz ** 2
    return float(np.abs(r).max() / (normL * np.abs(phi).max() + np.abs(b0).max()))
