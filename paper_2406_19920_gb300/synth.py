"""Seeded synthetic inputs for the solver, the tests and the benchmark.

This module only generates inputs (right-hand sides, velocity fields, marker
sets).  It holds none of the solver's arithmetic: no Laplacian inverse, no
interpolation or spreading, no projection.  Both the CUDA path and the CPU
reference receive the arrays it returns.  Every field has shape (ny, nz, nx)
(x fastest), FP64 on the host; callers cast to the precision they run.

Workload shapes follow the paper's use cases: a sphere resolved by markers
spaced about one cell apart (Sec. 3, Sec. 2.1) and a heaving flat plate
standing in for the bio-inspired external flows of Sec. 5.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

# Seed = 1000 * workload id + stream id
STREAM_RHS, STREAM_NOISE, STREAM_FORCE, STREAM_VEL, STREAM_ARRIVAL, STREAM_GRID, STREAM_MARKERS = range(7)


def seed_of(workload: int, stream: int) -> int:
    return 1000 * workload + stream


def rng(workload: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(seed_of(workload, stream))


def grid(nx: int, ny: int, nz: int, Lx: float = 2 * math.pi, Ly: float = 2.0,
         Lz: float = 2 * math.pi):
    """(nx, ny, nz, hx, hy, hz) for a box [0,Lx) x [0,Ly] x [0,Lz)."""
    return (nx, ny, nz, Lx / nx, Ly / ny, Lz / nz)


# ---------------------------------------------------------------------------
# Right-hand sides
# ---------------------------------------------------------------------------

def _mode_1d_periodic(n, m, kind):
    i = np.arange(n, dtype=np.float64)
    return np.cos(2 * np.pi * m * i / n) if kind == 0 else np.sin(2 * np.pi * m * i / n)


def rhs_eigen_sum(nx, ny, nz, workload=0, n_modes=4, noise=1e-3):
    """Sum of n_modes separable grid modes (cosine/sine in x and z, cosine
    about cell centres in y) with N(0,1) amplitudes and indices drawn in the
    lowest third of each axis, plus white noise of std `noise`; mean removed.

    Returns (rhs, modes) with modes = [(amp, (mx, kindx), my, (mz, kindz))].
    """
    r = rng(workload, STREAM_RHS)
    f = np.zeros((ny, nz, nx))
    modes = []
    j = np.arange(ny, dtype=np.float64)
    for _ in range(n_modes):
        mx = int(r.integers(0, max(1, nx // 6) + 1))
        my = int(r.integers(0, max(1, ny // 3)))
        mz = int(r.integers(0, max(1, nz // 6) + 1))
        kx, kz = int(r.integers(0, 2)), int(r.integers(0, 2))
        if mx == 0:
            kx = 0
        if mz == 0:
            kz = 0
        amp = float(r.standard_normal())
        fx = _mode_1d_periodic(nx, mx, kx)
        fz = _mode_1d_periodic(nz, mz, kz)
        fy = np.cos(np.pi * my * (j + 0.5) / ny)
        f += amp * fy[:, None, None] * fz[None, :, None] * fx[None, None, :]
        modes.append((amp, (mx, kx), my, (mz, kz)))
    f += noise * rng(workload, STREAM_NOISE).standard_normal(f.shape)
    return f - f.mean(), modes


def rhs_lowpass_noise(nx, ny, nz, Lx=2 * math.pi, Ly=2.0, Lz=2 * math.pi,
                      kmax=32.0, workload=1, stream=STREAM_RHS):
    """Zero-mean N(0,1) white noise, low-pass filtered to physical |k| <= kmax.

    Wavenumbers: kx = 2 pi m / Lx, kz = 2 pi m / Lz (periodic axes) and
    ky = pi m / Ly (cosine series between the walls).  The filter is a plain
    spectral mask applied with library transforms (input shaping only).
    """
    f = rng(workload, stream).standard_normal((ny, nz, nx))
    c = sfft.dct(f, type=2, axis=0, norm="ortho")
    c = np.fft.rfft(c, axis=2)
    c = np.fft.fft(c, axis=1)
    kx = 2 * np.pi * np.fft.rfftfreq(nx, d=1.0 / nx) / Lx
    kz = 2 * np.pi * np.fft.fftfreq(nz, d=1.0 / nz) / Lz
    ky = np.pi * np.arange(ny) / Ly
    K2 = ky[:, None, None] ** 2 + kz[None, :, None] ** 2 + kx[None, None, :] ** 2
    c[K2 > kmax * kmax] = 0.0
    c = np.fft.ifft(c, axis=1)
    c = np.fft.irfft(c, n=nx, axis=2)
    f = sfft.idct(c.real, type=2, axis=0, norm="ortho")
    f = f - f.mean()
    return f / np.sqrt(np.mean(f * f))


def white_noise(nx, ny, nz, workload, stream):
    return rng(workload, stream).standard_normal((ny, nz, nx))


# ---------------------------------------------------------------------------
# Velocity fields
# ---------------------------------------------------------------------------

def _filtered_periodic_noise(shape, kmax, exponent, r):
    """Periodic noise with spectral amplitude |k|^exponent for 0 < |k| <= kmax
    (integer wavenumbers of the index grid)."""
    ny, nz, nx = shape
    c = np.fft.rfftn(r.standard_normal(shape))
    ky = np.fft.fftfreq(ny, 1.0 / ny)[:, None, None]
    kz = np.fft.fftfreq(nz, 1.0 / nz)[None, :, None]
    kx = np.fft.rfftfreq(nx, 1.0 / nx)[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.where((k > 0) & (k <= kmax), np.power(np.maximum(k, 1.0), exponent), 0.0)
    return np.fft.irfftn(c * amp, s=shape, axes=(0, 1, 2))


def div_free_velocity(g, workload=1, kmax=16.0, slope=-5.0 / 3.0, rms=1.0):
    """Random velocity (u, v, w) that is discretely divergence-free on the
    staggered grid, with no flow through the walls.

    Built as the discrete curl of an edge-centred vector potential A whose
    spectrum gives a velocity energy spectrum ~ k^slope for k <= kmax; A is
    multiplied by sin^2(pi y / Ly) so it vanishes with its slope at both
    walls.  Ax, Az live on edges at y = j hy (j = 0..ny), Ay at y = (j+1/2)hy.
    """
    nx, ny, nz, hx, hy, hz = g
    Ly = ny * hy
    r = rng(workload, STREAM_VEL)
    # |u_hat| ~ k^(slope/2 - 1) in 3-D; A ~ u / k
    expo = slope / 2.0 - 2.0
    shape_e = (ny + 1, nz, nx)
    env_e = np.sin(np.pi * np.arange(ny + 1) * hy / Ly)[:, None, None] ** 2
    env_c = np.sin(np.pi * (np.arange(ny) + 0.5) * hy / Ly)[:, None, None] ** 2
    Ax = _filtered_periodic_noise(shape_e, kmax, expo, r)[: ny + 1] * env_e
    Az = _filtered_periodic_noise(shape_e, kmax, expo, r)[: ny + 1] * env_e
    Ay = _filtered_periodic_noise((ny, nz, nx), kmax, expo, r) * env_c
    Ax[0] = Ax[ny] = 0.0
    Az[0] = Az[ny] = 0.0
    xp = lambda f: np.roll(f, -1, 2)
    zp = lambda f: np.roll(f, -1, 1)
    u = (Az[1:] - Az[:-1]) / hy - (zp(Ay) - Ay) / hz
    v = (zp(Ax[:ny]) - Ax[:ny]) / hz - (xp(Az[:ny]) - Az[:ny]) / hx
    v[0] = 0.0
    w = (xp(Ay) - Ay) / hx - (Ax[1:] - Ax[:-1]) / hy
    s = math.sqrt(np.mean(u * u + v * v + w * w) / 3.0)
    return u * (rms / s), v * (rms / s), w * (rms / s)


# ---------------------------------------------------------------------------
# Lagrangian marker sets
# ---------------------------------------------------------------------------

def fibonacci_sphere(n, radius, centre, h):
    """n markers on a sphere, z_i = 1 - 2(i+1/2)/n with golden-angle azimuth.

    Returns (X (n,3), dV (n,)) with dV = (4 pi R^2 / n) h, the surface
    element times one cell width (the paper leaves dV to the user).
    """
    i = np.arange(n, dtype=np.float64)
    zc = 1.0 - 2.0 * (i + 0.5) / n
    rad = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    ga = math.pi * (3.0 - math.sqrt(5.0))
    th = ga * i
    X = np.stack([np.asarray(centre[0]) + radius * rad * np.cos(th),
                  np.asarray(centre[1]) + radius * zc,
                  np.asarray(centre[2]) + radius * rad * np.sin(th)], axis=1)
    dV = np.full(n, 4.0 * math.pi * radius * radius / n * h)
    return X, dV


def flat_plate(n_chord, n_span, chord, span, centre, h):
    """Lattice of n_chord x n_span markers on a plate normal to y.

    Chord along x, span along z, centred at `centre`.  dV = (area / n) h.
    """
    xs = (np.arange(n_chord) + 0.5) / n_chord * chord - 0.5 * chord
    zs = (np.arange(n_span) + 0.5) / n_span * span - 0.5 * span
    Xg, Zg = np.meshgrid(xs, zs, indexing="ij")
    X = np.stack([centre[0] + Xg.ravel(), np.full(Xg.size, float(centre[1])),
                  centre[2] + Zg.ravel()], axis=1)
    dV = np.full(X.shape[0], chord * span / X.shape[0] * h)
    return X, dV


def marker_forces(n, workload=0):
    return rng(workload, STREAM_FORCE).standard_normal((n, 3))
