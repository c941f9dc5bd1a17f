"""Helpers shared by the GPU tests (device transfer, tolerances, errors).

Every parity gate compares a GPU result x with the oracle's ref through
rel_err: the larger of the relative L2 error ||x - ref||_2 / ||ref||_2 and
the relative max-abs error ||x - ref||_inf / ||ref||_inf, so that an error
confined to a few points (one wall row of one plane) is not diluted by the
square root of the number of points.  Assertion messages print both."""

import math

import numpy as np

# Relative L2 tolerances against the FP64 oracle.
#   FP64 path: direct method, round-off only (accuracy target 1e-12).
#   FP32 path after refinement: 1e-6 (accuracy target); FP32 storage of the
#   result alone contributes ~6e-8.
TOL_FP64 = 1e-12
TOL_FP32 = 1e-6
# Interpolation / spreading in FP32: the weights are evaluated in FP32 from an
# FP64 offset, each of the <= 64 products rounds once and the sums are FP32
# (spreading adds atomics in any order).  Error bound ~ (support + log2 K)
# eps32 relative to the sum of magnitudes; 2e-6 relative L2 covers it.
TOL_IBM_FP32 = 2e-6
TOL_IBM_FP64 = 1e-13


def grid(nx, ny, nz, Lx=2 * math.pi, Ly=2.0, Lz=2 * math.pi):
    return (nx, ny, nz, Lx / nx, Ly / ny, Lz / nz)


def dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def host(t):
    return t.detach().double().cpu().numpy()


def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((x - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def rel_inf(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(x - ref).max(initial=0.0) / max(np.abs(ref).max(initial=0.0), 1e-300))


class RelErr(float):
    """max(relative L2, relative max-abs) error, printing both."""

    def __new__(cls, l2, inf):
        e = super().__new__(cls, max(l2, inf))
        e.l2, e.inf = l2, inf
        return e

    def __repr__(self):
        return "(l2 %.3g, max %.3g)" % (self.l2, self.inf)

    __str__ = __repr__


def rel_err(x, ref, inf_ratio=1.0):
    """max(relative L2, relative max-abs / inf_ratio): gates both norms, the
    max-abs one at inf_ratio times the tolerance."""
    l2, inf = rel_l2(x, ref), rel_inf(x, ref)
    return RelErr(l2, inf) if inf_ratio == 1.0 else _Scaled(l2, inf, inf_ratio)


class _Scaled(RelErr):
    def __new__(cls, l2, inf, ratio):
        obj = float.__new__(cls, max(l2, inf / ratio))
        obj.l2, obj.inf, obj.ratio = l2, inf, ratio
        return obj

    def __repr__(self):
        return "(l2 %.3g, max %.3g gated at %g x)" % (self.l2, self.inf, self.ratio)

    __str__ = __repr__


# Interpolation / spreading in FP32: a grid point sums up to hundreds of
# stencil contributions in an arbitrary (atomic) order, so the error at the
# densest points runs above the field's typical error; the max-abs error is
# gated at twice the L2 tolerance (measured: 2.1e-6 max, 7.8e-7 L2 for 48k
# markers at 96x64x96).
IBM_INF_RATIO = 2.0
