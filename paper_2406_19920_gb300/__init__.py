"""GB300 (sm_103a) hot path of the immersed-boundary fractional-step solver.

Thin Python binding over libibm.so (C ABI in include/ibm.h).  The functions
below carry the C names and only marshal arguments: torch tensors (device
memory) become raw pointers, the current CUDA stream becomes a handle.  All
arithmetic runs in the library's CUDA kernels.  There is no CPU fallback:
importing a function raises if the library has not been built.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libibm.so")

IBM_OK, IBM_PENDING = 0, 1
IBM_ERR_ARG, IBM_ERR_OOM, IBM_ERR_CUDA, IBM_ERR_TIMEOUT, IBM_ERR_BUSY, IBM_ERR_UNSUPPORTED, IBM_ERR_CANCELLED = \
    -1, -2, -3, -4, -5, -6, -7
IBM_BC_PXZ_WALL_Y, IBM_BC_TRIPLY_PERIODIC = 1, 2
IBM_FP64, IBM_FP32_REFINED = 0, 1
IBM_FIELD_CELL_NEUMANN, IBM_FIELD_CELL_DIRICHLET, IBM_FIELD_FACE_DIRICHLET, IBM_FIELD_PERIODIC = 0, 1, 2, 3
IBM_DELTA_ROMA3, IBM_DELTA_PESKIN4 = 0, 1
IBM_SPREAD_ATOMIC, IBM_SPREAD_GATHER, IBM_SPREAD_ATOMIC_DIRECT = 0, 1, 2
IBM_MOTION_STATIC, IBM_MOTION_TRANSLATE, IBM_MOTION_HEAVE = 0, 1, 2
IBM_SELFTEST_TENSOR_MEMORY, IBM_SELFTEST_BULK_COPY = 0, 1
IBM_REQ_POISSON, IBM_REQ_HELMHOLTZ, IBM_REQ_SUBSTEP = 0, 1, 2
IBM_DATA_HOST_FP64, IBM_DATA_DEVICE = 0, 1


class IbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libibm error %d: %s" % (code, msg))
        self.code = code


IBM_K_COUNT = 11


class ibm_info(ctypes.Structure):
    _fields_ = [("rel_residual", ctypes.c_double), ("removed_mean", ctypes.c_double),
                ("div_max", ctypes.c_double), ("div_before", ctypes.c_double),
                ("t_ms", ctypes.c_double), ("refine_iters", ctypes.c_int), ("reserved", ctypes.c_int),
                ("phase_ms", ctypes.c_double * IBM_K_COUNT)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("reserved", "phase_ms")}
        d["phase_ms"] = {k: self.phase_ms[i] for i, k in enumerate(KERNEL_KINDS)}
        return d


class ibm_state(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("Nu", ctypes.c_void_p), ("Nv", ctypes.c_void_p), ("Nw", ctypes.c_void_p), ("t", ctypes.c_double)]


class ibm_markers(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("X0", ctypes.c_void_p), ("dV", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("Ud", ctypes.c_void_p), ("F", ctypes.c_void_p), ("motion", ctypes.c_int),
                ("params", ctypes.c_double * 4)]


class ibm_inout(ctypes.Structure):
    _fields_ = [("v_in", ctypes.c_double), ("c_out", ctypes.c_double), ("u_out", ctypes.c_void_p),
                ("v_out", ctypes.c_void_p), ("w_out", ctypes.c_void_p)]


class ibm_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double * 3), ("precision", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("c", ctypes.c_double), ("field_bc", ctypes.c_int),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("n_markers", ctypes.c_int), ("X0", ctypes.c_void_p), ("dV", ctypes.c_void_p),
                ("motion", ctypes.c_int), ("params", ctypes.c_double * 4),
                ("dt", ctypes.c_double), ("nu", ctypes.c_double), ("rk_stage", ctypes.c_int),
                ("data", ctypes.c_int)]


class ibm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("queue_ms", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("removed_mean", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIG = {
    "ibm_plan_create": (_I, [_I, _I, _I, _I, ctypes.POINTER(_D), _I, _I, ctypes.POINTER(_P)]),
    "ibm_plan_destroy": (_I, [_P]),
    "ibm_plan_set_delta": (_I, [_P, _I]),
    "ibm_plan_set_spread": (_I, [_P, _I]),
    "ibm_plan_workspace_bytes": (ctypes.c_size_t, [_P]),
    "ibm_plan_check": (_I, [_P]),
    "ibm_selftest_timeout": (_I, [_P, _I, _D, _P]),
    "ibm_plan_profile": (_I, [_P, _I]),
    "ibm_plan_profile_read": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "ibm_poisson_solve": (_I, [_P, _P, _P, _P, ctypes.POINTER(ibm_info)]),
    "ibm_helmholtz_solve": (_I, [_P, _D, _I, _P, _P, _P, ctypes.POINTER(ibm_info)]),
    "ibm_poisson_solve_bc": (_I, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(ibm_info)]),
    "ibm_helmholtz_solve_bc": (_I, [_P, _D, _I, _P, _P, _P, _P, _P, ctypes.POINTER(ibm_info)]),
    "ibm_poisson_solve_noalloc": (_I, [_I, _I, _I, ctypes.POINTER(_D), _I, _P, _P, ctypes.POINTER(_I), _P]),
    "ibm_interp": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "ibm_spread": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "ibm_substep": (_I, [_P, ctypes.POINTER(ibm_state), _I, _D, _D, ctypes.POINTER(ibm_markers), _P,
                         ctypes.POINTER(ibm_info)]),
    "ibm_substep_inout": (_I, [_P, ctypes.POINTER(ibm_state), ctypes.POINTER(ibm_inout), _I, _D, _D,
                               ctypes.POINTER(ibm_markers), _P, ctypes.POINTER(ibm_info)]),
    "ibm_batch_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_D), _I, _I, ctypes.POINTER(_P)]),
    "ibm_batch_destroy": (_I, [_P]),
    "ibm_batch_poisson": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    "ibm_batch_substep": (_I, [_P, ctypes.POINTER(ibm_state), ctypes.POINTER(ibm_markers), _I, _D, _D, _P]),
    "ibm_server_create": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_P)]),
    "ibm_server_destroy": (_I, [_P]),
    "ibm_submit": (_I, [_P, ctypes.POINTER(ibm_request), ctypes.POINTER(ctypes.c_uint64)]),
    "ibm_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(ibm_result)]),
    "ibm_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(ibm_result)]),
    "ibm_cancel": (_I, [_P, ctypes.c_uint64]),
    "ibm_last_error": (ctypes.c_char_p, []),
    "ibm_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libibm.so (raises ImportError when it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libibm.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                              "g.build()\"`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise IbmError(rc, lib().ibm_last_error().decode())
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _field(t, dtype):
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError("field must be a contiguous CUDA tensor of %s, got %s %s contiguous=%s"
                         % (dtype, t.device, t.dtype, t.is_contiguous()))
    return t.data_ptr()


# ---------------------------------------------------------------------------
# C names
# ---------------------------------------------------------------------------

def ibm_plan_create(nx, ny, nz, h, precision=IBM_FP32_REFINED, refine_iters=1, bc=IBM_BC_PXZ_WALL_Y):
    out = _P()
    hh = (_D * 3)(*[float(x) for x in h])
    _check(lib().ibm_plan_create(nx, ny, nz, bc, hh, precision, refine_iters, ctypes.byref(out)))
    return out.value


def ibm_plan_destroy(plan):
    return _check(lib().ibm_plan_destroy(plan))


def ibm_plan_set_delta(plan, kernel):
    return _check(lib().ibm_plan_set_delta(plan, kernel))


def ibm_plan_set_spread(plan, mode):
    return _check(lib().ibm_plan_set_spread(plan, mode))


def ibm_plan_check(plan):
    return _check(lib().ibm_plan_check(plan))


def ibm_plan_workspace_bytes(plan):
    return int(lib().ibm_plan_workspace_bytes(plan))


KERNEL_KINDS = ("forward", "pencil", "inverse", "residual", "explicit", "motion", "interp", "spread",
                "divergence", "project", "outflow")


def ibm_plan_profile(plan, enable=True):
    return _check(lib().ibm_plan_profile(plan, 1 if enable else 0))


def ibm_plan_profile_read(plan):
    """{kind: (total_ms, launches)} accumulated since the last read."""
    n = len(KERNEL_KINDS)
    ms = (_D * n)()
    cnt = (_I * n)()
    _check(lib().ibm_plan_profile_read(plan, n, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def ibm_poisson_solve(plan, rhs, phi, stream=None, info=False):
    inf = ibm_info() if info else None
    _check(lib().ibm_poisson_solve(plan, _ptr(rhs), _ptr(phi), _stream(stream),
                                   ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def ibm_poisson_solve_noalloc(nx, ny, nz, h, refine_iters, rhs, phi, stream=None, status=None):
    """FP32 Poisson solve whose workspace is the library's static device
    scratch (no device allocation; see include/ibm.h).  status: None, or a
    ctypes.c_int that receives the solve's device error word (valid once
    the stream has finished the call)."""
    hh = (_D * 3)(*[float(x) for x in h])
    return _check(lib().ibm_poisson_solve_noalloc(nx, ny, nz, hh, refine_iters, _ptr(rhs), _ptr(phi),
                                                  ctypes.byref(status) if status is not None else None,
                                                  _stream(stream)))


def ibm_helmholtz_solve(plan, c, field_bc, rhs, u, stream=None, info=False):
    inf = ibm_info() if info else None
    _check(lib().ibm_helmholtz_solve(plan, float(c), field_bc, _ptr(rhs), _ptr(u), _stream(stream),
                                     ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def ibm_poisson_solve_bc(plan, rhs, phi, q_lo=None, q_hi=None, stream=None, info=False):
    """Poisson solve with dphi/dy = q_lo, q_hi ([nz][nx] planes or None) at the walls."""
    inf = ibm_info() if info else None
    _check(lib().ibm_poisson_solve_bc(plan, _ptr(rhs), _ptr(phi), _ptr(q_lo), _ptr(q_hi), _stream(stream),
                                      ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def ibm_helmholtz_solve_bc(plan, c, field_bc, rhs, u, g_lo=None, g_hi=None, stream=None, info=False):
    """Helmholtz solve with wall data g_lo, g_hi ([nz][nx] planes or None)."""
    inf = ibm_info() if info else None
    _check(lib().ibm_helmholtz_solve_bc(plan, float(c), field_bc, _ptr(rhs), _ptr(u), _ptr(g_lo), _ptr(g_hi),
                                        _stream(stream), ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def ibm_interp(plan, n, X, u, v, w, U, stream=None):
    return _check(lib().ibm_interp(plan, n, _ptr(X), _ptr(u), _ptr(v), _ptr(w), _ptr(U), _stream(stream)))


def ibm_spread(plan, n, X, F, dV, fu, fv, fw, stream=None):
    return _check(lib().ibm_spread(plan, n, _ptr(X), _ptr(F), _ptr(dV), _ptr(fu), _ptr(fv), _ptr(fw),
                                   _stream(stream)))


def ibm_substep(plan, state, rk_stage, dt, nu, markers, stream=None, info=False):
    """state: ibm_state (device pointers), markers: ibm_markers."""
    inf = ibm_info() if info else None
    _check(lib().ibm_substep(plan, ctypes.byref(state), rk_stage, float(dt), float(nu), ctypes.byref(markers),
                             _stream(stream), ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def ibm_substep_inout(plan, state, inout, rk_stage, dt, nu, markers, stream=None, info=False):
    """As ibm_substep with inflow-outflow walls; inout: ibm_inout (outlet
    planes as device pointers, updated in place)."""
    inf = ibm_info() if info else None
    _check(lib().ibm_substep_inout(plan, ctypes.byref(state), ctypes.byref(inout), rk_stage, float(dt), float(nu),
                                   ctypes.byref(markers), _stream(stream),
                                   ctypes.byref(inf) if inf is not None else None))
    return inf.as_dict() if inf is not None else None


def ibm_selftest_timeout(plan, limit_ms, stream=None, path=None):
    """Runs one bounded wait that cannot complete (path: IBM_SELFTEST_TENSOR_MEMORY,
    the default, or IBM_SELFTEST_BULK_COPY); see include/ibm.h."""
    path = IBM_SELFTEST_TENSOR_MEMORY if path is None else path
    return _check(lib().ibm_selftest_timeout(plan, int(path), float(limit_ms), _stream(stream)))


def ibm_batch_create(dims, hs, precision=IBM_FP32_REFINED, refine_iters=1):
    n = len(dims)
    d = (_I * (3 * n))(*[int(v) for t in dims for v in t])
    h = (_D * (3 * n))(*[float(v) for t in hs for v in t])
    out = _P()
    _check(lib().ibm_batch_create(n, d, h, precision, refine_iters, ctypes.byref(out)))
    return out.value


def ibm_batch_destroy(batch):
    return _check(lib().ibm_batch_destroy(batch))


def ibm_batch_poisson(batch, rhs_list, phi_list, stream=None):
    n = len(rhs_list)
    r = (_P * n)(*[_ptr(t) for t in rhs_list])
    p = (_P * n)(*[_ptr(t) for t in phi_list])
    return _check(lib().ibm_batch_poisson(batch, r, p, _stream(stream)))


def ibm_batch_substep(batch, states, markers, rk_stage, dt, nu, stream=None):
    """One RK stage of every instance (states: list of ibm_state, markers:
    list of ibm_markers or None); the states' t are advanced in place."""
    n = len(states)
    S = (ibm_state * n)(*states)
    M = (ibm_markers * n)(*markers) if markers is not None else None
    _check(lib().ibm_batch_substep(batch, S, M, int(rk_stage), float(dt), float(nu), _stream(stream)))
    for i, st in enumerate(states):
        st.t = S[i].t


def ibm_server_create(hbm_budget_bytes, n_streams=4, max_queue=4096):
    out = _P()
    _check(lib().ibm_server_create(int(hbm_budget_bytes), n_streams, max_queue, ctypes.byref(out)))
    return out.value


def ibm_server_destroy(server):
    return _check(lib().ibm_server_destroy(server))


def ibm_submit(server, req):
    t = ctypes.c_uint64()
    rc = lib().ibm_submit(server, ctypes.byref(req), ctypes.byref(t))
    if rc == IBM_ERR_BUSY:
        return None
    _check(rc)
    return t.value


def ibm_poll(server, ticket):
    res = ibm_result()
    rc = lib().ibm_poll(server, ticket, ctypes.byref(res))
    return rc, res


def ibm_wait(server, ticket, timeout_s=60.0):
    res = ibm_result()
    rc = lib().ibm_wait(server, ticket, float(timeout_s), ctypes.byref(res))
    return rc, res


def ibm_cancel(server, ticket):
    return lib().ibm_cancel(server, ticket)


def ibm_last_error():
    return lib().ibm_last_error().decode()


def ibm_version():
    return lib().ibm_version().decode()
