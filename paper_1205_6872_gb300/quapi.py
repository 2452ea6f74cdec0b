"""Thin ctypes binding of libquapi.so (C ABI in include/quapi.h).

Every function keeps the C entry point's name and only marshals arguments:
numpy arrays for host buffers, torch CUDA tensors (or raw integer device
addresses) for device buffers, torch streams for ``cuda_stream``.  All compute
runs in the library's CUDA kernels; if the library cannot be loaded every call
raises, there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libquapi.so")

QUAPI_OK = 0
QUAPI_ERR_ARG = 1
QUAPI_ERR_OOM = 2
QUAPI_ERR_CUDA = 3
QUAPI_ERR_TIMEOUT = 4
QUAPI_ERR_UNSUPPORTED = 5
STATUS_NAMES = {0: "QUAPI_OK", 1: "QUAPI_ERR_ARG", 2: "QUAPI_ERR_OOM", 3: "QUAPI_ERR_CUDA",
                4: "QUAPI_ERR_TIMEOUT", 5: "QUAPI_ERR_UNSUPPORTED"}

QUAPI_J_OHMIC_EXP = 0
QUAPI_J_SUPEROHMIC_GAUSS = 1
QUAPI_J_TABULATED = 2
QUAPI_FP64 = 64
QUAPI_FP32 = 32
QUAPI_DF64 = 48
QUAPI_ENDPOINT_STRANG = 0
QUAPI_ENDPOINT_INTERIOR = 1

JKIND = {"ohmic_exp": QUAPI_J_OHMIC_EXP, "superohmic_gauss": QUAPI_J_SUPEROHMIC_GAUSS,
         "tabulated": QUAPI_J_TABULATED}

EXPORTED = ("quapi_opts_init", "quapi_query_memory", "quapi_query_memory_opts", "quapi_setup", "quapi_setup_eta",
            "quapi_propagate", "quapi_propagate_device", "quapi_step_device",
            "quapi_propagate_batch", "quapi_get_eta", "quapi_get_propagator",
            "quapi_readout_static", "quapi_get_state", "quapi_set_state", "quapi_propagate_resume",
            "quapi_kernel_launches", "quapi_last_error", "quapi_destroy")


class quapi_spectral(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", ctypes.c_double), ("wc", ctypes.c_double),
                ("omega", ctypes.POINTER(ctypes.c_double)), ("values", ctypes.POINTER(ctypes.c_double)),
                ("n", ctypes.c_int)]


class quapi_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("endpoint_mode", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("tune", ctypes.c_int),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("hermitian", ctypes.c_int)]


class QuapiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libquapi.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libquapi.so not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        ctxp = ctypes.c_void_p
        sig = {
            "quapi_opts_init": (None, [ctypes.POINTER(quapi_opts)]),
            "quapi_query_memory": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_size_t),
                                                  ctypes.POINTER(ctypes.c_size_t)]),
            "quapi_query_memory_opts": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(quapi_opts),
                                                       ctypes.POINTER(ctypes.c_size_t),
                                                       ctypes.POINTER(ctypes.c_size_t)]),
            "quapi_setup": (ctypes.c_int, [dp, ctypes.c_int, dp, ctypes.POINTER(quapi_spectral),
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(quapi_opts), ctypes.POINTER(ctxp)]),
            "quapi_setup_eta": (ctypes.c_int, [dp, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int,
                                               ctypes.POINTER(quapi_opts), ctypes.POINTER(ctxp)]),
            "quapi_propagate": (ctypes.c_int, [ctxp, dp, i64p, ctypes.c_int, dp]),
            "quapi_propagate_device": (ctypes.c_int, [ctxp, vp, i64p, ctypes.c_int, vp]),
            "quapi_step_device": (ctypes.c_int, [ctxp, ctypes.c_int64, vp, vp, vp]),
            "quapi_propagate_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctxp),
                                                     ctypes.POINTER(dp), i64p, ctypes.POINTER(dp)]),
            "quapi_get_eta": (ctypes.c_int, [ctxp, dp]),
            "quapi_get_propagator": (ctypes.c_int, [ctxp, dp, dp]),
            "quapi_readout_static": (ctypes.c_int, [ctxp, ctypes.c_int64, vp, vp]),
            "quapi_get_state": (ctypes.c_int, [ctxp, i64p, vp, ctypes.POINTER(ctypes.c_size_t)]),
            "quapi_set_state": (ctypes.c_int, [ctxp, ctypes.c_int64, vp, ctypes.c_size_t]),
            "quapi_propagate_resume": (ctypes.c_int, [ctxp, i64p, ctypes.c_int, dp]),
            "quapi_kernel_launches": (ctypes.c_uint64, []),
            "quapi_last_error": (ctypes.c_char_p, [ctxp]),
            "quapi_destroy": (None, [ctxp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} complex values, got {a.size}")
    return a


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _check(status, ctx=None):
    if status != QUAPI_OK:
        msg = load().quapi_last_error(ctx)
        raise QuapiError(status, msg.decode() if msg else "")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def quapi_opts_init(precision=QUAPI_FP64, endpoint_mode=QUAPI_ENDPOINT_STRANG, cuda_stream=None,
                    tune=0, workspace=None, workspace_bytes=0, hermitian=0) -> quapi_opts:
    o = quapi_opts()
    load().quapi_opts_init(ctypes.byref(o))
    o.precision = int(precision)
    o.endpoint_mode = int(endpoint_mode)
    o.cuda_stream = _stream_handle(cuda_stream)
    o.tune = int(tune)
    o.workspace = _dev_ptr(workspace)
    o.workspace_bytes = int(workspace_bytes)
    o.hermitian = int(hermitian)
    return o


def quapi_query_memory(M, dkmax, precision=QUAPI_FP64):
    t, tot = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().quapi_query_memory(int(M), int(dkmax), int(precision), ctypes.byref(t), ctypes.byref(tot)))
    return t.value, tot.value


def quapi_query_memory_opts(M, dkmax, opts):
    """(tensor_bytes, total_bytes) for the precision and layout of opts (quapi_opts_init(...))."""
    t, tot = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().quapi_query_memory_opts(int(M), int(dkmax), ctypes.byref(opts), ctypes.byref(t),
                                          ctypes.byref(tot)))
    return t.value, tot.value


def quapi_setup(s, H, jkind, a, wc, beta, dt, dkmax, opts=None, omega=None, values=None):
    """Returns an opaque context handle (int); release it with quapi_destroy.
    jkind "tabulated": J given by the arrays omega (ascending, > 0) and values; a and wc unused."""
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    M = s.size
    Hc = _c128(H, M * M)
    J = quapi_spectral(JKIND.get(jkind, jkind) if isinstance(jkind, str) else int(jkind), float(a), float(wc))
    if omega is not None:
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        va = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
        if om.shape != va.shape:
            raise ValueError("omega and values must have the same length")
        J.omega, J.values, J.n = _dp(om), _dp(va), int(om.size)
    o = opts if opts is not None else quapi_opts_init()
    ctx = ctypes.c_void_p()
    _check(load().quapi_setup(_dp(s), M, _dp(Hc.view(np.float64)), ctypes.byref(J), float(beta), float(dt),
                              int(dkmax), ctypes.byref(o), ctypes.byref(ctx)))
    return ctx.value


def quapi_setup_eta(s, H, eta, dt, dkmax, opts=None):
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64))
    M = s.size
    Hc = _c128(H, M * M)
    e = _c128(eta, 4 * int(dkmax) + 3)
    o = opts if opts is not None else quapi_opts_init()
    ctx = ctypes.c_void_p()
    _check(load().quapi_setup_eta(_dp(s), M, _dp(Hc.view(np.float64)), _dp(e.view(np.float64)), float(dt),
                                  int(dkmax), ctypes.byref(o), ctypes.byref(ctx)))
    return ctx.value


def quapi_propagate(ctx, rho0, steps, M):
    """rho at the requested steps, shape (len(steps), M, M) complex128 (host)."""
    r0 = _c128(rho0, M * M)
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
    out = np.empty(st.size * M * M, dtype=np.complex128)
    _check(load().quapi_propagate(ctx, _dp(r0.view(np.float64)),
                                  st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), st.size,
                                  _dp(out.view(np.float64))), ctx)
    return out.reshape(st.size, M, M)


def quapi_propagate_device(ctx, rho0_dev, steps, rho_out_dev):
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
    _check(load().quapi_propagate_device(ctx, _dev_ptr(rho0_dev),
                                         st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), st.size,
                                         _dev_ptr(rho_out_dev)), ctx)


def quapi_step_device(ctx, n, A_in_dev, A_out_dev=None, rho_dev=None):
    _check(load().quapi_step_device(ctx, int(n), _dev_ptr(A_in_dev), _dev_ptr(A_out_dev), _dev_ptr(rho_dev)), ctx)


def quapi_propagate_batch(ctxs, rho0s, nsteps_each, M=2):
    n = len(ctxs)
    arr_ctx = (ctypes.c_void_p * n)(*ctxs)
    r0 = [_c128(r, M * M) for r in rho0s]
    outs = [np.empty(M * M, dtype=np.complex128) for _ in range(n)]
    arr_r0 = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(r.view(np.float64)) for r in r0])
    arr_out = (ctypes.POINTER(ctypes.c_double) * n)(*[_dp(o.view(np.float64)) for o in outs])
    ns = np.ascontiguousarray(np.asarray(nsteps_each, dtype=np.int64))
    _check(load().quapi_propagate_batch(n, arr_ctx, arr_r0, ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        arr_out))
    return [o.reshape(M, M) for o in outs]


def quapi_get_eta(ctx, dkmax):
    out = np.empty(4 * int(dkmax) + 3, dtype=np.complex128)
    _check(load().quapi_get_eta(ctx, _dp(out.view(np.float64))), ctx)
    return out


def quapi_get_propagator(ctx, M):
    U = np.empty(M * M, dtype=np.complex128)
    K = np.empty(M ** 4, dtype=np.complex128)
    _check(load().quapi_get_propagator(ctx, _dp(U.view(np.float64)), _dp(K.view(np.float64))), ctx)
    return U.reshape(M, M), K.reshape(M * M, M * M)


def quapi_readout_static(ctx, n, A_in_dev, rho_dev):
    """rho(t_n) from A_{n-1} into rho_dev, with the readout scratch in the library's fixed array."""
    _check(load().quapi_readout_static(ctx, int(n), _dev_ptr(A_in_dev), _dev_ptr(rho_dev)), ctx)


def quapi_get_state(ctx):
    """(n, bytes) of the context's kept tensor A_n, copied to host as a uint8 numpy array."""
    n = ctypes.c_int64()
    nb = ctypes.c_size_t(0)
    _check(load().quapi_get_state(ctx, ctypes.byref(n), None, ctypes.byref(nb)), ctx)
    buf = np.empty(nb.value, dtype=np.uint8)
    _check(load().quapi_get_state(ctx, ctypes.byref(n), buf.ctypes.data, ctypes.byref(nb)), ctx)
    return n.value, buf


def quapi_set_state(ctx, n, state):
    buf = np.ascontiguousarray(state).view(np.uint8)
    _check(load().quapi_set_state(ctx, int(n), buf.ctypes.data, buf.nbytes), ctx)


def quapi_propagate_resume(ctx, steps, M):
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
    out = np.empty(st.size * M * M, dtype=np.complex128)
    _check(load().quapi_propagate_resume(ctx, st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), st.size,
                                         _dp(out.view(np.float64))), ctx)
    return out.reshape(st.size, M, M)


def quapi_kernel_launches() -> int:
    return int(load().quapi_kernel_launches())


def quapi_last_error(ctx=None) -> str:
    m = load().quapi_last_error(ctx)
    return m.decode() if m else ""


def quapi_destroy(ctx):
    if ctx:
        load().quapi_destroy(ctx)
