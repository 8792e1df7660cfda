"""Thin ctypes binding of libzm.so (include/zm.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module converts
arguments (numpy arrays, torch tensors on CPU or GPU, or raw integer addresses) to pointers and
raises ZMError on a non-zero status.  If the shared library has not been built the first call
raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ZM_OK = 0
ZM_ERR_INVALID = -1
ZM_ERR_NOMEM = -2
ZM_ERR_CUDA = -3
ZM_ERR_TIMEOUT = -4
ZM_ERR_UNSUPPORTED = -5
ZM_ERR_NONFINITE = -6
ZM_ERR_BUSY = -7

ZM_ORDER_LOW = 0
ZM_ORDER_MEDIUM = 1
ZM_ORDER_HIGH = 2
ZM_PREC_FP64 = 0x000
ZM_PREC_FP32C = 0x100
ZM_PREC_DF64 = 0x200

ZM_K_GEOMETRY, ZM_K_BR, ZM_K_REDUCE, ZM_K_VORT, ZM_K_FFT, ZM_K_COUNT = range(6)
KERNEL_NAMES = ["geometry", "br", "reduce", "vorticity", "fft"]


class ZMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class zm_mesh(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int32), ("n2", ctypes.c_int32), ("L1", ctypes.c_double),
                ("L2", ctypes.c_double), ("periodic", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("iterations", "steps", "pairs", "completed", "failed",
                                               "queued", "running", "peak_running", "bytes_in_use",
                                               "peak_bytes")] + [("busy_s", ctypes.c_double)]


ZM_REQ_QUEUED, ZM_REQ_RUNNING, ZM_REQ_DONE, ZM_REQ_FAILED = 0, 1, 2, 3


class zm_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * ZM_K_COUNT), ("launches", ctypes.c_int64 * ZM_K_COUNT),
                ("pairs", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None
VP = ctypes.c_void_p


def lib_path() -> str:
    """libzm.so, or the checked build libzm_checked.so when ZM_LIB=checked."""
    return _build.LIB_CHECKED if os.environ.get("ZM_LIB") == "checked" else _build.LIB


def load():
    """Load libzm.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise ZMError(ZM_ERR_CUDA, f"libzm.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        I, D = ctypes.c_int, ctypes.c_double
        sig = {
            "zm_create": (I, [ctypes.POINTER(zm_mesh), D, D, D, D, I, ctypes.POINTER(VP)]),
            "zm_set_stream": (I, [VP, VP]),
            "zm_set_state": (I, [VP, VP, VP]),
            "zm_get_state": (I, [VP, VP, VP]),
            "zm_velocity": (I, [VP, VP, VP, VP, VP]),
            "zm_step": (I, [VP, D, I]),
            "zm_sync": (I, [VP]),
            "zm_destroy": (None, [VP]),
            "zm_error_string": (ctypes.c_char_p, [I]),
            "zm_last_error": (ctypes.c_char_p, []),
            "zm_set_profiling": (I, [VP, I]),
            "zm_get_profile": (I, [VP, ctypes.POINTER(zm_profile)]),
            "zm_reset_profile": (I, [VP]),
            "zm_check_finite": (I, [VP]),
            "zm_measure_peak": (I, [I, ctypes.POINTER(D)]),
            "zm_wait_selftest": (I, [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(D)]),
            "zm_wait_poll_limit": (ctypes.c_int64, []),
            "zm_checked_build": (I, []),
            "zm_set_tile_shape": (I, [VP, ctypes.c_int32, ctypes.c_int32]),
            "zm_get_tile_shape": (I, [VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
            "zm_bounds_status": (I, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
            "zm_br_velocity_noalloc": (I, [ctypes.c_int32, VP, VP, D, VP, VP, VP]),
            "zm_batch_create": (I, [ctypes.c_int32, ctypes.POINTER(zm_mesh), ctypes.POINTER(D), D, D,
                                    ctypes.POINTER(D), ctypes.POINTER(VP)]),
            "zm_batch_set_stream": (I, [VP, VP]),
            "zm_batch_set_state": (I, [VP, ctypes.c_int32, VP, VP]),
            "zm_batch_get_state": (I, [VP, ctypes.c_int32, VP, VP]),
            "zm_batch_velocity": (I, [VP]),
            "zm_batch_get_velocity": (I, [VP, ctypes.c_int32, VP, VP]),
            "zm_batch_step": (I, [VP, D, ctypes.c_int32]),
            "zm_batch_sync": (I, [VP]),
            "zm_batch_set_chunk": (I, [VP, ctypes.c_int32]),
            "zm_batch_autotune": (I, [VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_float)]),
            "zm_autotune": (I, [VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]),
            "zm_autotune_tiles": (I, [VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
            "zm_batch_set_tile_shape": (I, [VP, ctypes.c_int32, ctypes.c_int32]),
            "zm_batch_get_tile_shape": (I, [VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
            "zm_batch_autotune_tiles": (I, [VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_float)]),
            "zm_set_cutoff": (I, [VP, D]),
            "zm_set_far_path": (I, [VP, ctypes.c_int32]),
            "zm_get_far_path": (I, [VP, ctypes.POINTER(ctypes.c_int32)]),
            "zm_batch_set_far_path": (I, [VP, ctypes.c_int32]),
            "zm_batch_get_far_path": (I, [VP, ctypes.POINTER(ctypes.c_int32)]),
            "zm_batch_set_cutoff": (I, [VP, ctypes.c_int32, D]),
            "zm_batch_info": (I, [VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
            "zm_batch_set_profiling": (I, [VP, I]),
            "zm_batch_get_profile": (I, [VP, ctypes.POINTER(zm_profile)]),
            "zm_batch_destroy": (None, [VP]),
            "zm_server_create": (I, [ctypes.c_size_t, ctypes.c_int32, D, D, ctypes.POINTER(VP)]),
            "zm_server_submit": (I, [VP, ctypes.POINTER(zm_mesh), D, D, D, ctypes.c_int32, VP, VP,
                                     ctypes.POINTER(ctypes.c_int64)]),
            "zm_server_poll": (I, [VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]),
            "zm_server_request_bytes": (I, [ctypes.POINTER(zm_mesh), ctypes.POINTER(ctypes.c_size_t)]),
            "zm_server_wait": (I, [VP, ctypes.c_int64, D]),
            "zm_server_result": (I, [VP, ctypes.c_int64, VP, VP, ctypes.POINTER(D), ctypes.POINTER(D)]),
            "zm_server_cancel": (I, [VP, ctypes.c_int64]),
            "zm_server_get_stats": (I, [VP, ctypes.POINTER(ServerStats)]),
            "zm_server_set_policy": (I, [VP, ctypes.c_int32, ctypes.c_int64]),
            "zm_server_destroy": (None, [VP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(code):
    if code != ZM_OK:
        lib = load()
        raise ZMError(code, f"{lib.zm_error_string(code).decode()}: {lib.zm_last_error().decode()}")


def ptr(x):
    """Address of a float64 contiguous buffer: numpy array, torch tensor, int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ZMError(ZM_ERR_INVALID, "numpy buffers must be C-contiguous float64")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ZMError(ZM_ERR_INVALID, "torch buffers must be contiguous float64")
        return x.data_ptr()
    raise ZMError(ZM_ERR_INVALID, f"unsupported buffer type {type(x)}")


# ---- the C ABI, one function per entry point ------------------------------------------------

def zm_create(n1, n2=None, L1=1.0, L2=1.0, periodic=True, atwood=0.5, g=1.0, mu=0.0, delta=None,
              order=ZM_ORDER_HIGH):
    lib = load()
    n2 = n1 if n2 is None else n2
    if delta is None:
        delta = 0.1 * L1 / n1
    m = zm_mesh(int(n1), int(n2), float(L1), float(L2), int(bool(periodic)))
    h = VP()
    _check(lib.zm_create(ctypes.byref(m), float(atwood), float(g), float(mu), float(delta), int(order),
                         ctypes.byref(h)))
    return h


def zm_set_stream(h, stream):
    _check(load().zm_set_stream(h, stream))


def zm_set_state(h, z, w):
    _check(load().zm_set_state(h, ptr(z), ptr(w)))


def zm_get_state(h, z, w):
    _check(load().zm_get_state(h, ptr(z), ptr(w)))


def zm_velocity(h, z, w, u, wdot=None):
    _check(load().zm_velocity(h, ptr(z), ptr(w), ptr(u), ptr(wdot)))


def zm_step(h, dt, nsteps):
    _check(load().zm_step(h, float(dt), int(nsteps)))


def zm_sync(h):
    _check(load().zm_sync(h))


def zm_destroy(h):
    if h:
        load().zm_destroy(h)


def zm_set_profiling(h, on):
    _check(load().zm_set_profiling(h, int(bool(on))))


def zm_get_profile(h):
    p = zm_profile()
    _check(load().zm_get_profile(h, ctypes.byref(p)))
    return {"ms": {KERNEL_NAMES[k]: p.ms[k] for k in range(ZM_K_COUNT)},
            "launches": {KERNEL_NAMES[k]: int(p.launches[k]) for k in range(ZM_K_COUNT)},
            "pairs": int(p.pairs)}


def zm_reset_profile(h):
    _check(load().zm_reset_profile(h))


def zm_check_finite(h):
    return load().zm_check_finite(h)


PEAK_FP32, PEAK_FP64, PEAK_RSQRT, PEAK_FP32X2, PEAK_MIXED = 0, 1, 2, 3, 4


def zm_measure_peak(kind):
    v = ctypes.c_double()
    _check(load().zm_measure_peak(int(kind), ctypes.byref(v)))
    return v.value


def zm_wait_selftest(max_polls, arrive):
    """Run the bounded device-side wait once: returns (status code, kernel ms) without raising,
    so that ZM_ERR_TIMEOUT (nothing arrived, the wait gave up) can be checked."""
    ms = ctypes.c_double()
    rc = load().zm_wait_selftest(int(max_polls), int(arrive), ctypes.byref(ms))
    return rc, ms.value


def zm_wait_poll_limit():
    return int(load().zm_wait_poll_limit())


def _numel(x):
    if isinstance(x, np.ndarray):
        return x.size
    if hasattr(x, "numel"):
        return int(x.numel())
    return None  # a raw address: the caller vouches for its size


def zm_br_velocity_noalloc(n, z, gamma, delta, u, status=None, stream=None):
    """FP64 all-pairs sum on caller-owned device buffers; the library allocates nothing (its
    workspace is a static device array, shared by all calls; n <= 65536).  z, gamma and u must
    hold at least 3 n float64 values; status, if given, is an int32 CUDA tensor."""
    n = int(n)
    for name, x in (("z", z), ("gamma", gamma), ("u", u)):
        k = _numel(x)
        if k is not None and k < 3 * max(n, 0):
            raise ZMError(ZM_ERR_INVALID, f"zm_br_velocity_noalloc: {name} holds {k} values, needs 3 n = {3 * n}")
    sp = None
    if status is not None:
        import torch
        if not (isinstance(status, torch.Tensor) and status.dtype == torch.int32 and status.is_cuda
                and status.numel() >= 1):
            raise ZMError(ZM_ERR_INVALID, "zm_br_velocity_noalloc: status must be an int32 CUDA tensor")
        sp = status.data_ptr()
    _check(load().zm_br_velocity_noalloc(n, ptr(z), ptr(gamma), float(delta), ptr(u), sp, stream))


def _profile_dict(p):
    return {"ms": {KERNEL_NAMES[k]: p.ms[k] for k in range(ZM_K_COUNT)},
            "launches": {KERNEL_NAMES[k]: int(p.launches[k]) for k in range(ZM_K_COUNT)},
            "pairs": int(p.pairs)}


def zm_batch_create(meshes, atwood, g=1.0, mu=0.0, delta=None):
    """meshes: list of (n1, n2, L1, L2, periodic) tuples; atwood/delta: per-interface lists."""
    lib = load()
    k = len(meshes)
    arr = (zm_mesh * k)(*[zm_mesh(int(m[0]), int(m[1]), float(m[2]), float(m[3]), int(bool(m[4])))
                          for m in meshes])
    if delta is None:
        delta = [0.1 * m[2] / m[0] for m in meshes]
    at = (ctypes.c_double * k)(*[float(a) for a in atwood])
    de = (ctypes.c_double * k)(*[float(d) for d in delta])
    h = VP()
    _check(lib.zm_batch_create(k, arr, at, float(g), float(mu), de, ctypes.byref(h)))
    return h


def zm_batch_set_stream(h, stream):
    _check(load().zm_batch_set_stream(h, stream))


def zm_batch_set_state(h, index, z, w):
    _check(load().zm_batch_set_state(h, int(index), ptr(z), ptr(w)))


def zm_batch_get_state(h, index, z, w):
    _check(load().zm_batch_get_state(h, int(index), ptr(z), ptr(w)))


def zm_batch_velocity(h):
    _check(load().zm_batch_velocity(h))


def zm_batch_get_velocity(h, index, u, wdot=None):
    _check(load().zm_batch_get_velocity(h, int(index), ptr(u), ptr(wdot)))


def zm_batch_step(h, dt, nsteps):
    _check(load().zm_batch_step(h, float(dt), int(nsteps)))


def zm_batch_sync(h):
    _check(load().zm_batch_sync(h))


def zm_batch_set_chunk(h, chunk):
    _check(load().zm_batch_set_chunk(h, int(chunk)))


def zm_batch_autotune(h, cache_path=None):
    c = ctypes.c_int32()
    ms = ctypes.c_float()
    p = cache_path.encode() if cache_path else None
    _check(load().zm_batch_autotune(h, p, ctypes.byref(c), ctypes.byref(ms)))
    return c.value, ms.value


def zm_set_cutoff(h, cutoff):
    _check(load().zm_set_cutoff(h, float(cutoff)))


ZM_FAR_TENSOR, ZM_FAR_CUDA = 0, 1


def zm_set_far_path(h, path):
    _check(load().zm_set_far_path(h, int(path)))


def zm_get_far_path(h):
    v = ctypes.c_int32()
    _check(load().zm_get_far_path(h, ctypes.byref(v)))
    return v.value


def zm_batch_set_far_path(h, path):
    _check(load().zm_batch_set_far_path(h, int(path)))


def zm_batch_get_far_path(h):
    v = ctypes.c_int32()
    _check(load().zm_batch_get_far_path(h, ctypes.byref(v)))
    return v.value


def zm_batch_set_cutoff(h, index, cutoff):
    _check(load().zm_batch_set_cutoff(h, int(index), float(cutoff)))


def zm_autotune(h, cache_path=None):
    c = ctypes.c_int32()
    p = cache_path.encode() if cache_path else None
    _check(load().zm_autotune(h, p, ctypes.byref(c)))
    return c.value


def zm_checked_build():
    return bool(load().zm_checked_build())


def zm_bounds_status(clear=True):
    """Index violations counted by the checked build: (hits, first index, source line)."""
    h, f, ln = ctypes.c_uint32(), ctypes.c_int64(), ctypes.c_int32()
    _check(load().zm_bounds_status(ctypes.byref(h), ctypes.byref(f), ctypes.byref(ln), int(bool(clear))))
    return h.value, f.value, ln.value


def zm_autotune_tiles(h, cache_path=None):
    """Tile shape and work-item size of an FP32C context, tuned together: ((tp1, tp2), chunk)."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    p = cache_path.encode() if cache_path else None
    _check(load().zm_autotune_tiles(h, p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return (a.value, b.value), c.value


def zm_set_tile_shape(h, tp1, tp2):
    _check(load().zm_set_tile_shape(h, int(tp1), int(tp2)))


def zm_get_tile_shape(h):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().zm_get_tile_shape(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def zm_batch_set_tile_shape(h, tp1, tp2):
    _check(load().zm_batch_set_tile_shape(h, int(tp1), int(tp2)))


def zm_batch_get_tile_shape(h):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().zm_batch_get_tile_shape(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def zm_batch_autotune_tiles(h, cache_path=None):
    """((tp1, tp2), chunk, ms per evaluation or -1 when remembered)."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_float()
    p = cache_path.encode() if cache_path else None
    _check(load().zm_batch_autotune_tiles(h, p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(ms)))
    return (a.value, b.value), c.value, ms.value


def zm_batch_info(h):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    d = ctypes.c_int32()
    _check(load().zm_batch_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return {"points": a.value, "pairs_per_eval": b.value, "work_items": c.value, "ctas": d.value}


def zm_batch_set_profiling(h, on):
    _check(load().zm_batch_set_profiling(h, int(bool(on))))


def zm_batch_get_profile(h):
    p = zm_profile()
    _check(load().zm_batch_get_profile(h, ctypes.byref(p)))
    return _profile_dict(p)


def zm_batch_destroy(h):
    if h:
        load().zm_batch_destroy(h)


def zm_server_create(mem_budget_bytes, max_slots, g=1.0, mu=0.0):
    h = VP()
    _check(load().zm_server_create(int(mem_budget_bytes), int(max_slots), float(g), float(mu),
                                   ctypes.byref(h)))
    return h


def zm_server_submit(h, n1, n2, z, w, atwood, delta, dt, nsteps, L1=1.0, L2=1.0, periodic=True):
    m = zm_mesh(int(n1), int(n2), float(L1), float(L2), int(bool(periodic)))
    z = np.ascontiguousarray(z, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    rid = ctypes.c_int64()
    _check(load().zm_server_submit(h, ctypes.byref(m), float(atwood), float(delta), float(dt),
                                   int(nsteps), ptr(z), ptr(w), ctypes.byref(rid)))
    return rid.value


def zm_server_request_bytes(n1, n2, L1=1.0, L2=1.0, periodic=True):
    m = zm_mesh(int(n1), int(n2), float(L1), float(L2), int(bool(periodic)))
    b = ctypes.c_size_t()
    _check(load().zm_server_request_bytes(ctypes.byref(m), ctypes.byref(b)))
    return b.value


def zm_server_poll(h, rid):
    st = ctypes.c_int32()
    _check(load().zm_server_poll(h, int(rid), ctypes.byref(st)))
    return st.value


def zm_server_wait(h, rid, timeout_s=-1.0):
    return load().zm_server_wait(h, int(rid), float(timeout_s))


def zm_server_result(h, rid, N):
    """(status, z, w, latency_s, queue_s) of a finished request; releases it."""
    z = np.empty((3, N))
    w = np.empty((2, N))
    lat, q = ctypes.c_double(), ctypes.c_double()
    st = load().zm_server_result(h, int(rid), ptr(z), ptr(w), ctypes.byref(lat), ctypes.byref(q))
    return st, z, w, lat.value, q.value


def zm_server_cancel(h, rid):
    _check(load().zm_server_cancel(h, int(rid)))


def zm_server_get_stats(h):
    s = ServerStats()
    _check(load().zm_server_get_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in s._fields_}


ZM_SERVE_ALL, ZM_SERVE_SRPT = 0, 1


def zm_server_set_policy(h, policy, pairs_per_iteration=0):
    _check(load().zm_server_set_policy(h, int(policy), int(pairs_per_iteration)))


def zm_server_destroy(h):
    if h:
        load().zm_server_destroy(h)


# ---- a small convenience wrapper -------------------------------------------------------------

class ZModel:
    """One interface on the current GPU; owns a zm_ctx.  Arrays are (3, N) / (2, N) float64."""

    def __init__(self, n1, n2=None, L1=1.0, L2=1.0, periodic=True, atwood=0.5, g=1.0, mu=0.0,
                 delta=None, order=ZM_ORDER_HIGH, fp32c=False, df64=False, stream=None):
        self.n1 = int(n1)
        self.n2 = int(n1 if n2 is None else n2)
        self.N = self.n1 * self.n2
        self.order = order | (ZM_PREC_FP32C if fp32c else 0) | (ZM_PREC_DF64 if df64 else 0)
        self.h = zm_create(self.n1, self.n2, L1, L2, periodic, atwood, g, mu, delta, self.order)
        if stream is not None:
            zm_set_stream(self.h, stream)

    def close(self):
        if self.h:
            zm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, z, w):
        zm_set_state(self.h, z, w)

    def get_state(self):
        z = np.empty((3, self.N))
        w = np.empty((2, self.N))
        zm_get_state(self.h, z, w)
        return z, w

    def velocity(self, z=None, w=None, want_wdot=True):
        u = np.empty((3, self.N))
        wd = np.empty((2, self.N)) if want_wdot else None
        zs = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
        ws = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        zm_velocity(self.h, zs, ws, u, wd)
        return (u, wd) if want_wdot else u

    def step(self, dt, nsteps=1):
        zm_step(self.h, dt, nsteps)

    def sync(self):
        zm_sync(self.h)
