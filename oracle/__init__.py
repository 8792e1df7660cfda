"""Serial FP64 CPU oracle for the Z-Model velocity path (ctypes wrapper around zm_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use this package; the product library never does.  It shares no code with
the CUDA library and imports nothing from it.

The equations it evaluates (all FP64, see zm_oracle.c for the full statement):
  * fourth-order two-deep stencils with periodic (seam-shifted) or free-edge ghosts
    (Beatnik, Sec. 3.1 SurfaceMesh / BoundaryCondition);
  * tangents, metric, unit normal and sheet strength gamma = w1 a2 - w2 a1 (Sec. 2, ZModel);
  * the exact all-pairs desingularised Birkhoff-Rott sum (Sec. 3.2.1, ExactBRSolver);
  * the low-order FFT Riesz velocity u = -1/2 (R1 w1 + R2 w2) N (Sec. 2);
  * the vorticity derivative dw/dt = -2 A grad Phi + mu Lap w, and SSP-RK3 (Sec. 3.1).

Parity status per function (what pins each one to something other than itself lives in
tests/test_oracle_pins.py):
  diff1 / laplacian / geometry / sheet_strength / br_velocity / riesz_scalar / fft2 /
  derivative (linear part) / rk3_step: pinned.
  The nonlinear vorticity closure terms of Phi (1/8 w^T h^-1 w and 1/2 |u|^2): parity
  unpinned against the full Z-Model (only internal identities and the linear limit pin them).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zm_oracle.c")
_HDR = os.path.join(_HERE, "zm_oracle.h")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORDER_LOW = 0
ORDER_MEDIUM = 1
ORDER_HIGH = 2


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile zm_oracle.c into oracle/_build/liboracle.so (gcc, no FMA contraction); with
    openmp=True the same source into liboracle_omp.so, whose Birkhoff-Rott sums split their
    targets across threads (same bits; used to write stored expected states)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    lib = os.path.join(_LIBDIR, "liboracle_omp.so") if openmp else _LIB
    stale = (not os.path.exists(lib)
             or os.path.getmtime(lib) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
               "-fno-fast-math"] + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


class _Mesh(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("L1", ctypes.c_double),
                ("L2", ctypes.c_double), ("periodic", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [("atwood", ctypes.c_double), ("g", ctypes.c_double), ("mu", ctypes.c_double),
                ("delta", ctypes.c_double), ("order", ctypes.c_int), ("cutoff", ctypes.c_double)]


_P = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # ZM_ORACLE_LIB lets the mutation test load a deliberately broken copy of the oracle
            path = os.environ.get("ZM_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            M, PR = ctypes.POINTER(_Mesh), ctypes.POINTER(_Params)
            sz, d, i = ctypes.c_size_t, ctypes.c_double, ctypes.c_int
            sig = {
                "zmo_diff1": (None, [M, _P, d, i, _P]),
                "zmo_laplacian": (None, [M, _P, _P]),
                "zmo_geometry": (None, [M, _P, _P, _P, _P, _P]),
                "zmo_sheet_strength": (None, [sz, _P, _P, _P, _P]),
                "zmo_br_velocity": (None, [sz, _P, sz, _P, _P, d, d, _P]),
                "zmo_br_velocity_cutoff": (None, [sz, _P, sz, _P, _P, d, d, d, _P]),
                "zmo_within_cutoff": (i, [_P, sz, _P, sz, d]),
                "zmo_fft2": (None, [i, i, _P, _P, i]),
                "zmo_riesz_scalar": (None, [M, _P, _P]),
                "zmo_phi": (None, [sz, _P, _P, _P, _P, d, _P]),
                "zmo_wdot": (None, [M, _P, _P, d, d, _P]),
                "zmo_derivative": (i, [M, PR, _P, _P, _P, _P]),
                "zmo_rk3_step": (i, [M, PR, _P, _P, d]),
                "zmo_run": (i, [M, PR, _P, _P, d, i]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _arr(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


class Mesh:
    """n1 x n2 interface mesh on [0, L1) x [0, L2); periodic or free edges."""

    def __init__(self, n1, n2=None, L1=1.0, L2=1.0, periodic=True):
        self.n1 = int(n1)
        self.n2 = int(n1 if n2 is None else n2)
        self.L1, self.L2, self.periodic = float(L1), float(L2), bool(periodic)

    @property
    def N(self):
        return self.n1 * self.n2

    def c(self):
        return _Mesh(self.n1, self.n2, self.L1, self.L2, int(self.periodic))


def _params(atwood, g, mu, delta, order, cutoff=0.0):
    return _Params(float(atwood), float(g), float(mu), float(delta), int(order), float(cutoff))


def diff1(mesh, f, axis, shift=0.0):
    lib = _load()
    f = _arr(f, (mesh.N,))
    out = np.empty(mesh.N)
    m = mesh.c()
    lib.zmo_diff1(ctypes.byref(m), _ptr(f), float(shift), int(axis), _ptr(out))
    return out


def laplacian(mesh, f):
    lib = _load()
    f = _arr(f, (mesh.N,))
    out = np.empty(mesh.N)
    m = mesh.c()
    lib.zmo_laplacian(ctypes.byref(m), _ptr(f), _ptr(out))
    return out


def geometry(mesh, z):
    """Return (a1, a2, h, nrm): tangents (3,N), metric (h11,h12,h22,det) (4,N), normal (3,N)."""
    lib = _load()
    z = _arr(z, (3, mesh.N))
    a1, a2 = np.empty((3, mesh.N)), np.empty((3, mesh.N))
    h, nrm = np.empty((4, mesh.N)), np.empty((3, mesh.N))
    m = mesh.c()
    lib.zmo_geometry(ctypes.byref(m), _ptr(z), _ptr(a1), _ptr(a2), _ptr(h), _ptr(nrm))
    return a1, a2, h, nrm


def sheet_strength(w, a1, a2):
    lib = _load()
    w = _arr(w)
    N = w.shape[-1]
    w = w.reshape(2, N)
    a1, a2 = _arr(a1, (3, N)), _arr(a2, (3, N))
    g = np.empty((3, N))
    lib.zmo_sheet_strength(N, _ptr(w), _ptr(a1), _ptr(a2), _ptr(g))
    return g


def br_velocity(zt, zs, gamma, weight, delta):
    """u_i = -(weight/4pi) sum_j (zt_i - zs_j) x gamma_j / (|zt_i - zs_j|^2 + delta^2)^(3/2)."""
    lib = _load()
    zt = _arr(zt)
    zs = _arr(zs)
    nt, ns = zt.shape[-1], zs.shape[-1]
    zt, zs, gamma = zt.reshape(3, nt), zs.reshape(3, ns), _arr(gamma, (3, ns))
    u = np.empty((3, nt))
    lib.zmo_br_velocity(nt, _ptr(zt), ns, _ptr(zs), _ptr(gamma), float(weight), float(delta),
                        _ptr(u))
    return u


def br_velocity_cutoff(zt, zs, gamma, weight, delta, cutoff):
    """br_velocity over the sources with |zt_i - zs_j| <= cutoff (decided in FP64)."""
    lib = _load()
    zt = _arr(zt)
    zs = _arr(zs)
    nt, ns = zt.shape[-1], zs.shape[-1]
    zt, zs, gamma = zt.reshape(3, nt), zs.reshape(3, ns), _arr(gamma, (3, ns))
    u = np.empty((3, nt))
    lib.zmo_br_velocity_cutoff(nt, _ptr(zt), ns, _ptr(zs), _ptr(gamma), float(weight), float(delta),
                               float(cutoff), _ptr(u))
    return u


def within_cutoff(zi, zj, cutoff):
    """The oracle's in/out decision for one pair: |zi - zj|^2 <= cutoff^2 in FP64."""
    lib = _load()
    a, b = _arr(zi, (3,)), _arr(zj, (3,))
    return bool(lib.zmo_within_cutoff(_ptr(a), 1, _ptr(b), 1, float(cutoff)))


def fft2(re, im, sign):
    lib = _load()
    re = _arr(re).copy()
    im = _arr(im).copy()
    n1, n2 = re.shape
    lib.zmo_fft2(n1, n2, _ptr(re), _ptr(im), int(sign))
    return re, im


def riesz_scalar(mesh, w):
    lib = _load()
    w = _arr(w, (2, mesh.N))
    s = np.empty(mesh.N)
    m = mesh.c()
    lib.zmo_riesz_scalar(ctypes.byref(m), _ptr(w), _ptr(s))
    return s


def phi(z, w, h, u, g):
    lib = _load()
    N = _arr(z).size // 3
    z, w, h, u = _arr(z, (3, N)), _arr(w, (2, N)), _arr(h, (4, N)), _arr(u, (3, N))
    out = np.empty(N)
    lib.zmo_phi(N, _ptr(z), _ptr(w), _ptr(h), _ptr(u), float(g), _ptr(out))
    return out


def wdot(mesh, phi_, w, atwood, mu):
    lib = _load()
    phi_, w = _arr(phi_, (mesh.N,)), _arr(w, (2, mesh.N))
    out = np.empty((2, mesh.N))
    m = mesh.c()
    lib.zmo_wdot(ctypes.byref(m), _ptr(phi_), _ptr(w), float(atwood), float(mu), _ptr(out))
    return out


def derivative(mesh, z, w, atwood, g, mu, delta, order=ORDER_HIGH, cutoff=0.0):
    """One evaluation L(z, w) = (u, wdot) of the Z-Model derivative."""
    lib = _load()
    z, w = _arr(z, (3, mesh.N)), _arr(w, (2, mesh.N))
    u, wd = np.empty((3, mesh.N)), np.empty((2, mesh.N))
    m, p = mesh.c(), _params(atwood, g, mu, delta, order, cutoff)
    lib.zmo_derivative(ctypes.byref(m), ctypes.byref(p), _ptr(z), _ptr(w), _ptr(u), _ptr(wd))
    return u, wd


def run(mesh, z, w, atwood, g, mu, delta, dt, nsteps, order=ORDER_HIGH, cutoff=0.0):
    """Advance (z, w) by nsteps SSP-RK3 steps; returns new arrays."""
    lib = _load()
    z, w = _arr(z, (3, mesh.N)).copy(), _arr(w, (2, mesh.N)).copy()
    m, p = mesh.c(), _params(atwood, g, mu, delta, order, cutoff)
    lib.zmo_run(ctypes.byref(m), ctypes.byref(p), _ptr(z), _ptr(w), float(dt), int(nsteps))
    return z, w
