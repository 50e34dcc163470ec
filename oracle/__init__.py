"""FP64 CPU oracle for GLAMER's ray shooting (arXiv:1312.1128).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the product library never
imports, links or calls it.  The arithmetic lives in ``lens_oracle.c`` (plain
C, FP64, OpenMP over rays); this module compiles it on first use and wraps it
with ctypes.

Functions
---------
eval_component(comp, x, y)      one component's (a1, a2, kappa, g1, g2)
direct_sum(comps, rx, ry)       Sec. 5.1 theta=0 limit: sum over all components
direct_vjp(comps, rx, ry, G)    gradient of a loss of alpha w.r.t. (m, x, y[, p0, p1])
potential_component / direct_potential   lensing potential psi (Eq. alpha, Eq. timedelay)
PaperTree(comps, leaf_max, th)  Sec. 3.2 tree, evaluated ray by ray, with counts
refine.refine_cells(...)        Sec. 3.4 cell interpolation with A from App. A (numpy)
knn.kth_neighbour_distance(...)  Sec. 3.1 3D smoothing lengths (brute force / cKDTree)
images.find_images(...)         Sec. 4 image finding by grid refinement (pure Python)
images.sis_finite_source_mu     App. B finite-source SIS magnification (quadrature)

Components are a numpy structured array of ``COMP_DTYPE`` (see
``make_components``); types follow ``POINT, GAUSS, NFW, SIS, DISK``.
Parity is pinned for every function by tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

POINT, GAUSS, NFW, SIS, DISK = 0, 1, 2, 3, 4

COMP_DTYPE = np.dtype([("x", "<f8"), ("y", "<f8"), ("m", "<f8"), ("p0", "<f8"),
                       ("p1", "<f8"), ("type", "<i4"), ("pad", "<i4")])
assert COMP_DTYPE.itemsize == 48

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lens_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblens_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lens_oracle.c into liblens_oracle.so (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_eval_component.argtypes = [vp, d, d, vp]
        lib.or_eval_component.restype = None
        lib.or_direct_sum.argtypes = [vp, i64, vp, vp, i64, vp, vp, i32]
        lib.or_direct_sum.restype = i32
        lib.or_potential_component.argtypes = [vp, d, d]
        lib.or_potential_component.restype = d
        lib.or_direct_potential.argtypes = [vp, i64, vp, vp, i64, vp, vp, i32]
        lib.or_direct_potential.restype = i32
        lib.or_direct_vjp.argtypes = [vp, i64, vp, vp, i64, vp, vp, i32, i32]
        lib.or_direct_vjp.restype = i32
        lib.or_tree_build.argtypes = [vp, i64, i32, d]
        lib.or_tree_build.restype = vp
        lib.or_tree_free.argtypes = [vp]
        lib.or_tree_free.restype = None
        lib.or_tree_nboxes.argtypes = [vp]
        lib.or_tree_nboxes.restype = i64
        lib.or_tree_eval.argtypes = [vp, vp, vp, i64, vp, vp, i32]
        lib.or_tree_eval.restype = i32
        lib.or_max_threads.argtypes = []
        lib.or_max_threads.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def make_components(type_, x, y, m, p0=0.0, p1=0.0) -> np.ndarray:
    """Structured component array from broadcastable fields."""
    x = np.asarray(x, dtype=np.float64)
    n = np.broadcast(x, np.asarray(y), np.asarray(m), np.asarray(p0), np.asarray(p1),
                     np.asarray(type_)).shape
    c = np.zeros(n, dtype=COMP_DTYPE)
    c["x"], c["y"], c["m"], c["p0"], c["p1"], c["type"] = x, y, m, p0, p1, type_
    return c.reshape(-1)


def concat(*parts) -> np.ndarray:
    return np.ascontiguousarray(np.concatenate([np.asarray(p, COMP_DTYPE).reshape(-1) for p in parts]))


def max_threads() -> int:
    return int(_load().or_max_threads())


def eval_component(comp, x: float, y: float) -> np.ndarray:
    """(alpha1, alpha2, kappa, gamma1, gamma2) of one component at (x, y)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(comp, COMP_DTYPE).reshape(1))
    out = np.zeros(5)
    lib.or_eval_component(_ptr(c), float(x), float(y), _ptr(out))
    return out


def direct_sum(comps, rx, ry, nthreads: int = 0, with_absum: bool = False):
    """Direct FP64 sum over all components for every ray: (nr, 5) array
    [alpha1, alpha2, kappa, gamma1, gamma2]; optionally also sum |term|."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(comps, COMP_DTYPE).reshape(-1))
    rx = np.ascontiguousarray(rx, dtype=np.float64).reshape(-1)
    ry = np.ascontiguousarray(ry, dtype=np.float64).reshape(-1)
    assert rx.shape == ry.shape
    out = np.zeros((rx.size, 5))
    ab = np.zeros((rx.size, 5)) if with_absum else None
    lib.or_direct_sum(_ptr(c), c.size, _ptr(rx), _ptr(ry), rx.size, _ptr(out),
                      _ptr(ab) if ab is not None else None, int(nthreads))
    return (out, ab) if with_absum else out


def potential_component(comp, x: float, y: float) -> float:
    """One component's lensing potential psi at (x, y) (alpha = grad psi)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(comp, COMP_DTYPE).reshape(-1)[:1])
    return lib.or_potential_component(_ptr(c), float(x), float(y))


def direct_potential(comps, rx, ry, nthreads: int = 0, with_absum: bool = False):
    """Direct FP64 sum of the lensing potential over all components (Eq.
    alpha, Eq. timedelay); optionally also sum |term| per ray."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(comps, COMP_DTYPE).reshape(-1))
    rx = np.ascontiguousarray(rx, dtype=np.float64).reshape(-1)
    ry = np.ascontiguousarray(ry, dtype=np.float64).reshape(-1)
    out = np.zeros(rx.size)
    ab = np.zeros(rx.size) if with_absum else None
    lib.or_direct_potential(_ptr(c), c.size, _ptr(rx), _ptr(ry), rx.size, _ptr(out),
                            _ptr(ab) if ab is not None else None, int(nthreads))
    return (out, ab) if with_absum else out


def direct_vjp(comps, rx, ry, G, nthreads: int = 0, params: bool = False) -> np.ndarray:
    """dL/d(m, x, y) for every component, given G = dL/d(outputs) (nr, 5);
    only the alpha columns of G may be non-zero.  With params, (nc, 5):
    also dL/d(p0, p1), the component's shape parameters (GAUSS r_sm, q; NFW
    r_s, R_max; SIS r_E; DISK R)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(comps, COMP_DTYPE).reshape(-1))
    rx = np.ascontiguousarray(rx, dtype=np.float64).reshape(-1)
    ry = np.ascontiguousarray(ry, dtype=np.float64).reshape(-1)
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(rx.size, 5)
    grad = np.zeros((c.size, 5 if params else 3))
    rc = lib.or_direct_vjp(_ptr(c), c.size, _ptr(rx), _ptr(ry), rx.size, _ptr(G), _ptr(grad),
                           1 if params else 0, int(nthreads))
    if rc != 0:
        raise ValueError("direct_vjp supports gradients of alpha only")
    return grad


class PaperTree:
    """The tree of Sec. 3.2, built on the CPU and walked ray by ray."""

    def __init__(self, comps, leaf_max: int = 5, theta: float = 0.1):
        self._lib = _load()
        self.comps = np.ascontiguousarray(np.asarray(comps, COMP_DTYPE).reshape(-1))
        h = self._lib.or_tree_build(_ptr(self.comps), self.comps.size, int(leaf_max), float(theta))
        if not h:
            raise ValueError("tree build rejected its input (empty, leaf_max < 1 or SIS component)")
        self._h = ctypes.c_void_p(h)

    @property
    def n_boxes(self) -> int:
        return int(self._lib.or_tree_nboxes(self._h))

    def eval(self, rx, ry, nthreads: int = 0):
        """Returns (out (nr, 5), counts (nr, 5)); counts columns are far cells,
        near point evaluations, near full-profile evaluations, big-list
        corrections and boxes visited."""
        rx = np.ascontiguousarray(rx, dtype=np.float64).reshape(-1)
        ry = np.ascontiguousarray(ry, dtype=np.float64).reshape(-1)
        out = np.zeros((rx.size, 5))
        counts = np.zeros((rx.size, 5), dtype=np.int64)
        self._lib.or_tree_eval(self._h, _ptr(rx), _ptr(ry), rx.size, _ptr(out), _ptr(counts),
                               int(nthreads))
        return out, counts

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_tree_free(h)
            self._h = None
