"""GB300 ray shooting for gravitational lensing (GLAMER Part I, arXiv:1312.1128).

Thin Python binding over liblens (include/lens.h): it marshals PyTorch CUDA
tensors into the C ABI and back, nothing more -- every step of the path runs
in the library's CUDA kernels.  There is no CPU fallback: if liblens.so is
missing or CUDA is unavailable, the calls raise.

    lens = Lens(species=[Species.gauss(parts, q=3.0)], halos=[Halo.sis(0, 0, 0.5)],
                theta=0.3)
    a1, a2, kappa, g1, g2 = lens.shoot(rx, ry)          # device tensors (Sec. 3.2)
    lens.shoot_batches(offsets, origins, rx, ry)          # uneven batches, one launch
    psi, a1, a2 = lens.potential(rx, ry)                  # lensing potential (time delay)
    grads = lens.backward(rx, ry, g_alpha1, g_alpha2)     # adjoint w.r.t. (m, x, y, size)
    alpha = shoot(lens, rx, ry, species_data=parts)       # differentiable (autograd)
    images, stats = lens.find_images(sources, x0, y0, side, n)   # Sec. 4 image finding
    refine_cells(...)                                      # Sec. 3.4 cell interpolation
    r_sm = smoothing_lengths(xyz, 32)                      # Sec. 3.1 smoothing lengths

Ray positions are an FP64 origin plus offsets (float32 or float64 tensors), so
microlensing-scale patches keep their resolution (the paper stores alpha in
higher precision than kappa/gamma for the same reason, Sec. 3.4).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = ["Lens", "Species", "Halo", "LensError", "shoot", "lib", "fp32_peak", "fp64_peak", "fail_allocations",
           "refine_cells", "smoothing_lengths",
           "POINT", "GAUSS", "NFW", "SIS", "DISK", "ALPHA_ONLY", "DIRECT", "ACCUMULATE", "USE_GRAPH",
           "COUNT", "TIMING", "REFINE_KAPPA_GAMMA", "REFINE_DEFLECTION"]

POINT, GAUSS, NFW, SIS, DISK = 0, 1, 2, 3, 4
F32, F64 = 0, 1
PREC_FP32, PREC_FP64 = 0, 1
ALPHA_ONLY, DIRECT, ACCUMULATE, USE_GRAPH, COUNT, TIMING, KEEP_LISTS = 1, 2, 4, 8, 16, 32, 64
WALK_DEFAULT, WALK_WARP, WALK_PAIRS, WALK_TRIOS = 0, 1, 2, 3
TILE_DEFAULT, TILE_STANDARD, TILE_LARGE = 0, 1, 2
REFINE_KAPPA_GAMMA, REFINE_DEFLECTION = 0, 1

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "liblens.so")
_lib = None


class LensError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"liblens status {status}: {msg}")
        self.status = status


class _Species(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("n", ctypes.c_int64),
                ("data", ctypes.c_void_p), ("shape", ctypes.c_double)]


class _Halo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("x", ctypes.c_double),
                ("y", ctypes.c_double), ("m", ctypes.c_double), ("p0", ctypes.c_double),
                ("p1", ctypes.c_double)]


class _AmrParams(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("side", ctypes.c_double),
                ("n", ctypes.c_int32), ("l_max", ctypes.c_int32), ("mu_min", ctypes.c_double),
                ("f_area", ctypes.c_double), ("n_min", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("max_cells", ctypes.c_int64)]


class _Image(ctypes.Structure):
    _fields_ = [("source", ctypes.c_int32), ("n_cells", ctypes.c_int32), ("area", ctypes.c_double),
                ("mu", ctypes.c_double), ("first", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("leaf_max", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("group_rays", ctypes.c_int32),
                ("walk", ctypes.c_int32), ("tile", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_halos", ctypes.c_int64), ("n_particles", ctypes.c_int64 * 8),
                ("n_nodes", ctypes.c_int64 * 8), ("n_leaves", ctypes.c_int64 * 8),
                ("n_big", ctypes.c_int64 * 8), ("depth", ctypes.c_int32 * 8),
                ("root", (ctypes.c_double * 3) * 8), ("build_ms", (ctypes.c_double * 4) * 8),
                ("group_rays", ctypes.c_int32), ("walk", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("split_groups", ctypes.c_int32)]


def lib():
    """Load liblens.so (built by __graft_entry__.build() or _build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"liblens.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.lens_build_tree.argtypes = [ctypes.POINTER(_Species), i32, ctypes.POINTER(_Halo), i64,
                                  ctypes.POINTER(_Params), vp, ctypes.POINTER(vp)]
    L.lens_shoot_rays.argtypes = [vp, d, d, vp, vp, i32, i64, vp, vp, vp, vp, vp, i32, vp]
    L.lens_shoot_batches.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_double), vp, vp, i32, vp, vp, vp, vp,
                                     vp, i32, vp]
    L.lens_shoot_rays_backward.argtypes = [vp, d, d, vp, vp, i32, i64, vp, vp, vp, vp, vp,
                                           ctypes.POINTER(vp), vp, i32, vp]
    L.lens_reserve.argtypes = [vp, i64, i64]
    L.lens_shoot_rays_direct_noalloc.argtypes = [vp, d, d, vp, vp, i32, i64, vp, vp, vp, vp, vp, i32, vp]
    L.lens_autotune.argtypes = [vp, d, d, vp, vp, i32, i64, vp, ctypes.POINTER(ctypes.c_int32)]
    L.lens_sync_status.argtypes = [vp, vp]
    L.lens_set_wait_limit.argtypes = [vp, i64]
    L.lens_tree_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    L.lens_tree_export.argtypes = [vp, i32, vp, vp, vp, vp]
    L.lens_fp32_peak.argtypes = [i64, ctypes.POINTER(ctypes.c_double), vp]
    L.lens_fp64_peak.argtypes = [i64, ctypes.POINTER(ctypes.c_double), vp]
    L.lens_fail_allocations.argtypes = [i64]
    L.lens_fail_allocations.restype = None
    L.lens_tree_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), i32]
    L.lens_last_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.lens_refine_cells.argtypes = [d, d, d, i64, i64, vp, vp, i32, vp, vp, vp, vp, i64, i32, d, i32, vp, vp,
                                    vp, vp, vp]
    L.lens_smoothing_lengths.argtypes = [vp, i64, i32, vp, vp]
    L.lens_shoot_potential.argtypes = [vp, d, d, vp, vp, i32, i64, vp, vp, vp, i32, vp]
    L.lens_find_images.argtypes = [vp, vp, i32, vp, i32, vp, vp, vp, vp]
    L.lens_kernel_launches.argtypes = []
    L.lens_kernel_launches.restype = ctypes.c_int64
    L.lens_free_tree.argtypes = [vp]
    L.lens_free_tree.restype = None
    L.lens_status_string.restype = ctypes.c_char_p
    L.lens_last_error.restype = ctypes.c_char_p
    for name in ["lens_build_tree", "lens_shoot_rays", "lens_shoot_batches",
                 "lens_shoot_rays_backward", "lens_reserve", "lens_sync_status",
                 "lens_tree_get_info", "lens_tree_export", "lens_fp32_peak", "lens_fp64_peak", "lens_api_version",
                 "lens_tree_counters", "lens_last_timing", "lens_autotune",
                 "lens_shoot_rays_direct_noalloc", "lens_refine_cells", "lens_smoothing_lengths",
                 "lens_shoot_potential", "lens_find_images", "lens_set_wait_limit"]:
        getattr(L, name).restype = ctypes.c_int32
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise LensError(status, lib().lens_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("liblens takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("liblens takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _out_ptr(t):
    """An output array: a CUDA tensor, or a page-locked CPU tensor (the
    kernels write each element once, straight into host memory)."""
    if t is not None and not t.is_cuda:
        if not t.is_pinned():
            raise ValueError("host outputs must be page-locked (tensor.pin_memory())")
        if not t.is_contiguous():
            raise ValueError("liblens takes contiguous tensors")
        return ctypes.c_void_p(t.data_ptr())
    return _dev_ptr(t)


@dataclass
class Species:
    """A homogeneous particle set: data is an (n, 4) CUDA tensor {x, y, m, p}."""
    kind: int
    data: object
    shape: float = 0.0

    @staticmethod
    def points(data):
        return Species(POINT, data, 0.0)

    @staticmethod
    def gauss(data, q: float = 3.0):
        return Species(GAUSS, data, float(q))

    @staticmethod
    def nfw(data, conc: float):
        return Species(NFW, data, float(conc))


@dataclass
class Halo:
    kind: int
    x: float
    y: float
    m: float = 0.0
    p0: float = 0.0
    p1: float = 0.0

    @staticmethod
    def sis(x, y, r_e):
        return Halo(SIS, x, y, 0.0, r_e, 0.0)

    @staticmethod
    def disk(x, y, m, radius):
        return Halo(DISK, x, y, m, radius, 0.0)

    @staticmethod
    def nfw(x, y, m, r_s, r_max):
        return Halo(NFW, x, y, m, r_s, r_max)

    @staticmethod
    def point(x, y, m):
        return Halo(POINT, x, y, m)

    @staticmethod
    def gauss(x, y, m, r_sm, q):
        return Halo(GAUSS, x, y, m, r_sm, q)


class Lens:
    """A built lens: one quadtree per species plus analytic halos."""

    def __init__(self, species=(), halos=(), theta: float = 0.1, leaf_max: int = 5,
                 precision: str = "fp32", group_rays: int = 0, walk: str = "default", tile: str = "default",
                 stream=None):
        L = lib()
        self._keep = []
        sp = (_Species * max(1, len(species)))()
        for i, s in enumerate(species):
            t = s.data
            torch = _torch()
            if t.dim() != 2 or t.shape[1] != 4:
                raise ValueError("species data must be (n, 4)")
            if t.dtype not in (torch.float32, torch.float64):
                raise ValueError("species data must be float32 or float64")
            self._keep.append(t)
            sp[i] = _Species(s.kind, F32 if t.dtype == torch.float32 else F64, t.shape[0],
                             _dev_ptr(t) if t.shape[0] > 0 else None, s.shape)
        hs = (_Halo * max(1, len(halos)))()
        for i, h in enumerate(halos):
            hs[i] = _Halo(h.kind, 0, h.x, h.y, h.m, h.p0, h.p1)
        prec = {"fp32": PREC_FP32, "fp64": PREC_FP64}[precision]
        wk = {"default": WALK_DEFAULT, "warp": WALK_WARP, "pairs": WALK_PAIRS, "trios": WALK_TRIOS}[walk]
        tl = {"default": TILE_DEFAULT, "standard": TILE_STANDARD, "large": TILE_LARGE}[tile]
        params = _Params(float(theta), int(leaf_max), prec, int(group_rays), wk, tl, 0)
        h = ctypes.c_void_p()
        _check(L.lens_build_tree(sp, len(species), hs, len(halos), ctypes.byref(params),
                                 _stream_ptr(stream), ctypes.byref(h)))
        self._h = h
        self.precision = precision
        self.n_species = len(species)
        self.n_halos = len(halos)
        self.species = list(species)
        self.halos = list(halos)
        self.theta = theta
        self._build_args = dict(theta=theta, leaf_max=leaf_max, precision=precision)
        # what the tree was built from: storage and in-place version of every
        # species tensor (a differentiable shoot rebuilds when they change)
        self._built_from = [(s.data.data_ptr(), s.data._version) for s in self.species]

    def built_from(self, species_data) -> bool:
        """True if the tree was built from these tensors' current values."""
        if len(species_data) != len(self._built_from):
            return False
        return all(t.data_ptr() == p and t._version == v for t, (p, v) in zip(species_data, self._built_from))

    def rebuild(self, species_data, stream=None):
        """Rebuild the tree from new values of the species tensors (same
        kinds, shapes, halos and parameters; the tuned group size and walk
        form are kept)."""
        if len(species_data) != len(self.species):
            raise ValueError("rebuild takes one tensor per species")
        inf = self.info()
        new = Lens([Species(s.kind, t.detach(), s.shape) for s, t in zip(self.species, species_data)],
                   self.halos, group_rays=inf["group_rays"], walk=inf["walk"], tile=inf["tile"], stream=stream,
                   **self._build_args)
        self.close()
        self._h, new._h = new._h, None
        self._keep, self.species, self._built_from = new._keep, new.species, new._built_from

    # ------------------------------------------------------------------
    @property
    def out_dtype(self):
        torch = _torch()
        return torch.float64 if self.precision == "fp64" else torch.float32

    def info(self) -> dict:
        inf = _Info()
        _check(lib().lens_tree_get_info(self._h, ctypes.byref(inf)))
        k = inf.n_species
        return dict(n_species=k, precision=inf.precision, n_halos=inf.n_halos,
                    n_particles=list(inf.n_particles[:k]), n_nodes=list(inf.n_nodes[:k]),
                    n_leaves=list(inf.n_leaves[:k]), n_big=list(inf.n_big[:k]),
                    depth=list(inf.depth[:k]), root=[tuple(inf.root[i]) for i in range(k)],
                    build_ms=[tuple(inf.build_ms[i]) for i in range(k)], group_rays=inf.group_rays,
                    walk={WALK_WARP: "warp", WALK_PAIRS: "pairs", WALK_TRIOS: "trios"}.get(inf.walk, "default"),
                    tile={TILE_STANDARD: "standard", TILE_LARGE: "large"}.get(inf.tile, "default"),
                    split_groups=inf.split_groups)

    def export(self, species: int = 0):
        """Host copies of one species' tree: nodes (n_nodes, 8), links
        (n_nodes, 4), perm (n,), listed (n,)."""
        inf = self.info()
        nn, n = inf["n_nodes"][species], inf["n_particles"][species]
        nodes = np.zeros((nn, 8), np.float64 if self.precision == "fp64" else np.float32)
        links = np.zeros((nn, 4), np.int32)
        perm = np.zeros(n, np.int32)
        listed = np.zeros(n, np.int32)
        _check(lib().lens_tree_export(self._h, species, nodes.ctypes.data, links.ctypes.data,
                                      perm.ctypes.data, listed.ctypes.data))
        return nodes, links, perm, listed

    def counters(self, reset: bool = True) -> dict:
        """Walk counters accumulated by calls made with COUNT."""
        a = (ctypes.c_int64 * 8)()
        _check(lib().lens_tree_counters(self._h, a, 1 if reset else 0))
        keys = ["groups", "visited", "cells", "leaf_particles", "big_scanned", "big_kept",
                "ray_interactions", "reserved"]
        return dict(zip(keys, list(a)))

    def last_timing(self):
        """(group_ms, walk_ms) of the last call made with TIMING."""
        g, w = ctypes.c_double(), ctypes.c_double()
        _check(lib().lens_last_timing(self._h, ctypes.byref(g), ctypes.byref(w)))
        return g.value, w.value

    def sync(self, stream=None):
        _check(lib().lens_sync_status(self._h, _stream_ptr(stream)))

    def set_wait_limit(self, cycles: int = 0):
        """Bound of the pairs walk's waits between warps, in SM clock cycles
        (0: the default, about 2 s)."""
        _check(lib().lens_set_wait_limit(self._h, int(cycles)))

    def autotune(self, dx, dy, origin=(0.0, 0.0), stream=None) -> int:
        """Time the walk with 32- and 64-ray groups on these rays; keep and
        return the faster group size."""
        torch = _torch()
        g = ctypes.c_int32()
        rd = F32 if dx.dtype == torch.float32 else F64
        _check(lib().lens_autotune(self._h, float(origin[0]), float(origin[1]), _dev_ptr(dx),
                                   _dev_ptr(dy), rd, dx.numel(), _stream_ptr(stream), ctypes.byref(g)))
        return g.value

    def reserve(self, max_rays: int, max_batches: int = 1):
        _check(lib().lens_reserve(self._h, int(max_rays), int(max_batches)))

    def _outs(self, n, alpha_only, out):
        torch = _torch()
        k = 2 if alpha_only else 5
        if out is None:
            out = [torch.empty(n, dtype=self.out_dtype, device="cuda") for _ in range(k)]
            out += [None] * (5 - k)
            return out
        out = list(out) + [None] * (5 - len(out))
        for q, o in enumerate(out):
            if o is None:
                if q < k:
                    raise ValueError("alpha outputs (and kappa, gamma without ALPHA_ONLY) are required")
            elif o.dtype != self.out_dtype or o.numel() < n:
                raise ValueError(f"outputs must be {self.out_dtype} with at least {n} elements")
        return out

    def shoot(self, dx, dy, origin=(0.0, 0.0), flags: int = 0, out=None, stream=None):
        """alpha1, alpha2, kappa, gamma1, gamma2 at rays origin + (dx, dy).
        `out` may hold CUDA tensors or page-locked CPU tensors (written
        directly; synchronise the stream before reading them)."""
        torch = _torch()
        n = dx.numel()
        if dy.numel() != n or dx.dtype != dy.dtype or dx.dtype not in (torch.float32, torch.float64):
            raise ValueError("dx, dy must be float32 or float64 of the same size")
        out = self._outs(n, bool(flags & ALPHA_ONLY), out)
        rd = F32 if dx.dtype == torch.float32 else F64
        _check(lib().lens_shoot_rays(self._h, float(origin[0]), float(origin[1]), _dev_ptr(dx),
                                     _dev_ptr(dy), rd, n, *[_out_ptr(o) for o in out], int(flags),
                                     _stream_ptr(stream)))
        return out

    def potential(self, dx, dy, origin=(0.0, 0.0), flags: int = 0, out=None, stream=None):
        """Lensing potential psi and alpha1, alpha2 at rays origin + (dx, dy)
        (lens_shoot_potential; the time delay is |alpha|^2/2 - psi)."""
        torch = _torch()
        n = dx.numel()
        if dy.numel() != n or dx.dtype != dy.dtype:
            raise ValueError("dx, dy must match in size and dtype")
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        if out is None:
            out = [torch.empty(n, dtype=dt, device=dx.device) for _ in range(3)]
        out = list(out) + [None] * (3 - len(out))
        if out[0] is None:
            raise ValueError("psi output is required")
        for o in out:
            if o is not None and (o.dtype != dt or o.numel() < n):
                raise ValueError(f"outputs must be {dt} with at least {n} elements")
        rd = F32 if dx.dtype == torch.float32 else F64
        _check(lib().lens_shoot_potential(self._h, float(origin[0]), float(origin[1]), _dev_ptr(dx), _dev_ptr(dy),
                                          rd, n, *[_out_ptr(o) for o in out], int(flags), _stream_ptr(stream)))
        return out

    def find_images(self, sources, x0, y0, side, n=64, l_max=12, mu_min=0.01, f_area=5e-4, n_min=50,
                    max_cells=0, max_rounds=0, max_images=4096, stream=None):
        """Images of uniform circular sources (lens_find_images, Sec. 4).
        sources: (k, 3) array-like of {y_c1, y_c2, R}.  Returns (images,
        stats): images a list of dicts (source, n_cells, area, mu, first)
        ordered by source, stats {rays, cells, rounds, label_cells, label_ms,
        shoot_ms}: rays shot, final cells, refinement rounds, cells visited by
        the image-labelling passes and their device time, the shooting's."""
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.float64).reshape(-1, 3))
        prm = _AmrParams(float(x0), float(y0), float(side), int(n), int(l_max), float(mu_min), float(f_area),
                         int(n_min), int(max_rounds), int(max_cells))
        out = (_Image * max(1, int(max_images)))()
        cnt = ctypes.c_int32()
        st = (ctypes.c_int64 * 6)()
        _check(lib().lens_find_images(self._h, ctypes.byref(prm), src.shape[0], src.ctypes.data_as(ctypes.c_void_p),
                                      int(max_images), out, ctypes.byref(cnt), st, _stream_ptr(stream)))
        imgs = [{"source": out[k].source, "n_cells": out[k].n_cells, "area": out[k].area, "mu": out[k].mu,
                 "first": out[k].first} for k in range(cnt.value)]
        return imgs, {"rays": st[0], "cells": st[1], "rounds": st[2], "label_cells": st[3],
                      "label_ms": st[4] * 1e-6, "shoot_ms": st[5] * 1e-6}

    def shoot_direct_noalloc(self, dx, dy, out, origin=(0.0, 0.0), flags: int = 0, stream=None):
        """Direct sum into caller-provided outputs without any device
        allocation (lens_shoot_rays_direct_noalloc: at most 262,144 rays per
        call, calls must not overlap on the GPU).  out: five tensors (kappa,
        gamma1, gamma2 may be None with ALPHA_ONLY) of the tree's output dtype
        and at least n elements each."""
        torch = _torch()
        n = dx.numel()
        if dy.numel() != n or dx.dtype != dy.dtype or dx.dtype not in (torch.float32, torch.float64):
            raise ValueError("dx, dy must be float32 or float64 of the same size")
        out = list(out) + [None] * (5 - len(out))
        need = 2 if flags & ALPHA_ONLY else 5
        for k, o in enumerate(out):
            if o is None:
                if k < need:
                    raise ValueError("alpha outputs (and kappa, gamma without ALPHA_ONLY) are required")
                continue
            if o.dtype != self.out_dtype or o.numel() < n:
                raise ValueError(f"outputs must be {self.out_dtype} with at least {n} elements")
        rd = F32 if dx.dtype == torch.float32 else F64
        _check(lib().lens_shoot_rays_direct_noalloc(
            self._h, float(origin[0]), float(origin[1]), _dev_ptr(dx), _dev_ptr(dy), rd, n,
            *[_dev_ptr(o) for o in out], int(flags), _stream_ptr(stream)))
        return out

    def shoot_batches(self, offsets, origins, dx, dy, flags: int = 0, out=None, stream=None):
        """Many ray batches (host int64 offsets (B+1,), host float64 origins (B, 2))."""
        torch = _torch()
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        origins = np.ascontiguousarray(origins, dtype=np.float64).reshape(-1, 2)
        n = int(offsets[-1])
        out = self._outs(n, bool(flags & ALPHA_ONLY), out)
        rd = F32 if dx.dtype == torch.float32 else F64
        _check(lib().lens_shoot_batches(
            self._h, origins.shape[0], offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            origins.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _dev_ptr(dx), _dev_ptr(dy), rd,
            *[_out_ptr(o) for o in out], int(flags), _stream_ptr(stream)))
        return out

    def backward(self, dx, dy, g_alpha1, g_alpha2, origin=(0.0, 0.0), flags: int = 0,
                 grads=None, g_halos=None, stream=None):
        """Accumulate dL/d(m, x, y, size) of every particle ((n, 4) per
        species, input order) and, when g_halos is an (n_halos, 5) float64
        CUDA tensor, dL/d(m or r_E, x, y, p0, p1) of every halo."""
        torch = _torch()
        n = dx.numel()
        if dy.numel() != n or dx.dtype != dy.dtype or dx.dtype not in (torch.float32, torch.float64):
            raise ValueError("dx, dy must be float32 or float64 of the same size")
        for g in (g_alpha1, g_alpha2):
            if g.dtype != self.out_dtype or g.numel() < n:
                raise ValueError(f"upstream gradients must be {self.out_dtype} with n elements")
        if grads is None:
            grads = [torch.zeros(s.data.shape[0], 4, dtype=self.out_dtype, device="cuda")
                     for s in self.species]
        for s, g in zip(self.species, grads):
            if g.dtype != self.out_dtype or g.numel() < 4 * s.data.shape[0]:
                raise ValueError(f"species gradients must be ({s.data.shape[0]}, 4) {self.out_dtype}")
        if g_halos is not None and (g_halos.dtype != torch.float64 or g_halos.numel() < 5 * self.n_halos):
            raise ValueError(f"g_halos must be ({self.n_halos}, 5) float64")
        arr = (ctypes.c_void_p * max(1, len(grads)))(*[g.data_ptr() for g in grads])
        rd = F32 if dx.dtype == torch.float32 else F64
        _check(lib().lens_shoot_rays_backward(
            self._h, float(origin[0]), float(origin[1]), _dev_ptr(dx), _dev_ptr(dy), rd, n,
            _dev_ptr(g_alpha1), _dev_ptr(g_alpha2), None, None, None, arr,
            _dev_ptr(g_halos) if g_halos is not None else None, int(flags), _stream_ptr(stream)))
        return grads

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.lens_free_tree(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_peak(iters: int = 4096, stream=None) -> float:
    """Measured FP32 FFMA rate of the current GPU (FLOP/s)."""
    v = ctypes.c_double()
    _check(lib().lens_fp32_peak(int(iters), ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def fp64_peak(iters: int = 1024, stream=None) -> float:
    """Measured FP64 DFMA rate of the current GPU (FLOP/s)."""
    v = ctypes.c_double()
    _check(lib().lens_fp64_peak(int(iters), ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def fail_allocations(after: int):
    """Failure injection for error-path tests (lens_fail_allocations): the
    library's next `after` device allocations succeed and the following one
    fails as out of memory; a negative value turns the hook off."""
    lib().lens_fail_allocations(int(after))


def refine_cells(x0, y0, h, nx, ny, alpha1, alpha2, kappa=None, gamma1=None, gamma2=None, cells=None,
                 k: int = 3, tol: float = 1e-4, mode: int = REFINE_KAPPA_GAMMA, n_nonuniform=None,
                 out=None, stream=None):
    """lens_refine_cells on device tensors (grid arrays of nx*ny; cells: int64
    flat indices, default every interior ray).  Returns (uniform uint8 (n,),
    amat float32 (n, 4): a11, a21, a12, a22, y_sub float64 (n, k, k, 2)),
    written into `out` (that triple) when given."""
    torch = _torch()
    dev = alpha1.device
    n = cells.numel() if cells is not None else (nx - 2) * (ny - 2)  # None: every interior cell, row-major
    if out is not None:
        uniform, amat, y_sub = out
        if uniform.numel() < n or amat.numel() < 4 * n or y_sub.numel() < 2 * k * k * n:
            raise ValueError("refine outputs too small")
    else:
        uniform = torch.empty(n, dtype=torch.uint8, device=dev)
        amat = torch.empty(n, 4, dtype=torch.float32, device=dev)
        y_sub = torch.empty(n, k, k, 2, dtype=torch.float64, device=dev)
    ad = F32 if alpha1.dtype == torch.float32 else F64
    for t in (kappa, gamma1, gamma2):
        if t is not None and t.dtype != torch.float32:
            raise ValueError("kappa and gamma must be float32")
    _check(lib().lens_refine_cells(float(x0), float(y0), float(h), int(nx), int(ny), _dev_ptr(alpha1),
                                   _dev_ptr(alpha2), ad, _dev_ptr(kappa) if kappa is not None else None,
                                   _dev_ptr(gamma1) if gamma1 is not None else None,
                                   _dev_ptr(gamma2) if gamma2 is not None else None,
                                   _dev_ptr(cells) if cells is not None else None, n,
                                   int(k), float(tol), int(mode), _dev_ptr(uniform), _dev_ptr(amat),
                                   _dev_ptr(y_sub), _dev_ptr(n_nonuniform) if n_nonuniform is not None
                                   else None, _stream_ptr(stream)))
    return uniform, amat, y_sub


def smoothing_lengths(xyz, k: int = 32, out=None, stream=None):
    """Distance from every particle to its k-th nearest other particle in 3D
    (lens_smoothing_lengths): xyz a (n, 3) float32 CUDA tensor; returns (n,)
    float32 (written into `out` when given)."""
    torch = _torch()
    if xyz.dim() != 2 or xyz.shape[1] != 3 or xyz.dtype != torch.float32:
        raise ValueError("xyz must be (n, 3) float32")
    n = xyz.shape[0]
    r = out if out is not None else torch.empty(n, dtype=torch.float32, device=xyz.device)
    _check(lib().lens_smoothing_lengths(_dev_ptr(xyz), n, int(k), _dev_ptr(r), _stream_ptr(stream)))
    return r


def shoot(lens: Lens, dx, dy, origin=(0.0, 0.0), species_data=None):
    """Differentiable alpha (n, 2) through lens_shoot_rays / _backward: the
    gradient flows to the (n, 4) species tensors' columns (x, y, m and the
    size r_sm or r_s).  If ``species_data`` is not what the tree was built
    from, or was changed in place since, the tree is rebuilt from its current
    values first."""
    from ._autograd import shoot_alpha
    return shoot_alpha(lens, dx, dy, origin, species_data)
