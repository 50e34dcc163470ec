"""The C ABI without a GPU: liblens loads, exports every function that
include/lens.h declares, and rejects bad arguments with a status code before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_1128_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    with open(os.path.join(ROOT, "include", "lens.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lens_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_status_strings(lib):
    lib.lens_api_version.restype = ctypes.c_int32
    assert lib.lens_api_version() == 2
    lib.lens_status_string.restype = ctypes.c_char_p
    lib.lens_status_string.argtypes = [ctypes.c_int]
    assert lib.lens_status_string(0) == b"ok"
    assert lib.lens_status_string(1) == b"invalid argument"
    assert lib.lens_status_string(99) == b"unknown status"


def test_bad_arguments_return_status(lib):
    import paper_1312_1128_gb300 as L
    L.lib()  # sets argtypes
    lt = L.lib()
    h = ctypes.c_void_p()
    # NULL params
    assert lt.lens_build_tree(None, 0, None, 0, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    # negative theta, bad leaf size, unknown precision, unknown walk
    for th, leaf, prec, res in [(-1.0, 5, 0, 0), (0.1, 0, 0, 0), (0.1, 5, 7, 0), (0.1, 5, 0, 4), (0.1, 5, 0, -1)]:
        p = L._Params(th, leaf, prec, 0, res)
        assert lt.lens_build_tree(None, 0, None, 0, ctypes.byref(p), None, ctypes.byref(h)) == 1
    # unknown near-field tile
    p = L._Params(0.1, 5, 0, 0, 0, 3)
    assert lt.lens_build_tree(None, 0, None, 0, ctypes.byref(p), None, ctypes.byref(h)) == 1
    # unknown species kind
    sp = (L._Species * 1)(L._Species(9, 0, 10, 1, 3.0))
    p = L._Params(0.1, 5, 0, 0, 0)
    assert lt.lens_build_tree(sp, 1, None, 0, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert b"kind" in lt.lens_last_error()
    # a halo with a non-positive radius
    hs = (L._Halo * 1)(L._Halo(4, 0, 0.0, 0.0, 1.0, -1.0, 0.0))
    assert lt.lens_build_tree(None, 0, hs, 1, ctypes.byref(p), None, ctypes.byref(h)) == 1
    # shooting with a NULL tree
    assert lt.lens_shoot_rays(None, 0.0, 0.0, None, None, 0, 10, None, None, None, None, None, 0, None) == 1
    # batches: offsets must start at 0 and not decrease
    off = (ctypes.c_int64 * 3)(1, 2, 3)
    org = (ctypes.c_double * 4)(0, 0, 0, 0)
    assert lt.lens_shoot_batches(None, 2, off, org, None, None, 0, None, None, None, None, None, 0, None) == 1
    off = (ctypes.c_int64 * 3)(0, 5, 3)
    assert lt.lens_shoot_batches(None, 2, off, org, None, None, 0, None, None, None, None, None, 0, None) == 1
    # the wait limit needs a tree
    lt.lens_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lt.lens_set_wait_limit(None, 0) == 1
    # backward: kappa/gamma gradients are declared unsupported in this version
    assert lt.lens_shoot_rays_backward(None, 0.0, 0.0, None, None, 0, 1, None, None, None, None, None,
                                       None, None, 0, None) == 1


def test_refine_cells_argument_checks():
    """lens_refine_cells rejects bad arguments before touching the device;
    n_cells == 0 is a no-op (no device call)."""
    import paper_1312_1128_gb300 as L
    lt = L.lib()
    fake = ctypes.c_void_p(16)  # never dereferenced: every case fails or returns first

    def call(h=0.01, nx=8, ny=8, dtype=0, n=4, k=3, tol=1e-4, mode=0, arrays=True, kg=True):
        a = fake if arrays else None
        g = fake if kg else None
        return lt.lens_refine_cells(0.0, 0.0, h, nx, ny, a, a, dtype, g, g, g, a, n, k, tol, mode, a, a, a,
                                    None, None)

    assert call(n=0) == 0
    for kw in [dict(n=-1), dict(nx=2), dict(ny=2), dict(h=0.0), dict(h=float("nan")), dict(k=2), dict(k=0),
               dict(k=17), dict(tol=-1.0), dict(mode=5), dict(dtype=3), dict(arrays=False),
               dict(kg=False, mode=0)]:
        assert call(**kw) == 1, kw
    assert b"kappa" in lt.lens_last_error()


def test_smoothing_lengths_argument_checks():
    import paper_1312_1128_gb300 as L
    lt = L.lib()
    fake = ctypes.c_void_p(16)  # never dereferenced: every case fails or returns first
    assert lt.lens_smoothing_lengths(fake, 0, 32, fake, None) == 0
    for n, k, arr in [(100, 0, fake), (100, 65, fake), (-1, 8, fake), (32, 32, fake), (5, 32, fake),
                      (100, 8, None), (1 << 33, 8, fake)]:
        assert lt.lens_smoothing_lengths(arr, n, k, arr, None) == 1, (n, k)


def test_shoot_potential_argument_checks():
    """lens_shoot_potential rejects a NULL tree before anything else."""
    import paper_1312_1128_gb300 as L
    lt = L.lib()
    fake = ctypes.c_void_p(16)  # never dereferenced: every case fails first
    for flags in (0, 1, 8):
        assert lt.lens_shoot_potential(None, 0.0, 0.0, fake, fake, 0, 10, fake, None, None, flags, None) == 1
    assert b"tree" in lt.lens_last_error()


def test_find_images_argument_checks():
    """lens_find_images rejects bad parameters before touching the tree or the
    device."""
    import paper_1312_1128_gb300 as L
    lt = L.lib()
    cnt = ctypes.c_int32(7)
    assert lt.lens_find_images(None, None, 0, None, 0, None, ctypes.byref(cnt), None, None) == 1
    fake = ctypes.c_void_p(16)  # never dereferenced: every case fails first
    src = (ctypes.c_double * 3)(0.5, 0.0, 0.1)
    imgs = (L._Image * 4)()

    def call(n_src=1, s=src, **kw):
        p = dict(x0=-10.0, y0=-10.0, side=20.0, n=64, l_max=12, mu_min=0.01, f_area=5e-4, n_min=50,
                 max_rounds=0, max_cells=0)
        p.update(kw)
        prm = L._AmrParams(**p)
        return lt.lens_find_images(fake, ctypes.byref(prm), n_src, s, 4, imgs, ctypes.byref(cnt), None, None)

    assert call(n_src=0) == 0 and cnt.value == 0
    for kw in [dict(n=0), dict(n=5000), dict(l_max=-1), dict(l_max=20), dict(side=0.0), dict(side=float("nan")),
               dict(mu_min=0.0), dict(mu_min=1.5), dict(f_area=0.0), dict(n_min=-1), dict(n_src=-1),
               dict(n=4096, l_max=19), dict(max_cells=100)]:
        assert call(**kw) == 1, kw
    bad = (ctypes.c_double * 3)(0.5, 0.0, -1.0)
    assert call(s=bad) == 1
    assert b"radius" in lt.lens_last_error()
