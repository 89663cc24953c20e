"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/sf.h declares; host-side validation paths need no device."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("sf_create", "sf_solve", "sf_solve_backward", "sf_destroy", "sf_get_status"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2510_09204_b300 import build
    path = build.build()
    L = ct.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), name
    from paper_2510_09204_b300 import EXPORTS
    assert sorted(EXPORTS) == declared_functions()


def test_bounds_checked_build_exports_the_same_symbols():
    from paper_2510_09204_b300 import build
    L = ct.CDLL(build.build_check())
    for name in declared_functions():
        assert hasattr(L, name), name
    L.sf_strerror.restype = ct.c_char_p
    assert L.sf_strerror(10).startswith(b"device-side bounds")


def test_strerror_and_version_need_no_device():
    from paper_2510_09204_b300 import lib
    L = lib()
    assert L.sf_strerror(0) == b"ok"
    assert L.sf_strerror(6).startswith(b"non-finite")
    assert L.sf_version() >= 100


def test_create_rejects_bad_descriptors_without_touching_the_device():
    from paper_2510_09204_b300 import sf
    L = sf.lib()
    shapes = (sf.sf_shape * 1)()
    shapes[0].n, shapes[0].n_obs, shapes[0].H = 4, 2, 50
    shapes[0].a = shapes[0].b = 0.5
    for ax in range(2):
        shapes[0].p_min[ax], shapes[0].p_max[ax] = -5.0, 5.0
    good = dict(n_d=2, n_xi=11, rho=0.3, precision=1, proj=0, n_refine=0, max_iters=10, ckpt_every=0, tol=1e-3,
                n_inst=1, cost=0, dt=0.1, n_bc=2)
    bad_cases = [dict(n_d=4), dict(n_xi=1), dict(rho=0.0), dict(rho=float("nan")), dict(precision=9), dict(n_inst=0),
                 dict(max_iters=-1), dict(n_bc=4), dict(n_bc=3, dt=0.0), dict(n_bc=3, n_xi=4)]
    for bad in bad_cases:
        kw = dict(good, **bad)
        d = sf.sf_desc(kw["n_d"], kw["n_xi"], kw["rho"], kw["precision"], kw["proj"], kw["n_refine"],
                       kw["max_iters"], kw["ckpt_every"], kw["tol"], kw["n_inst"], shapes, None, kw["cost"], kw["dt"],
                       kw["n_bc"])
        h = ct.c_void_p()
        assert L.sf_create(ct.byref(d), ct.byref(h)) == sf.SF_EINVAL, bad
    shapes[0].a = -1.0
    d = sf.sf_desc(2, 11, 0.3, 1, 0, 0, 10, 0, 1e-3, 1, shapes, None)
    h = ct.c_void_p()
    assert L.sf_create(ct.byref(d), ct.byref(h)) == sf.SF_EINVAL
    assert L.sf_solve(None, None, None, None, None, 0, None, None, None, None, None) == sf.SF_EINVAL
    assert L.sf_solve_backward(None, None, None, None, None, None, None, None, None) == sf.SF_EINVAL
