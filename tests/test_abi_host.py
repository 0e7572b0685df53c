"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every symbol include/ag.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2605_26137_b300 import _lib
from paper_2605_26137_b300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build_cuda()
    return _lib.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                src = f.read()
            names |= set(re.findall(r"AG_API\s+[\w\s\*]+?\b(ag_\w+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 15
    assert names == set(_lib.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_version_and_status_strings(lib):
    assert lib.ag_version() >= 100
    assert lib.ag_status_string(_lib.AG_ERR_TRAVERSAL_LIMIT) == b"AG_ERR_TRAVERSAL_LIMIT"
    assert lib.ag_status_string(0) == b"AG_OK"


def test_opts_default(lib):
    o = _lib.default_opts()
    assert o.bvh_layout == _lib.AG_BVH_Q8 and o.gutter == 2 and o.disp_fp16 == 1
    assert o.schedule == _lib.AG_SCHED_AUTO and o.max_steps == 0
    assert o.query == _lib.AG_QUERY_RAY
    assert o.render == _lib.AG_RENDER_RASTER and o.filter == _lib.AG_FILTER_ANISO
    assert o.collapse == _lib.AG_COLLAPSE_SAH
    assert o.build_async == 0
    assert ctypes.sizeof(_lib.AgOpts) == 64   # 16 int32: query, render, filter, build_async took reserved slots
    assert _lib.AgOpts.render.offset == 40 and _lib.AgOpts.filter.offset == 44
    assert _lib.AgOpts.build_async.offset == 48


def test_host_argument_checks(lib):
    o = _lib.default_opts()
    h = ctypes.c_void_p()
    # NULL out / NULL inputs / bad sizes are rejected before any device call
    assert lib.ag_bvh_build(1, 3, 1, 1, ctypes.byref(o), None, None) == _lib.AG_ERR_INVALID_ARG
    assert lib.ag_bvh_build(None, 3, 1, 1, ctypes.byref(o), None, ctypes.byref(h)) == _lib.AG_ERR_INVALID_ARG
    assert b"non-NULL" in lib.ag_last_error()
    assert lib.ag_bvh_build(1, 2, 1, 1, ctypes.byref(o), None, ctypes.byref(h)) == _lib.AG_ERR_INVALID_ARG
    assert lib.ag_bvh_build(1, 3, 1, 0, ctypes.byref(o), None, ctypes.byref(h)) == _lib.AG_ERR_INVALID_ARG
    bad = _lib.default_opts(gutter=99)
    assert lib.ag_bvh_build(1, 3, 1, 1, ctypes.byref(bad), None, ctypes.byref(h)) == _lib.AG_ERR_INVALID_ARG
    assert b"gutter" in lib.ag_last_error()
    bad = _lib.default_opts(query=7)
    assert lib.ag_bvh_build(1, 3, 1, 1, ctypes.byref(bad), None, ctypes.byref(h)) == _lib.AG_ERR_INVALID_ARG
    assert b"query" in lib.ag_last_error()
    for field in ("render", "filter", "build_async"):
        bad = _lib.default_opts(**{field: 7})
        assert lib.ag_bvh_build(1, 3, 1, 1, ctypes.byref(bad), None, ctypes.byref(h)) == _lib.AG_ERR_INVALID_ARG
        assert field.encode() in lib.ag_last_error()
    # backprojection: RGBA8 images must be 4-byte aligned (checked before any device call)
    cams = (ctypes.c_float * 16)(*([1.0] * 16))
    wts = (ctypes.c_float * 1)(1.0)
    tex = ctypes.c_void_p(256)
    st = lib.ag_backproject(256, None, 256, 256, 3, 1, 8, 8, 1, cams, wts, 258, 256, 256, 4, 4, 1.0, 0.0, 0.01,
                            None, None, tex, None)
    assert st == _lib.AG_ERR_INVALID_ARG and b"aligned" in lib.ag_last_error()
    # bad handles
    assert lib.ag_bvh_free(None) == _lib.AG_OK
    info = _lib.AgBvhInfo()
    assert lib.ag_bvh_info(None, ctypes.byref(info)) == _lib.AG_ERR_BAD_HANDLE
    assert lib.ag_bake(None, 1, None, 1, 1, 3, 1, 8, 8, 0.1, None, None, 1, 1, 1, None) == _lib.AG_ERR_BAD_HANDLE
    assert lib.ag_bake_backward(None, 1, 1, 1, 3, 1, 8, 8, 0.1, 0.1, None, None, 1, 1) == _lib.AG_ERR_BAD_HANDLE
    assert lib.ag_batch_plan_launch(None, None) == _lib.AG_ERR_BAD_HANDLE
    assert lib.ag_batch_plan_free(None) == _lib.AG_OK
    assert lib.ag_bake_batch(0, None, None, None) == _lib.AG_ERR_INVALID_ARG


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()
