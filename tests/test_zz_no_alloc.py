"""ag_vertex_normals_noalloc: vertex normals for callers that cannot allocate
device memory (a host application that owns the device-memory budget, a
plugin that must not touch the CUDA allocator, a latency-critical loop).  The
call's scratch is a static array inside the library, so the only memory it
touches is the caller's three buffers and that array.

Checked through the C ABI against the normals the existing entry point
(ag_bvh_build, read back with ag_bvh_copy_out) computes for the same mesh,
on two calls in a row: a larger mesh first, then a smaller one, so stale
adjacency left in the shared array by the first call would show up in the
second.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2605_26137_b300 import _lib, synth

pytestmark = pytest.mark.gpu

TOL = 1e-6  # same bound the BVH-structure test puts on these normals


def _noalloc(lib):
    fn = lib.ag_vertex_normals_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    return fn


def _existing_normals(V, F):
    import paper_2605_26137_b300 as pb
    bvh = pb.Bvh(V, F)
    _, _, _, vn = bvh.copy_out()
    bvh.free()
    return vn


def test_noalloc_normals_match_existing_entry_point_twice():
    lib = _lib.load()
    fn = _noalloc(lib)
    stream = torch.cuda.current_stream().cuda_stream
    meshes = [synth.sdf_mesh(synth.sdf_union_params(21, 12), 40, device="cuda"),   # larger first
              synth.sh_displaced_sphere(3, 4)]                                       # then smaller
    for hv, hf in meshes:
        assert len(hv) <= 1 << 17 and len(hf) <= 1 << 18
        V = torch.from_numpy(np.ascontiguousarray(hv)).cuda()
        F = torch.from_numpy(np.ascontiguousarray(hf)).cuda()
        out = torch.full((len(hv), 4), float("nan"), dtype=torch.float32, device="cuda")
        st = fn(V.data_ptr(), len(hv), F.data_ptr(), len(hf), out.data_ptr(), stream)
        assert st == _lib.AG_OK, lib.ag_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _existing_normals(V, F)
        assert np.abs(got - ref).max() <= TOL


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    lib = _lib.load()
    fn = _noalloc(lib)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = fn(buf.data_ptr(), (1 << 17) + 1, buf.data_ptr(), 1, buf.data_ptr(), None)
    assert st == _lib.AG_ERR_INVALID_ARG
    assert b"static scratch limit" in lib.ag_last_error()
    st = fn(buf.data_ptr(), 3, buf.data_ptr(), (1 << 18) + 1, buf.data_ptr(), None)
    assert st == _lib.AG_ERR_INVALID_ARG
