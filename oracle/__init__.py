"""FP64 CPU oracle for the tangent-space normal bake (Sec. 6.4).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_2605_26137_b300``): the two meet
only in the seeded input generators (``paper_2605_26137_b300.synth``), which
hold none of the baking arithmetic.

The arithmetic lives in ``oracle.c`` (plain C, double precision, compiled
with -ffp-contract=off); this module only marshals numpy arrays.

Pins (see tests/test_oracle_*.py): every function here is checked against
closed forms, brute force or invariants that a wrong sign, index or dropped
term would break.  No function of the oracle is left unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # AG_ORACLE_LIB (tests only): load another build of oracle.c, e.g. one
        # with a planted mistake, to show that the pins catch it
        path = os.environ.get("AG_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        lib.or_vertex_normals.argtypes = [_P, _I64, _P, _I64, _P]
        lib.or_vertex_normals.restype = None
        lib.or_snap.argtypes = [ctypes.c_float, _I]
        lib.or_snap.restype = _I64
        lib.or_raster.argtypes = [_P, _I64, _I, _I, _I, _P, _P, _P]
        lib.or_raster.restype = _I
        lib.or_face_frames.argtypes = [_P, _P, _I64, _P, _I, _I, _P, _P, _P, _P]
        lib.or_face_frames.restype = None
        lib.or_bvh_build.argtypes = [_P, _P, _I64]
        lib.or_bvh_build.restype = _P
        lib.or_bvh_free.argtypes = [_P]
        lib.or_bvh_free.restype = None
        lib.or_closest_hit.argtypes = [_P, _P, _I64, _P, _P, _P, _D, _P]
        lib.or_closest_hit.restype = _I
        lib.or_closest_point.argtypes = [_P, _P, _I64, _P, _P, _D, _P]
        lib.or_closest_point.restype = _I
        lib.or_trace.argtypes = [_P, _I64, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                 _I, _I, _D, _D, _P, _I64, _I, _P, _P, _P, _P, _P, _P, _P, _I, _P]
        lib.or_trace.restype = _I
        lib.or_normal_map_error.argtypes = [_P, _I64, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _P,
                                            _P, _P, _I64, _D, _D, _I, _P, _P]
        lib.or_normal_map_error.restype = _I
        lib.or_encode.argtypes = [_P, _P, _I64, _P]
        lib.or_encode.restype = None
        lib.or_dilate.argtypes = [_I, _I, _I, _P, _P, _P]
        lib.or_dilate.restype = _I
        lib.or_loss_grad.argtypes = [_P, _P, _P, _P, _I64, _P, _I64, _P, _P, _P, _I64, _D, _P]
        lib.or_loss_grad.restype = _D
        lib.or_view_basis.argtypes = [_I, _I, _P]
        lib.or_view_basis.restype = None
        lib.or_visibility.argtypes = [_P, _P, _I64, _P, _I, _I, _D, _I, _P, _P, _P, _P, _P, _P, _P, _I64]
        lib.or_visibility.restype = _I
        lib.or_exterior_fill.argtypes = [_P, _P, _I64, _I64, _P, _P]
        lib.or_exterior_fill.restype = _I
        lib.or_qem_simplify.argtypes = [_P, _I64, _P, _I64, _I64, _P, _P, _I, _P, _I]
        lib.or_qem_simplify.restype = _I
        lib.or_render_view.argtypes = [_P, _P, _I64, _P, _P, _I, _I, _D, _P, _P, _P]
        lib.or_render_view.restype = _I
        lib.or_edge_mask.argtypes = [_P, _P, _I, _I, _D, _P]
        lib.or_edge_mask.restype = _I
        lib.or_backproject.argtypes = [_P, _I64, _P, _I64, _P, _P, _P, _P, _I, _I, _I, _P, _P, _I, _I, _P, _P, _P,
                                       _P, _D, _D, _D, _D, _D, _I, _D, _I, _D, _P, _P, _P, _P, _P, _I64, _I64,
                                       _P, _P, _P, _P]
        lib.or_mip_levels.argtypes = [_P, _I, _I, _D, _P, _P, _P]
        lib.or_mip_levels.restype = _I
        lib.or_backproject.restype = _I
        lib.or_qem_face_quadric.argtypes = [_P, _P]
        lib.or_qem_face_quadric.restype = None
        lib.or_qem_eval.argtypes = [_P, _P]
        lib.or_qem_eval.restype = _D
        lib.or_qem_place.argtypes = [_P, _P, _P, _P]
        lib.or_qem_place.restype = _D
        _lib = lib
        return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data


# ----------------------------------------------------------------- pieces

def vertex_normals(V, F):
    """Area-weighted unit vertex normals, FP64 [nv,3]."""
    lib = _load()
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    N = np.zeros((len(V), 3), np.float64)
    lib.or_vertex_normals(_p(V), len(V), _p(F), len(F), _p(N))
    return N


def snap(u: float, W: int) -> int:
    return int(_load().or_snap(ctypes.c_float(u), W))


def raster(uv, W: int, H: int, brute: bool = False):
    """Texel -> (owning low face, barycentrics).  Returns (face i32 [H,W],
    bary f64 [H,W,3], a2 i64 [F]) with a2 = twice the signed UV area in
    snapped (1/256 texel) units."""
    lib = _load()
    uv = _c(uv, np.float32)
    nf = uv.shape[0]
    face = np.empty((H, W), np.int32)
    bary = np.empty((H, W, 3), np.float64)
    a2 = np.empty(nf, np.int64)
    if lib.or_raster(_p(uv), nf, W, H, int(brute), _p(face), _p(bary), _p(a2)) != 0:
        raise MemoryError("oracle raster: allocation failed")
    return face, bary, a2


def face_frames(V, F, uv, W, H, N):
    """Per-corner unit tangents [F,3,3], handedness [F], degenerate flag [F]."""
    lib = _load()
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    uv = _c(uv, np.float32)
    N = _c(N, np.float64)
    T = np.empty((len(F), 3, 3), np.float64)
    w = np.empty(len(F), np.float64)
    dg = np.empty(len(F), np.uint8)
    lib.or_face_frames(_p(V), _p(F), len(F), _p(uv), W, H, _p(N), _p(T), _p(w), _p(dg))
    return T, w, dg


class Bvh:
    """Median-split binary BVH over a triangle mesh (FP64 bounds)."""

    def __init__(self, V, F):
        self._lib = _load()
        self.V = _c(V, np.float32)
        self.F = _c(F, np.int32)
        self.h = self._lib.or_bvh_build(_p(self.V), _p(self.F), len(self.F))
        if not self.h:
            raise MemoryError("oracle BVH build failed")

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self._lib.or_bvh_free(h)


def closest_hit(V, F, o, d, tmax, bvh: Bvh | None = None):
    """Closest |t| hit of the line o + t d, |t| <= tmax.  Returns (tri, t, b[3])
    with tri = -1 on a miss."""
    lib = _load()
    if bvh is not None:
        V, F = bvh.V, bvh.F
    else:
        V, F = _c(V, np.float32), _c(F, np.int32)
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    out = np.zeros(5, np.float64)
    lib.or_closest_hit(_p(V), _p(F), len(F), bvh.h if bvh is not None else None, _p(o), _p(d), float(tmax), _p(out))
    return int(out[0]), float(out[1]), out[2:5].copy()


def closest_point(V, F, p, rmax, bvh: Bvh | None = None):
    """Closest point of the triangle mesh to p within distance rmax.
    Returns (tri, d2, x[3], b[3]) with tri = -1 when nothing is that close."""
    lib = _load()
    if bvh is not None:
        V, F = bvh.V, bvh.F
    else:
        V, F = _c(V, np.float32), _c(F, np.int32)
    p = _c(p, np.float64)
    out = np.zeros(8, np.float64)
    lib.or_closest_point(_p(V), _p(F), len(F), bvh.h if bvh is not None else None, _p(p), float(rmax), _p(out))
    return int(out[0]), float(out[1]), out[2:5].copy(), out[5:8].copy()


QUERIES = {"ray": 0, "closest": 1}


def encode(nts, filled):
    lib = _load()
    nts = _c(nts, np.float64)
    filled = _c(filled, np.uint8)
    n = filled.size
    rgba = np.empty(n * 4, np.uint8)
    lib.or_encode(_p(nts), _p(filled), n, _p(rgba))
    return rgba.reshape(filled.shape + (4,))


def dilate(W, H, gutter, filled, nts, disp):
    """In place on copies; returns (filled, nts, disp)."""
    lib = _load()
    filled = _c(filled, np.uint8).copy()
    nts = _c(nts, np.float64).copy()
    disp = _c(disp, np.float64).copy()
    if lib.or_dilate(W, H, gutter, _p(filled), _p(nts), _p(disp)) != 0:
        raise MemoryError("oracle dilate: allocation failed")
    return filled, nts, disp


# ----------------------------------------------------------------- full bake

def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def bake(high_v, high_f, low_v, low_f, low_uv, W, H, max_dist, gutter=2, *,
         diam=None, use_bvh=True, sample=None, nthreads=None, bvh: Bvh | None = None, query="ray",
         force=None):
    """The whole bake in FP64.  With ``sample`` (texel ids), only those texels
    are traced and dilation is skipped.  ``query`` is "ray" (the line along
    the texel normal) or "closest" (the nearest point of the high surface);
    ``hit_t`` is then the signed ray parameter or the signed distance.
    ``force`` ([H*W] int32, with ``sample``) evaluates the given triangle at
    each sampled texel instead of searching (see ``shade_given``).
    Returns a dict of numpy arrays."""
    lib = _load()
    hv = _c(high_v, np.float32)
    hf = _c(high_f, np.int32)
    lv = _c(low_v, np.float32)
    lf = _c(low_f, np.int32)
    luv = _c(low_uv, np.float32)
    if diam is None:
        diam = float(np.linalg.norm(hv.astype(np.float64).max(0) - hv.astype(np.float64).min(0)))
    hn = vertex_normals(hv, hf)
    ln = vertex_normals(lv, lf)
    face, bary, a2 = raster(luv, W, H)
    T, w, dg = face_frames(lv, lf, luv, W, H, ln)
    if use_bvh and bvh is None:
        bvh = Bvh(hv, hf)
    n = W * H
    mask = np.zeros(n, np.uint8)
    nts = np.zeros((n, 3), np.float64)
    nts[:, 2] = 1.0
    disp = np.zeros(n, np.float64)
    hit_tri = np.full(n, -1, np.int32)
    hit_t = np.zeros(n, np.float64)
    hit_b = np.zeros((n, 3), np.float64)
    flags = np.zeros(n, np.uint8)
    if sample is not None:
        texels = _c(sample, np.int64)
    else:
        texels = np.flatnonzero(face.reshape(-1) >= 0).astype(np.int64)
    nth = nthreads or default_threads()
    rc = lib.or_trace(_p(hv), len(hv), _p(hf), len(hf), _p(hn), bvh.h if use_bvh else None,
                      _p(lv), _p(lf), _p(ln), _p(luv), _p(T), _p(w), _p(dg),
                      _p(face), _p(bary), W, H, float(max_dist), float(diam),
                      _p(texels), len(texels), nth,
                      _p(mask), _p(nts), _p(disp), _p(hit_tri), _p(hit_t), _p(hit_b), _p(flags),
                      QUERIES[query], _p(force) if force is not None else None)
    if rc != 0:
        raise RuntimeError("oracle trace: thread start failed")
    filled = (face.reshape(-1) >= 0).astype(np.uint8)
    out = dict(face=face, bary=bary, a2=a2, degen=dg, tangents=T, wsign=w, low_normals=ln, high_normals=hn,
               mask=mask.reshape(H, W), hit_tri=hit_tri.reshape(H, W), hit_t=hit_t.reshape(H, W),
               hit_b=hit_b.reshape(H, W, 3), flags=flags.reshape(H, W), texels=texels, diam=diam)
    if sample is None:
        filled, nts, disp = dilate(W, H, gutter, filled, nts, disp)
    out["filled"] = filled.reshape(H, W)
    out["nts"] = nts.reshape(H, W, 3)
    out["disp"] = disp.reshape(H, W)
    out["rgba8"] = encode(nts, filled).reshape(H, W, 4)
    # binary16 straight from the FP64 value (IEEE round to nearest even)
    out["disp16"] = disp.astype(np.float16).reshape(H, W)
    return out


def shade_given(asset, texels, tris, query="ray"):
    """FP64 evaluation of one given high triangle per texel, for checking an
    answer where several are equally correct (two triangles within rounding
    of the closest hit).  Ray query: the line's crossing of the triangle's
    plane, with signed barycentrics (a triangle missed by a hair shows a
    slightly negative one); closest-point query: the triangle's nearest point.
    Returns (n_ts [n,3], t [n], barycentrics [n,3], valid [n])."""
    texels = np.asarray(texels, np.int64)
    force = np.full(asset.W * asset.H, -1, np.int32)
    force[texels] = np.asarray(tris, np.int32)
    r = bake_asset(asset, sample=texels, force=force, query=query, use_bvh=False)
    tri = r["hit_tri"].reshape(-1)[texels]
    return (r["nts"].reshape(-1, 3)[texels], r["hit_t"].reshape(-1)[texels], r["hit_b"].reshape(-1, 3)[texels],
            tri >= 0)


def normal_map_error(high_v, high_f, low_v, low_f, low_uv, W, H, rgba8, sample_face, sample_bary, max_dist, *,
                     diam=None, bvh: Bvh | None = None, use_bvh=True, nthreads=None):
    """The "baked mean" measure of Sec. 6.1 in FP64, per sample point of the
    low mesh (face id and barycentrics b1, b2 of corners 1 and 2): the angle
    in degrees between the normal the RGBA8 map gives there (decoded and
    taken to world space through the bake's tangent frame at the point; on a
    degenerate-UV face the interpolated low normal) and
    the raw mesh's smooth normal at its surface point nearest to the sample
    (-1 with none within max_dist).  Returns (angle [n], flags [n]); flag 1:
    two raw triangles within rounding of the nearest distance give different
    normals."""
    lib = _load()
    hv = _c(high_v, np.float32)
    hf = _c(high_f, np.int32)
    lv = _c(low_v, np.float32)
    lf = _c(low_f, np.int32)
    luv = _c(low_uv, np.float32)
    rgba = _c(rgba8, np.uint8)
    sf = _c(sample_face, np.int32)
    sb = _c(sample_bary, np.float64).reshape(-1, 2)
    if rgba.size != W * H * 4 or len(sb) != len(sf):
        raise ValueError("map or sample sizes do not match")
    if len(sf) and (sf.min() < 0 or sf.max() >= len(lf)):
        raise ValueError("sample face out of range")
    if diam is None:
        diam = float(np.linalg.norm(hv.astype(np.float64).max(0) - hv.astype(np.float64).min(0)))
    hn = vertex_normals(hv, hf)
    ln = vertex_normals(lv, lf)
    T, w, dg = face_frames(lv, lf, luv, W, H, ln)
    if use_bvh and bvh is None:
        bvh = Bvh(hv, hf)
    angle = np.zeros(len(sf), np.float64)
    flags = np.zeros(len(sf), np.uint8)
    rc = lib.or_normal_map_error(_p(hv), len(hv), _p(hf), len(hf), _p(hn), bvh.h if use_bvh else None,
                                 _p(lv), _p(lf), _p(ln), _p(luv), _p(_c(T, np.float64)), _p(_c(w, np.float64)),
                                 _p(_c(dg, np.uint8)), W, H, _p(rgba), _p(sf), _p(sb), len(sf), float(max_dist), float(diam),
                                 nthreads or default_threads(), _p(angle), _p(flags))
    if rc != 0:
        raise RuntimeError("oracle normal_map_error: thread start failed")
    return angle, flags


def bake_asset(asset, **kw):
    return bake(asset.high_v, asset.high_f, asset.low_v, asset.low_f, asset.low_uv,
                asset.W, asset.H, asset.max_dist, asset.gutter, diam=asset.diam, **kw)


# ----------------------------------------------------------------- loss / gradient

def loss_grad(high_v, high_f, high_normals, low_v64, low_f, face, bary, hit_tri, lam, want_grad=True):
    """Baking loss over hit texels with hit triangles held fixed, and its
    analytic gradient w.r.t. the low positions (FP64)."""
    lib = _load()
    hv = _c(high_v, np.float32)
    hf = _c(high_f, np.int32)
    hn = _c(high_normals, np.float64)
    lv = _c(low_v64, np.float64)
    lf = _c(low_f, np.int32)
    face = _c(face, np.int32).reshape(-1)
    bary = _c(bary, np.float64).reshape(-1, 3)
    hit_tri = _c(hit_tri, np.int32).reshape(-1)
    g = np.zeros(lv.shape, np.float64) if want_grad else None
    L = lib.or_loss_grad(_p(hv), _p(hf), _p(hn), _p(lv), len(lv), _p(lf), len(lf),
                         _p(face), _p(bary), _p(hit_tri), len(face), float(lam), _p(g))
    return L, g


def fd_grad(high_v, high_f, high_normals, low_v64, low_f, face, bary, hit_tri, lam, h=1e-4, coords=None):
    """Central finite differences (FP64, step h) of the fixed-hit loss."""
    lv = np.array(low_v64, dtype=np.float64)
    g = np.zeros_like(lv)
    idx = range(lv.size) if coords is None else coords
    flat = lv.reshape(-1)
    for c in idx:
        old = flat[c]
        flat[c] = old + h
        lp, _ = loss_grad(high_v, high_f, high_normals, lv, low_f, face, bary, hit_tri, lam, False)
        flat[c] = old - h
        lm, _ = loss_grad(high_v, high_f, high_normals, lv, low_f, face, bary, hit_tri, lam, False)
        flat[c] = old
        g.reshape(-1)[c] = (lp - lm) / (2 * h)
    return g


# ----------------------------------------------------------------- hidden-face removal (Sec. 6.2)

MAX_CAND = 16


def view_basis(k: int, n: int):
    """View k of n: (u, e1, e2), u on the Fibonacci lattice, rays along -u."""
    out = np.zeros(9, np.float64)
    _load().or_view_basis(k, n, _p(out))
    return out[:3].copy(), out[3:6].copy(), out[6:].copy()


def visibility(V, F, n_views: int, res: int, *, tol_rel: float = 1e-5, candidates: bool = True,
               bvh: Bvh | None = None, use_bvh: bool = True, nthreads=None, sample=None):
    """Per-face visibility from n_views orthographic res x res views.
    Returns a dict: visible [nf] u8, hit [n_views, res, res] i32 (-1 miss),
    and with ``candidates`` ncand [n_views, res, res], cand [..., 16] (faces
    within tol_rel*R of the ray, no farther than its first hit + tol_rel*R;
    -1 padded, ncand > 16 means the list is truncated), edge_near (the hit
    point within tol_rel*R of its triangle's boundary); frame = (c, R).
    With ``sample`` (ray ids view*res*res + j*res + i) only those rays are
    traced; the per-ray arrays are then flat, in sample order."""
    lib = _load()
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    if use_bvh and bvh is None:
        bvh = Bvh(V, F)
    nf = len(F)
    samp = None if sample is None else _c(sample, np.int64)
    nr = n_views * res * res if samp is None else len(samp)
    visible = np.zeros(nf, np.uint8)
    hit = np.empty(nr, np.int32)
    ncand = np.zeros(nr, np.int32) if candidates else None
    cand = np.full(nr * MAX_CAND, -1, np.int32) if candidates else None
    near = np.zeros(nr, np.uint8) if candidates else None
    frame = np.zeros(4, np.float64)
    rc = lib.or_visibility(_p(V), _p(F), nf, bvh.h if use_bvh else None, n_views, res, float(tol_rel),
                           nthreads or default_threads(), _p(visible), _p(hit), _p(ncand), _p(cand), _p(near),
                           _p(frame), _p(samp), 0 if samp is None else len(samp))
    if rc != 0:
        raise RuntimeError("oracle visibility: thread start failed")
    shape = (n_views, res, res) if samp is None else (len(samp),)
    out = dict(visible=visible, hit=hit.reshape(shape), frame=(frame[:3].copy(), float(frame[3])))
    if candidates:
        out.update(ncand=ncand.reshape(shape), cand=cand.reshape(shape + (MAX_CAND,)),
                   edge_near=near.reshape(shape))
    return out


def exterior_fill(V, F, visible, nv=None):
    """Exterior faces [nf] u8: every face linked to a visible face through
    edge-adjacent faces whose normals have a positive dot product."""
    lib = _load()
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    vis = _c(visible, np.uint8)
    ext = np.zeros(len(F), np.uint8)
    if lib.or_exterior_fill(_p(V), _p(F), nv if nv is not None else len(V), len(F), _p(vis), _p(ext)) != 0:
        raise MemoryError("oracle exterior fill: allocation failed")
    return ext


# ----------------------------------------------------------------- QEM simplification (Sec. 6.1)

def qem_face_quadric(P):
    """The 10 unique entries (q00 q01 q02 q03 q11 q12 q13 q22 q23 q33) of the
    plane quadric of triangle P [3,3]."""
    q = np.zeros(10, np.float64)
    _load().or_qem_face_quadric(_p(_c(P, np.float64)), _p(q))
    return q


def qem_eval(q, v) -> float:
    return float(_load().or_qem_eval(_p(_c(q, np.float64)), _p(_c(v, np.float64))))


def qem_place(q, v0, v1):
    """Edge parameter t of the paper's placement and the singular flag."""
    sing = ctypes.c_int()
    t = _load().or_qem_place(_p(_c(q, np.float64)), _p(_c(v0, np.float64)), _p(_c(v1, np.float64)),
                             ctypes.byref(sing))
    return float(t), bool(sing.value)


def qem_simplify(V, F, target: int, max_rounds: int = 100000, midpoint: bool = False):
    """Simplify to at most ``target`` faces.  Returns a dict: V (float64, the
    surviving vertices in increasing original id), F (renumbered, surviving
    faces in increasing original id), keep_v / keep_f (original ids),
    rounds, and per round the alive face count and the number of collapses."""
    lib = _load()
    V64 = np.array(V, dtype=np.float64, order="C")
    F32 = np.array(F, dtype=np.int32, order="C")
    nv, nf = len(V64), len(F32)
    va = np.zeros(nv, np.uint8)
    fa = np.zeros(nf, np.uint8)
    stats = np.zeros(2 * max_rounds, np.int64)
    r = lib.or_qem_simplify(_p(V64), nv, _p(F32), nf, int(target), _p(va), _p(fa), max_rounds, _p(stats),
                            int(bool(midpoint)))
    if r < 0:
        raise MemoryError("oracle QEM: allocation failed")
    keep_v = np.flatnonzero(va)
    keep_f = np.flatnonzero(fa)
    new_id = np.full(nv, -1, np.int64)
    new_id[keep_v] = np.arange(len(keep_v))
    Fo = new_id[F32[keep_f]].astype(np.int32)
    return dict(V=V64[keep_v], F=Fo, keep_v=keep_v, keep_f=keep_f, rounds=r,
                alive=stats[0:2 * r:2].copy(), collapses=stats[1:2 * r:2].copy())


# ----------------------------------------------------------------- UV-space backprojection (Sec. 7.4)

def render_views(V, F, cams, w: int, h: int, *, tol_rel: float = 1e-5, bvh: Bvh | None = None):
    """Depth [K,h,w] (camera z of the first hit, +inf on a miss), world points
    [K,h,w,3] (NaN on a miss) and near-edge flags [K,h,w] of K pinhole
    views (cams [K,16] f32: R row-major, t, fx, fy, cx, cy)."""
    lib = _load()
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    if bvh is None:
        bvh = Bvh(V, F)
    Vd = V.astype(np.float64)
    scale = float(np.linalg.norm(Vd.max(0) - Vd.min(0)))
    cams = _c(cams, np.float32).reshape(-1, 16)
    K = len(cams)
    depth = np.empty((K, h, w), np.float64)
    point = np.empty((K, h, w, 3), np.float64)
    near = np.empty((K, h, w), np.uint8)
    for k in range(K):
        lib.or_render_view(_p(V), _p(F), len(F), bvh.h, _p(cams[k]), w, h, tol_rel * scale,
                           _p(depth[k]), _p(point[k]), _p(near[k]))
    return depth, point, near


def edge_mask(depth, point, edge_tol: float):
    """Edge pixels [K,h,w] u8 of rendered views (depth [K,h,w], point
    [K,h,w,3]): a hit with a 4-neighbour that misses or whose world point
    lies farther than edge_tol from its own."""
    lib = _load()
    depth = _c(depth, np.float64)
    point = _c(point, np.float64)
    K, h, w = depth.shape
    edge = np.empty((K, h, w), np.uint8)
    for k in range(K):
        lib.or_edge_mask(_p(depth[k]), _p(point[k]), w, h, float(edge_tol), _p(edge[k]))
    return edge


def mip_levels(img, sharpen: float = 0.25):
    """Levels 1.. of one RGBA8 image's Lanczos-2 pyramid (the anisotropic
    filter's), each as ([h,w,3] unsharpened, [h,w,3] sharpened)."""
    lib = _load()
    img = _c(img, np.uint8)
    h, w = img.shape[:2]
    tot = 3 * sum(max(1, w >> l) * max(1, h >> l) for l in range(1, 17))
    plain = np.zeros(tot, np.float64)
    sharp = np.zeros(tot, np.float64)
    dims = np.zeros(32, np.int32)
    n = lib.or_mip_levels(_p(img), w, h, float(sharpen), _p(plain), _p(sharp), _p(dims))
    if n < 0:
        raise MemoryError("or_mip_levels failed")
    out, off = [], 0
    for l in range(n - 1):
        lw, lh = int(dims[2 * l]), int(dims[2 * l + 1])
        k = 3 * lw * lh
        out.append((plain[off:off + k].reshape(lh, lw, 3), sharp[off:off + k].reshape(lh, lw, 3)))
        off += k
    return out


def backproject(lv, lf, luv, W: int, H: int, cams, images, weights, *, alpha: float, eps: float,
                depth_tol: float, edge_tol: float, views=None, tol_rel: float = 1e-5, filter: str = "aniso",
                lod_bias: float = -0.5, max_taps: int = 8, sharpen: float = 0.25, sample=None,
                variants: bool = False):
    """Texture [H,W,3] (FP64), filled [H,W], flags [H,W] and incidence
    [K,H,W] of the blended backprojection of K views onto the low mesh's
    atlas.  ``views`` = (depth, point, near) from render_views, rendered here
    when None.  filter: "aniso" (footprint taps over a Lanczos-2 pyramid) or
    "bilinear" (one sample).  ``sample`` (texel ids): only those texels.
    ``variants``: for every flagged texel, the set of correct results
    ("variants": {texel: array [n, 4] of rgb + filled}, an empty array when
    there are too many to list)."""
    lib = _load()
    lv = _c(lv, np.float32)
    lf = _c(lf, np.int32)
    luv = _c(luv, np.float32)
    cams = _c(cams, np.float32).reshape(-1, 16)
    images = _c(images, np.uint8)
    K, ih, iw = images.shape[0], images.shape[1], images.shape[2]
    weights = _c(weights, np.float32)
    if views is None:
        views = render_views(lv, lf, cams, iw, ih, tol_rel=tol_rel)
    depth, point, near = (_c(views[0], np.float64), _c(views[1], np.float64), _c(views[2], np.uint8))
    face, bary, _ = raster(luv, W, H)
    ln = vertex_normals(lv, lf)
    Vd = lv.astype(np.float64)
    scale = float(np.linalg.norm(Vd.max(0) - Vd.min(0)))
    tex = np.zeros((H, W, 3), np.float64)
    filled = np.zeros((H, W), np.uint8)
    flags = np.zeros((H, W), np.uint8)
    incid = np.zeros((K, H, W), np.float64)
    texels = None if sample is None else _c(sample, np.int64)
    max_var = 0
    if variants:
        max_var = len(texels) if texels is not None else int((face >= 0).sum())
    var_tex = np.zeros(max(max_var, 1), np.int64)
    var_n = np.zeros(max(max_var, 1), np.uint8)
    var_rgbf = np.zeros((max(max_var, 1), 64, 4), np.float64)
    n_var = np.zeros(1, np.int64)
    rc = lib.or_backproject(_p(lv), len(lv), _p(lf), len(lf), _p(ln), _p(luv), _p(face), _p(bary), W, H, K,
                            _p(cams), _p(images), iw, ih, _p(depth), _p(point), _p(near), _p(weights), float(alpha),
                            float(eps), float(depth_tol), float(edge_tol), scale,
                            {"bilinear": 0, "aniso": 1}[filter], float(lod_bias), int(max_taps), float(sharpen),
                            _p(tex), _p(filled), _p(flags), _p(incid), _p(texels),
                            0 if texels is None else len(texels), max_var,
                            _p(var_tex) if variants else None, _p(var_n), _p(var_rgbf), _p(n_var))
    if rc != 0:
        raise MemoryError("or_backproject failed")
    out = dict(texture=tex, filled=filled, flags=flags, incidence=incid, face=face, bary=bary,
               depth=depth, point=point, near=near)
    if variants:
        out["variants"] = {int(var_tex[j]): var_rgbf[j, :var_n[j]].copy() for j in range(int(n_var[0]))}
    return out
