"""torch-facing wrappers of the C ABI (device memory and streams from torch;
every step of the bake runs in libagbake.so's kernels).

All tensors are CUDA tensors on the current device: vertices float32 [n,3],
faces int32 [m,3], per-corner UVs float32 [m,3,2].  Calls are ordered on the
current torch stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import AgAssetDesc, AgBakeAux, AgBvhInfo, check, default_opts

_LAYOUTS = {"q8": _lib.AG_BVH_Q8, "f32": _lib.AG_BVH_F32}
_SCHED = {"auto": _lib.AG_SCHED_AUTO, "batch": _lib.AG_SCHED_BATCH, "refill": _lib.AG_SCHED_REFILL,
          "coop4": _lib.AG_SCHED_COOP4, "coop8": _lib.AG_SCHED_COOP8, "coop2": _lib.AG_SCHED_COOP2}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _need(t: torch.Tensor, name: str, dtype, shape_tail=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} must have trailing shape {shape_tail}, got {tuple(t.shape)}")
    return t


_COLLAPSE = {"area_count": _lib.AG_COLLAPSE_AREA_COUNT, "area": _lib.AG_COLLAPSE_AREA, "count": _lib.AG_COLLAPSE_COUNT,
             "sah": _lib.AG_COLLAPSE_SAH}


_TILES = {"8x8": _lib.AG_TILE_8x8, "16x16": _lib.AG_TILE_16x16, "32x8": _lib.AG_TILE_32x8, "4x4": _lib.AG_TILE_4x4}


_QUERY = {"ray": _lib.AG_QUERY_RAY, "closest": _lib.AG_QUERY_CLOSEST}


def _opts(layout="q8", gutter=2, disp_fp16=True, schedule="auto", block_size=0, blocks_per_sm=0, max_steps=0,
          collapse="sah", ray_tile="8x8", query="ray", stack_limit=0):
    return default_opts(bvh_layout=_LAYOUTS[layout], gutter=gutter, disp_fp16=int(bool(disp_fp16)),
                        schedule=_SCHED[schedule] if isinstance(schedule, str) else schedule,
                        block_size=block_size, blocks_per_sm=blocks_per_sm, max_steps=max_steps,
                        collapse=_COLLAPSE[collapse],
                        ray_tile=_TILES[ray_tile] if isinstance(ray_tile, str) else ray_tile,
                        query=_QUERY[query] if isinstance(query, str) else query, stack_limit=stack_limit)


class Bvh:
    """8-wide BVH over a high-poly mesh (owns its device memory)."""

    def __init__(self, verts: torch.Tensor, faces: torch.Tensor, layout: str = "q8", stream=None,
                 collapse: str = "sah", async_build: bool = False):
        """async_build: return once the build is enqueued on the stream (no
        host round trip); the handle keeps verts and faces referenced until
        free(), and info() waits for the build the first time."""
        lib = _lib.load()
        _need(verts, "verts", torch.float32, (3,))
        _need(faces, "faces", torch.int32, (3,))
        h = ctypes.c_void_p()
        o = _opts(layout=layout, collapse=collapse)
        o.build_async = int(bool(async_build))
        check(lib.ag_bvh_build(verts.data_ptr(), verts.shape[0], faces.data_ptr(), faces.shape[0],
                               ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.layout = layout
        self._inputs = (verts, faces) if async_build else None

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("BVH has been freed")
        return self._h.value

    def info(self) -> dict:
        inf = AgBvhInfo()
        check(self._lib.ag_bvh_info(self.handle, ctypes.byref(inf)))
        return {"n_tris": inf.n_tris, "n_verts": inf.n_verts, "n_nodes": inf.n_nodes,
                "node_bytes": inf.node_bytes, "tri_bytes": inf.tri_bytes, "normal_bytes": inf.normal_bytes,
                "layout": inf.layout, "node_size": inf.node_size, "max_depth": inf.max_depth,
                "scene_lo": list(inf.scene_lo), "scene_hi": list(inf.scene_hi), "diam": inf.diam,
                "build_ms": inf.build_ms}

    def copy_out(self):
        """Host copies (numpy) of nodes (raw bytes), leaf-order triangle records
        [n,3,4] float32 (xyz + vertex index bits), original ids, vertex normals."""
        import numpy as np
        inf = self.info()
        nodes = np.empty(inf["node_bytes"], np.uint8)
        tris = np.empty((inf["n_tris"], 3, 4), np.float32)
        ids = np.empty(inf["n_tris"], np.int32)
        vn = np.empty((inf["n_verts"], 4), np.float32)
        check(self._lib.ag_bvh_copy_out(self.handle, nodes.ctypes.data, tris.ctypes.data, ids.ctypes.data,
                                        vn.ctypes.data))
        return nodes, tris, ids, vn

    def free(self, stream=None) -> None:
        """Release the handle: synchronously, or in the order of ``stream``
        (after the work already queued on it) when one is given."""
        if self._h:
            if stream is None:
                check(self._lib.ag_bvh_free(self._h))
            else:
                check(self._lib.ag_bvh_free_async(self._h, _stream(stream)))
            self._h = ctypes.c_void_p()
            self._inputs = None

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._lib.ag_bvh_free(self._h)
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


@dataclass
class BakeOutputs:
    normal_rgba8: torch.Tensor      # uint8 [H,W,4]
    mask: torch.Tensor              # uint8 [H,W]
    disp: torch.Tensor              # float16 or float32 [H,W]
    normal_ts: torch.Tensor | None = None   # float32 [H,W,3]
    disp_f32: torch.Tensor | None = None    # float32 [H,W]
    face: torch.Tensor | None = None        # int32 [H,W]
    bary: torch.Tensor | None = None        # float32 [H,W,3]
    hit_tri: torch.Tensor | None = None     # int32 [H,W]
    hit_t: torch.Tensor | None = None       # float32 [H,W]
    counters: torch.Tensor | None = None    # int64 [4]: rays, node visits, triangle tests, hits
    n_rays: torch.Tensor | None = None      # int32 [1]


def _check_low(low_verts, low_faces, low_uv, low_normals):
    _need(low_verts, "low_verts", torch.float32, (3,))
    _need(low_faces, "low_faces", torch.int32, (3,))
    _need(low_uv, "low_uv", torch.float32, (3, 2))
    if low_uv.shape[0] != low_faces.shape[0]:
        raise ValueError("low_uv must have one [3,2] entry per face")
    if low_normals is not None:
        _need(low_normals, "low_normals", torch.float32, (3,))
        if low_normals.shape[0] != low_verts.shape[0]:
            raise ValueError("low_normals must match low_verts")


def alloc_outputs(W: int, H: int, device, disp_fp16=True, aux=False, counters=False) -> BakeOutputs:
    out = BakeOutputs(torch.empty((H, W, 4), dtype=torch.uint8, device=device),
                      torch.empty((H, W), dtype=torch.uint8, device=device),
                      torch.empty((H, W), dtype=torch.float16 if disp_fp16 else torch.float32, device=device))
    if aux:
        out.normal_ts = torch.empty((H, W, 3), dtype=torch.float32, device=device)
        out.disp_f32 = torch.empty((H, W), dtype=torch.float32, device=device)
        out.face = torch.empty((H, W), dtype=torch.int32, device=device)
        out.bary = torch.empty((H, W, 3), dtype=torch.float32, device=device)
        out.hit_tri = torch.empty((H, W), dtype=torch.int32, device=device)
        out.hit_t = torch.empty((H, W), dtype=torch.float32, device=device)
        out.n_rays = torch.empty(1, dtype=torch.int32, device=device)
    if counters:
        out.counters = torch.zeros(4, dtype=torch.int64, device=device)
    return out


def _ptr(t):
    return None if t is None else t.data_ptr()


def bake(bvh: Bvh, low_verts, low_faces, low_uv, W: int, H: int, max_dist: float, *, low_normals=None,
         gutter: int = 2, disp_fp16: bool = True, aux: bool = False, counters: bool = False,
         out: BakeOutputs | None = None, schedule="auto", block_size=0, blocks_per_sm=0, max_steps=0,
         stream=None, events=None, ray_tile="8x8", query="ray", stack_limit=0) -> BakeOutputs:
    """One bake.  ``query`` is "ray" (the line along the texel normal) or
    "closest" (the nearest point of the high surface, Sec. 6.4 as worded).
    ``aux`` adds float tangent-space normals, raster and hit outputs (hit_t is
    the signed ray parameter or signed distance); ``counters`` selects the
    counting traversal build; ``events`` (4 torch.cuda.Event) are recorded
    before the raster, before and after the traversal and after the
    encoding.  ``stack_limit`` (with ``counters``; a test hook) caps the
    traversal stack so that an overflow can be provoked."""
    lib = _lib.load()
    _check_low(low_verts, low_faces, low_uv, low_normals)
    if out is None:
        out = alloc_outputs(W, H, low_verts.device, disp_fp16, aux, counters)
    o = _opts(gutter=gutter, disp_fp16=disp_fp16, schedule=schedule, block_size=block_size,
              blocks_per_sm=blocks_per_sm, max_steps=max_steps, ray_tile=ray_tile, query=query,
              stack_limit=stack_limit)
    ev = None
    if events is not None:
        if len(events) != 4:
            raise ValueError("events must hold 4 torch.cuda.Event")
        for e in events:
            if not e.cuda_event:   # torch creates the CUDA event lazily, on first record
                e.record()
        ev = (ctypes.c_void_p * 4)(*[e.cuda_event for e in events])
    ax = AgBakeAux(_ptr(out.normal_ts), _ptr(out.disp_f32), _ptr(out.face), _ptr(out.bary), _ptr(out.hit_tri),
                   _ptr(out.hit_t), _ptr(out.counters), _ptr(out.n_rays),
                   ctypes.cast(ev, ctypes.c_void_p) if ev is not None else None)
    check(lib.ag_bake(bvh.handle, low_verts.data_ptr(), _ptr(low_normals), low_uv.data_ptr(), low_faces.data_ptr(),
                      low_verts.shape[0], low_faces.shape[0], W, H, float(max_dist), ctypes.byref(o), _stream(stream),
                      out.normal_rgba8.data_ptr(), out.mask.data_ptr(), out.disp.data_ptr(), ctypes.byref(ax)))
    return out


def bake_backward(bvh: Bvh, low_verts, low_faces, low_uv, W: int, H: int, max_dist: float, lam: float, *,
                  want_loss=True, want_grad=True, stream=None, schedule="auto", block_size=0, blocks_per_sm=0):
    """(loss [1] float32 or None, dL/dV [n,3] float32 or None)."""
    lib = _lib.load()
    _check_low(low_verts, low_faces, low_uv, None)
    loss = torch.empty(1, dtype=torch.float32, device=low_verts.device) if want_loss else None
    grad = torch.empty_like(low_verts) if want_grad else None
    o = _opts(schedule=schedule, block_size=block_size, blocks_per_sm=blocks_per_sm)
    check(lib.ag_bake_backward(bvh.handle, low_verts.data_ptr(), low_uv.data_ptr(), low_faces.data_ptr(),
                               low_verts.shape[0], low_faces.shape[0], W, H, float(max_dist), float(lam),
                               ctypes.byref(o), _stream(stream), _ptr(loss), _ptr(grad)))
    return loss, grad


class BakeLoss(torch.autograd.Function):
    """L(low_verts) = mean_hit(t^2) + lam * mean_hit(1 - n_hit . d).
    Forward evaluates L with one traversal; backward recomputes the hits and
    runs the adjoint kernels (ag_bake_backward)."""

    @staticmethod
    def forward(ctx, low_verts, bvh, low_faces, low_uv, W, H, max_dist, lam):
        loss, _ = bake_backward(bvh, low_verts.detach().contiguous(), low_faces, low_uv, W, H, max_dist, lam,
                                want_grad=False)
        ctx.save_for_backward(low_verts)
        ctx.args = (bvh, low_faces, low_uv, W, H, max_dist, lam)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (low_verts,) = ctx.saved_tensors
        bvh, low_faces, low_uv, W, H, max_dist, lam = ctx.args
        _, grad = bake_backward(bvh, low_verts.detach().contiguous(), low_faces, low_uv, W, H, max_dist, lam,
                                want_loss=False)
        return grad * g, None, None, None, None, None, None, None


def bake_loss(bvh, low_verts, low_faces, low_uv, W, H, max_dist, lam):
    return BakeLoss.apply(low_verts, bvh, low_faces, low_uv, W, H, max_dist, lam)


@dataclass
class Asset:
    bvh: Bvh
    low_verts: torch.Tensor
    low_faces: torch.Tensor
    low_uv: torch.Tensor
    W: int
    H: int
    max_dist: float
    low_normals: torch.Tensor | None = None
    out: BakeOutputs | None = None


def _descs(assets, disp_fp16):
    arr = (AgAssetDesc * len(assets))()
    for i, a in enumerate(assets):
        _check_low(a.low_verts, a.low_faces, a.low_uv, a.low_normals)
        if a.out is None:
            a.out = alloc_outputs(a.W, a.H, a.low_verts.device, disp_fp16)
        arr[i] = AgAssetDesc(a.bvh.handle, a.low_verts.data_ptr(), _ptr(a.low_normals), a.low_uv.data_ptr(),
                             a.low_faces.data_ptr(), a.low_verts.shape[0], a.low_faces.shape[0], a.W, a.H,
                             float(a.max_dist), a.out.normal_rgba8.data_ptr(), a.out.mask.data_ptr(),
                             a.out.disp.data_ptr())
    return arr


def bake_batch(assets: list[Asset], *, gutter=2, disp_fp16=True, schedule="auto", block_size=0, blocks_per_sm=0,
               stream=None, ray_tile="8x8", query="ray"):
    lib = _lib.load()
    arr = _descs(assets, disp_fp16)
    o = _opts(gutter=gutter, disp_fp16=disp_fp16, schedule=schedule, block_size=block_size,
              blocks_per_sm=blocks_per_sm, ray_tile=ray_tile, query=query)
    check(lib.ag_bake_batch(len(assets), arr, ctypes.byref(o), _stream(stream)))
    return [a.out for a in assets]


class BatchPlan:
    """A batch captured once into a CUDA graph; ``launch`` replays it."""

    def __init__(self, assets: list[Asset], *, gutter=2, disp_fp16=True, schedule="auto", block_size=0,
                 blocks_per_sm=0, stream=None, ray_tile="8x8", query="ray"):
        self._lib = _lib.load()
        self.assets = assets
        arr = _descs(assets, disp_fp16)
        o = _opts(gutter=gutter, disp_fp16=disp_fp16, schedule=schedule, block_size=block_size,
                  blocks_per_sm=blocks_per_sm, ray_tile=ray_tile, query=query)
        h = ctypes.c_void_p()
        check(self._lib.ag_batch_plan_create(len(assets), arr, ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        check(self._lib.ag_batch_plan_launch(self._h, _stream(stream)))
        return [a.out for a in self.assets]

    def free(self):
        if self._h:
            check(self._lib.ag_batch_plan_free(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._lib.ag_batch_plan_free(self._h)
        except Exception:  # noqa: BLE001
            pass


# ----------------------------------------------------------------- hidden-face removal (Sec. 6.2)

def visibility(bvh: Bvh, n_views: int = 512, res: int = 1024, *, hit_ids: bool = False, counters: bool = False,
               block_size: int = 0, blocks_per_sm: int = 0, max_steps: int = 0, render: str = "raster", stream=None):
    """Per-face visibility of the mesh ``bvh`` was built on, from n_views
    orthographic res x res views on the Fibonacci lattice around it.
    Returns (visible u8 [n_faces], hit_ids int32 [n_views, res, res] or None,
    counters u64 [4] (rays, node visits, triangle tests, hits) or None).
    render: "raster" (z-buffer proposals confirmed by the ray test) or
    "trace" (every ray traced; always used with counters)."""
    lib = _lib.load()
    n = bvh.info()["n_tris"]
    dev = torch.device("cuda", torch.cuda.current_device())
    vis = torch.empty(n, dtype=torch.uint8, device=dev)
    hits = torch.empty((n_views, res, res), dtype=torch.int32, device=dev) if hit_ids else None
    cnt = torch.zeros(4, dtype=torch.int64, device=dev) if counters else None
    o = _opts(block_size=block_size, blocks_per_sm=blocks_per_sm, max_steps=max_steps)
    o.render = {"raster": _lib.AG_RENDER_RASTER, "trace": _lib.AG_RENDER_TRACE}[render]
    check(lib.ag_visibility(bvh.handle, n_views, res, ctypes.byref(o), _stream(stream), vis.data_ptr(), _ptr(hits),
                            _ptr(cnt)))
    return vis, hits, cnt


def exterior_fill(verts, faces, visible, *, stream=None):
    """Exterior faces (u8 [n_faces], 1 = keep) from a visibility mask by the
    normal-gated flood fill."""
    lib = _lib.load()
    _need(verts, "verts", torch.float32, (3,))
    _need(faces, "faces", torch.int32, (3,))
    _need(visible, "visible", torch.uint8)
    if visible.shape[0] != faces.shape[0]:
        raise ValueError("visible must have one entry per face")
    ext = torch.empty(faces.shape[0], dtype=torch.uint8, device=faces.device)
    check(lib.ag_exterior_fill(verts.data_ptr(), verts.shape[0], faces.data_ptr(), faces.shape[0],
                               visible.data_ptr(), _stream(stream), ext.data_ptr()))
    return ext


def hidden_faces(verts, faces, n_views: int = 512, res: int = 1024, *, stream=None, **kw):
    """Hidden-face removal in one call: (exterior u8 [n_faces], visible u8)."""
    bvh = Bvh(verts, faces, stream=stream)
    try:
        vis, _, _ = visibility(bvh, n_views, res, stream=stream, **kw)
        return exterior_fill(verts, faces, vis, stream=stream), vis
    finally:
        bvh.free()


# ----------------------------------------------------------------- QEM simplification (Sec. 6.1)

def qem_simplify(verts, faces, target: int, *, max_rounds: int = 0, placement: str = "optimal", stream=None):
    """Simplify to at most ``target`` faces.  ``placement`` is "optimal" (the
    paper's projected optimum) or "midpoint" (the baseline it improves on).
    Returns (verts f64 [n,3], faces i32 [m,3], keep_verts i32 [n] original
    ids, rounds)."""
    lib = _lib.load()
    _need(verts, "verts", torch.float32, (3,))
    _need(faces, "faces", torch.int32, (3,))
    vo = torch.empty((verts.shape[0], 3), dtype=torch.float64, device=verts.device)
    fo = torch.empty((faces.shape[0], 3), dtype=torch.int32, device=faces.device)
    keep = torch.empty(verts.shape[0], dtype=torch.int32, device=verts.device)
    res = (ctypes.c_int64 * 3)()
    mode = {"optimal": _lib.AG_QEM_OPTIMAL, "midpoint": _lib.AG_QEM_MIDPOINT}[placement]
    check(lib.ag_qem_simplify(verts.data_ptr(), verts.shape[0], faces.data_ptr(), faces.shape[0], int(target),
                              int(max_rounds), mode, _stream(stream), vo.data_ptr(), fo.data_ptr(), keep.data_ptr(),
                              res))
    n, m = int(res[0]), int(res[1])
    return vo[:n], fo[:m], keep[:n], int(res[2])


def point_distance(bvh: Bvh, points, max_dist: float, *, tri: bool = False, stream=None):
    """Distance from each point [n,3] f32 to the mesh ``bvh`` was built on
    (-1 where nothing lies within max_dist); with ``tri`` also the nearest
    triangle ids."""
    lib = _lib.load()
    _need(points, "points", torch.float32, (3,))
    d = torch.empty(points.shape[0], dtype=torch.float32, device=points.device)
    t = torch.empty(points.shape[0], dtype=torch.int32, device=points.device) if tri else None
    check(lib.ag_point_distance(bvh.handle, points.data_ptr(), points.shape[0], float(max_dist), None,
                                _stream(stream), d.data_ptr(), _ptr(t)))
    return (d, t) if tri else d


def normal_map_error(bvh: Bvh, low_verts, low_faces, low_uv, W: int, H: int, normal_rgba8, sample_face, sample_bary,
                     max_dist: float, *, stream=None):
    """The "baked mean" measure (Sec. 6.1) per sample point of the low mesh:
    the angle in degrees between the normal the RGBA8 map [H,W,4] gives at
    the point and the smooth normal of the mesh ``bvh`` was built on (the raw
    mesh) at its nearest point (-1 where none lies within max_dist).
    sample_face [n] i32 and sample_bary [n,2] f32 (b1, b2) place the samples."""
    lib = _lib.load()
    _check_low(low_verts, low_faces, low_uv, None)
    _need(normal_rgba8, "normal_rgba8", torch.uint8, (W, 4))
    _need(sample_face, "sample_face", torch.int32)
    _need(sample_bary, "sample_bary", torch.float32, (2,))
    if normal_rgba8.shape[0] != H or sample_bary.shape[0] != sample_face.shape[0]:
        raise ValueError("map or sample shapes do not match")
    ang = torch.empty(sample_face.shape[0], dtype=torch.float32, device=low_verts.device)
    check(lib.ag_normal_map_error(bvh.handle, low_verts.data_ptr(), low_uv.data_ptr(), low_faces.data_ptr(),
                                  low_verts.shape[0], low_faces.shape[0], W, H, normal_rgba8.data_ptr(),
                                  sample_face.data_ptr(), sample_bary.data_ptr(), sample_face.shape[0],
                                  float(max_dist), None, _stream(stream), ang.data_ptr()))
    return ang


# ----------------------------------------------------------------- UV-space backprojection (Sec. 7.4)

def render_views(bvh: Bvh, cams, w: int, h: int, *, edge_tol: float, points: bool = True, render: str = "raster",
                 stream=None):
    """Depth [K,h,w] f32 (+inf on a miss), world points [K,h,w,3] (NaN on a
    miss) and edge mask [K,h,w] u8 of K pinhole views (cams: host numpy
    [K,16] f32) of the mesh ``bvh`` was built on.  render: "raster"
    (z-buffer proposals confirmed by the ray test) or "trace" (every pixel
    traced)."""
    import numpy as np
    lib = _lib.load()
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    K = cams.shape[0]
    dev = torch.device("cuda", torch.cuda.current_device())
    depth = torch.empty((K, h, w), dtype=torch.float32, device=dev)
    pts = torch.empty((K, h, w, 3), dtype=torch.float32, device=dev) if points else None
    edge = torch.empty((K, h, w), dtype=torch.uint8, device=dev)
    o = default_opts(render={"raster": _lib.AG_RENDER_RASTER, "trace": _lib.AG_RENDER_TRACE}[render])
    check(lib.ag_render_views(bvh.handle, K, cams.ctypes.data, w, h, float(edge_tol), ctypes.byref(o), _stream(stream),
                              depth.data_ptr(), _ptr(pts), edge.data_ptr()))
    return depth, pts, edge


def backproject(low_verts, low_faces, low_uv, W: int, H: int, cams, weights, images, depth, edge, *,
                alpha: float, eps: float, depth_tol: float, low_normals=None, incidence: bool = False,
                filter: str = "aniso", ray_tile="8x8", stream=None):
    """Blended texture [H,W,4] f32 (RGB, 1 where filled) of K views (images
    [K,h,w,4] u8, depth / edge from render_views, cams [K,16] and weights [K]
    host numpy) on the low mesh's atlas; with ``incidence`` also [K,H,W].
    filter: "aniso" (footprint taps over each view's Lanczos-2 pyramid) or
    "bilinear" (one sample)."""
    import numpy as np
    lib = _lib.load()
    _check_low(low_verts, low_faces, low_uv, low_normals)
    _need(images, "images", torch.uint8, (4,))
    _need(depth, "depth", torch.float32)
    _need(edge, "edge", torch.uint8)
    cams = np.ascontiguousarray(cams, dtype=np.float32).reshape(-1, 16)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    K, h, w = images.shape[0], images.shape[1], images.shape[2]
    if cams.shape[0] != K or weights.shape[0] != K or tuple(depth.shape) != (K, h, w) or tuple(edge.shape) != (K, h, w):
        raise ValueError("cams, weights, images, depth and edge must describe the same K views")
    tex = torch.empty((H, W, 4), dtype=torch.float32, device=low_verts.device)
    inc = torch.empty((K, H, W), dtype=torch.float32, device=low_verts.device) if incidence else None
    o = _opts(ray_tile=ray_tile)
    o.filter = {"aniso": _lib.AG_FILTER_ANISO, "bilinear": _lib.AG_FILTER_BILINEAR}[filter]
    check(lib.ag_backproject(low_verts.data_ptr(), _ptr(low_normals), low_uv.data_ptr(), low_faces.data_ptr(),
                             low_verts.shape[0], low_faces.shape[0], W, H, K, cams.ctypes.data, weights.ctypes.data,
                             images.data_ptr(), depth.data_ptr(), edge.data_ptr(), w, h, float(alpha), float(eps),
                             float(depth_tol), ctypes.byref(o), _stream(stream), tex.data_ptr(), _ptr(inc)))
    return (tex, inc) if incidence else tex


def sync_status(stream=None) -> None:
    """Synchronise and raise AgError if a device-side limit was hit."""
    check(_lib.load().ag_sync_status(_stream(stream)))
