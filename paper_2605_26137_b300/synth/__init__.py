"""Seeded synthetic assets for the normal baker (input generation only).

The paper's workloads (benchmark assets with xatlas UVs, Sec. 6.4 and its
evaluation tables) are not available, so every input is synthetic, with the
shapes of the paper's outputs: a dense marching-grid source mesh of about
1-2M faces (Sec. 6, opening paragraph: 512^3 extraction) and a simplified
mesh of a few thousand to tens of thousands of faces with a UV atlas.

This module holds none of the baking arithmetic.  It only produces vertex
positions, triangle indices and per-corner UVs; both the CUDA path and the
FP64 oracle consume the same arrays.

Generators
----------
* ``icosphere(level)``                 - subdivided icosahedron on the unit sphere.
* ``sh_displaced_sphere(level, seed)``  - icosphere displaced radially by
  r = 1 + 0.05 * sum of 4 seeded real spherical harmonics (degree <= 4).
* ``sdf_union_params(seed, n)`` / ``sdf_grid`` / ``marching_tets`` - a seeded
  polynomial smooth-min union of ellipsoids and rounded boxes, sampled on a
  grid and meshed with marching tetrahedra (watertight, welded).
* ``grid_atlas(F, W, H)``               - the trivial atlas: faces paired into
  quads on a ceil(sqrt(F/2)) grid of cells with a texel gutter.
* ``jittered_atlas(F, W, H, seed)``     - random triangles inside the cells,
  corners off the texel lattice (exercises conservative coverage).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        lib.mt_extract.restype = ctypes.c_int
        lib.mt_extract.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.POINTER(ctypes.POINTER(ctypes.c_float)), ctypes.POINTER(ctypes.c_int64),
            ctypes.POINTER(ctypes.POINTER(ctypes.c_int32)), ctypes.POINTER(ctypes.c_int64)]
        lib.mt_free.restype = None
        lib.mt_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


# --------------------------------------------------------------------------
# icosphere and spherical-harmonic displacement
# --------------------------------------------------------------------------

def icosphere(level: int, radius: float = 1.0):
    """Icosahedron subdivided ``level`` times (4^level * 20 faces), projected
    onto the sphere.  Returns (V float32 [n,3], F int32 [m,3]), outward winding."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    F = list(faces)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    Vn = np.stack(V) * radius
    return Vn.astype(np.float32), np.asarray(F, dtype=np.int32)


def _real_sh(l: int, m: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonic Y_lm(theta = polar, phi = azimuth)."""
    from scipy.special import lpmv
    am = abs(m)
    k = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    p = lpmv(am, l, np.cos(theta))
    if m == 0:
        return k * p
    if m > 0:
        return math.sqrt(2.0) * k * np.cos(am * phi) * p
    return math.sqrt(2.0) * k * np.sin(am * phi) * p


def sh_terms(seed: int, n_terms: int = 4):
    """Seeded (l, m, c): l ~ U{0..4}, m ~ U{-l..l}, c ~ U(-1, 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_terms):
        l = int(rng.integers(0, 5))
        m = int(rng.integers(-l, l + 1))
        c = float(rng.uniform(-1.0, 1.0))
        out.append((l, m, c))
    return out


def sh_displaced_sphere(level: int, seed: int, amp: float = 0.05, n_terms: int = 4):
    """Icosphere with every vertex moved to radius 1 + amp * sum_k c_k Y_{l_k m_k}."""
    V, F = icosphere(level)
    Vd = V.astype(np.float64)
    r = np.linalg.norm(Vd, axis=1)
    theta = np.arccos(np.clip(Vd[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(Vd[:, 1], Vd[:, 0])
    rad = np.ones_like(r)
    for l, m, c in sh_terms(seed, n_terms):
        rad += amp * c * _real_sh(l, m, theta, phi)
    Vd = Vd / r[:, None] * rad[:, None]
    return Vd.astype(np.float32), F


# --------------------------------------------------------------------------
# SDF union of ellipsoids and rounded boxes
# --------------------------------------------------------------------------

@dataclass
class SdfParams:
    centres: np.ndarray      # [n,3]
    sizes: np.ndarray        # [n,3] radii (ellipsoid) / half extents (box)
    rots: np.ndarray         # [n,3,3] local->world rotation
    kinds: np.ndarray        # [n] 0 = ellipsoid, 1 = rounded box
    k: float = 0.03          # smooth-min width
    seed: int = 0
    meta: dict = field(default_factory=dict)


def _quat_to_mat(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def sdf_union_params(seed: int, n_prims: int = 32, k: float = 0.03,
                     centre_range: float = 0.8, size_range=(0.05, 0.4)) -> SdfParams:
    """Seeded primitive set: a 50/50 mix of ellipsoids and rounded boxes,
    centres ~ U(-0.8, 0.8)^3, radii / half extents ~ U(0.05, 0.4), uniformly
    random orientations (Shoemake's uniform quaternion)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-centre_range, centre_range, size=(n_prims, 3))
    sizes = rng.uniform(size_range[0], size_range[1], size=(n_prims, 3))
    kinds = (np.arange(n_prims) % 2).astype(np.int32)
    rng.shuffle(kinds)
    rots = np.empty((n_prims, 3, 3))
    for i in range(n_prims):
        u1, u2, u3 = rng.uniform(size=3)
        q = (math.sqrt(1 - u1) * math.sin(2 * math.pi * u2), math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
             math.sqrt(u1) * math.sin(2 * math.pi * u3), math.sqrt(u1) * math.cos(2 * math.pi * u3))
        rots[i] = _quat_to_mat(q)
    return SdfParams(centres, sizes, rots, kinds, k, seed)


def sdf_eval(points, params: SdfParams):
    """SDF of the smooth union at ``points`` (torch tensor [...,3], any device)."""
    import torch
    dev, dt = points.device, points.dtype
    d = None
    for i in range(len(params.kinds)):
        c = torch.as_tensor(params.centres[i], dtype=dt, device=dev)
        R = torch.as_tensor(params.rots[i], dtype=dt, device=dev)
        s = torch.as_tensor(params.sizes[i], dtype=dt, device=dev)
        q = (points - c) @ R  # world -> local (R is orthonormal, local->world)
        if params.kinds[i] == 0:
            di = (torch.linalg.vector_norm(q / s, dim=-1) - 1.0) * float(params.sizes[i].min())
        else:
            rr = 0.1 * float(params.sizes[i].min())
            qq = q.abs() - (s - rr)
            di = (torch.linalg.vector_norm(qq.clamp_min(0.0), dim=-1)
                  + qq.max(dim=-1).values.clamp_max(0.0) - rr)
        if d is None:
            d = di
        else:
            h = (params.k - (d - di).abs()).clamp_min(0.0) / params.k
            d = torch.minimum(d, di) - h * h * params.k * 0.25
    return d


def sdf_grid(params: SdfParams, n: int, lo: float = -1.25, hi: float = 1.25, device=None):
    """Sample the SDF on an n^3 node grid over [lo, hi]^3.  Returns
    (f float32 numpy [n,n,n] indexed [z,y,x], origin, spacing)."""
    import torch
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    h = (hi - lo) / (n - 1)
    xs = torch.linspace(lo, hi, n, dtype=torch.float32, device=device)
    out = np.empty((n, n, n), dtype=np.float32)
    yy, xx = torch.meshgrid(xs, xs, indexing="ij")
    slab = max(1, (1 << 24) // (n * n))
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        zz = xs[z0:z1].view(-1, 1, 1).expand(z1 - z0, n, n)
        pts = torch.stack([xx.expand(z1 - z0, n, n), yy.expand(z1 - z0, n, n), zz], dim=-1)
        out[z0:z1] = sdf_eval(pts, params).float().cpu().numpy()
    return out, lo, h


def marching_tets(f: np.ndarray, origin: float, h: float):
    """Watertight welded mesh of the f < 0 region of a node grid f[z,y,x]."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float32)
    nz, ny, nx = f.shape
    pv = ctypes.POINTER(ctypes.c_float)()
    pf = ctypes.POINTER(ctypes.c_int32)()
    nv = ctypes.c_int64()
    nf = ctypes.c_int64()
    rc = lib.mt_extract(f.ctypes.data, nx, ny, nz, origin, origin, origin, h,
                        ctypes.byref(pv), ctypes.byref(nv), ctypes.byref(pf), ctypes.byref(nf))
    if rc != 0:
        raise MemoryError("marching tetrahedra: allocation failed")
    try:
        V = np.ctypeslib.as_array(pv, shape=(nv.value, 3)).copy() if nv.value else np.zeros((0, 3), np.float32)
        F = np.ctypeslib.as_array(pf, shape=(nf.value, 3)).copy() if nf.value else np.zeros((0, 3), np.int32)
    finally:
        lib.mt_free(ctypes.cast(pv, ctypes.c_void_p))
        lib.mt_free(ctypes.cast(pf, ctypes.c_void_p))
    return V, F


def sdf_mesh(params: SdfParams, n: int, device=None):
    f, lo, h = sdf_grid(params, n, device=device)
    return marching_tets(f, lo, h)


def sdf_mesh_target(params: SdfParams, target_faces: int, probe_n: int = 64,
                    max_n: int = 1400, device=None):
    """Mesh the SDF at the grid size whose face count is closest to the target
    (face count grows as n^2: probe once, scale, then refine once)."""
    _, fp = sdf_mesh(params, probe_n, device=device)
    n = int(round(probe_n * math.sqrt(target_faces / max(1, len(fp)))))
    n = max(8, min(max_n, n))
    V, F = sdf_mesh(params, n, device=device)
    if abs(len(F) - target_faces) > 0.1 * target_faces:
        n2 = int(round(n * math.sqrt(target_faces / max(1, len(F)))))
        n2 = max(8, min(max_n, n2))
        if n2 != n:
            V, F = sdf_mesh(params, n2, device=device)
            n = n2
    params.meta[f"grid_for_{target_faces}"] = n
    return V, F


def hidden_face_mesh(seed: int, target_faces: int = 22_000, n_inner: int = 8, inner_level: int = 2,
                     n_prims: int = 16, device=None):
    """Stand-in for a generated mesh with interior faces (the input of
    hidden-face removal): the closed marching-grid surface of a seeded SDF
    union, plus n_inner closed icospheres (20 * 4^inner_level faces each)
    placed wholly inside the solid: a shell of radius r needs a field value
    below -(2 r + 2 h + k) at its centre (h the grid spacing, k the smooth-min
    width), room for the extracted surface's departures from the field's zero
    set on coarse grids.  Returns (V, F, inner) with inner [F] bool marking
    the interior shells' faces."""
    import torch
    params = sdf_union_params(seed, n_prims=n_prims)
    ico_v, ico_f = icosphere(inner_level)
    outer_target = max(1000, target_faces - n_inner * len(ico_f))
    Vo, Fo = sdf_mesh_target(params, outer_target, device=device)
    h = 2.5 / (params.meta[f"grid_for_{outer_target}"] - 1)
    rng = np.random.default_rng(seed + 7919)
    pts = rng.uniform(-1.0, 1.0, size=(20000, 3))
    d = sdf_eval(torch.as_tensor(pts, dtype=torch.float64), params).numpy()
    Vs, Fs, inner = [Vo], [Fo], [np.zeros(len(Fo), bool)]
    nv = len(Vo)
    placed = []
    for i in np.argsort(d):
        if len(placed) == n_inner or d[i] >= 0:
            break
        r = min(0.5 * (-d[i] - 2.0 * h - params.k), 0.12)
        c = pts[i]
        if r < 0.01 or any(np.linalg.norm(c - q) < r + rq + 0.01 for q, rq in placed):
            continue
        placed.append((c, r))
        Vs.append((ico_v.astype(np.float64) * r + c).astype(np.float32))
        Fs.append(ico_f + nv)
        inner.append(np.ones(len(ico_f), bool))
        nv += len(ico_v)
    return np.concatenate(Vs), np.concatenate(Fs).astype(np.int32), np.concatenate(inner)


# --------------------------------------------------------------------------
# UV atlases (per-corner UVs, [F,3,2] float32)
# --------------------------------------------------------------------------

def grid_cells(n_faces: int, W: int, H: int):
    g = int(math.ceil(math.sqrt(n_faces / 2.0)))
    return g, W // g, H // g


def grid_atlas(n_faces: int, W: int, H: int, gutter: int = 2):
    """Faces 2k and 2k+1 form a quad in cell k (row-major on a g x g grid).
    Quad corners sit on texel boundaries, ``gutter`` texels inside the cell:
    face 2k gets (x0,y0) (x1,y0) (x1,y1), face 2k+1 gets (x0,y0) (x1,y1) (x0,y1)."""
    g, sx, sy = grid_cells(n_faces, W, H)
    if sx - 2 * gutter < 1 or sy - 2 * gutter < 1:
        raise ValueError("atlas too small for this face count and gutter")
    uv = np.zeros((n_faces, 3, 2), dtype=np.float64)
    k = np.arange(n_faces) // 2
    cx, cy = k % g, k // g
    x0 = cx * sx + gutter
    x1 = cx * sx + sx - gutter
    y0 = cy * sy + gutter
    y1 = cy * sy + sy - gutter
    even = (np.arange(n_faces) % 2) == 0
    uv[even, 0] = np.stack([x0, y0], -1)[even]
    uv[even, 1] = np.stack([x1, y0], -1)[even]
    uv[even, 2] = np.stack([x1, y1], -1)[even]
    odd = ~even
    uv[odd, 0] = np.stack([x0, y0], -1)[odd]
    uv[odd, 1] = np.stack([x1, y1], -1)[odd]
    uv[odd, 2] = np.stack([x0, y1], -1)[odd]
    uv[..., 0] /= W
    uv[..., 1] /= H
    return uv.astype(np.float32)


def jittered_atlas(n_faces: int, W: int, H: int, seed: int, gutter: int = 2):
    """Like ``grid_atlas`` but each face is a random triangle inside its half
    of the cell with corners off the texel lattice; some faces get tiny or
    zero UV area so the degenerate-UV path is exercised."""
    rng = np.random.default_rng(seed)
    g, sx, sy = grid_cells(n_faces, W, H)
    uv = np.zeros((n_faces, 3, 2), dtype=np.float64)
    for f in range(n_faces):
        k = f // 2
        cx, cy = k % g, k // g
        x0, y0 = cx * sx + gutter * 0.5, cy * sy + gutter * 0.5
        w, h = sx - gutter, sy - gutter
        pts = np.stack([x0 + rng.uniform(0, w, 3), y0 + rng.uniform(0, h, 3)], -1)
        r = rng.uniform()
        if r < 0.03:
            pts[2] = pts[1]                      # zero UV area
        elif r < 0.06:
            pts[2] = pts[1] + rng.uniform(-1, 1, 2) * 1e-3  # tiny UV area
        uv[f] = pts
    uv[..., 0] /= W
    uv[..., 1] /= H
    return uv.astype(np.float32)


# --------------------------------------------------------------------------
# assembled assets
# --------------------------------------------------------------------------

def surface_samples(V, F, n: int, seed: int):
    """n seeded points spread uniformly by area over a triangle mesh, as
    (face id int32 [n], barycentrics (b1, b2) of corners 1 and 2 float32 [n, 2]):
    a face drawn with probability proportional to its area, then a uniform
    point of it (the square's two halves folded onto one triangle)."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    area = np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)
    rng = np.random.default_rng(seed)
    face = rng.choice(len(F), size=n, p=area / area.sum()).astype(np.int32)
    u, v = rng.random(n), rng.random(n)
    flip = u + v > 1.0
    u, v = np.where(flip, 1.0 - u, u), np.where(flip, 1.0 - v, v)
    return face, np.stack([u, v], -1).astype(np.float32)


@dataclass
class Asset:
    high_v: np.ndarray
    high_f: np.ndarray
    low_v: np.ndarray
    low_f: np.ndarray
    low_uv: np.ndarray
    W: int
    H: int
    max_dist: float
    gutter: int = 2
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def diam(self) -> float:
        lo = self.high_v.astype(np.float64).min(0)
        hi = self.high_v.astype(np.float64).max(0)
        return float(np.linalg.norm(hi - lo))


def tiny_asset(seed: int = 0, W: int = 128, H: int = 128) -> Asset:
    """320-face unit icosphere (trivial atlas, 128^2) over a 5,120-face icosphere
    displaced by 4 seeded spherical harmonics; max_dist 0.15."""
    lv, lf = icosphere(2)
    hv, hf = sh_displaced_sphere(4, seed)
    uv = grid_atlas(len(lf), W, H, 2)
    return Asset(hv, hf, lv, lf, uv, W, H, 0.15, 2, f"icosphere-320-over-sh5120-s{seed}",
                 {"seed": seed, "sh": sh_terms(seed)})


def sdf_asset(seed: int, high_faces: int, low_faces: int, W: int, H: int,
              n_prims: int = 32, max_dist_frac: float = 0.02, device=None,
              high_grid: int | None = None, low_grid: int | None = None) -> Asset:
    """Smooth-min union of ``n_prims`` primitives meshed twice: densely (high)
    and coarsely (low, trivial atlas).  max_dist = 2% of the high bbox diagonal."""
    p = sdf_union_params(seed, n_prims)
    if high_grid is None:
        hv, hf = sdf_mesh_target(p, high_faces, device=device)
    else:
        hv, hf = sdf_mesh(p, high_grid, device=device)
    if low_grid is None:
        lv, lf = sdf_mesh_target(p, low_faces, probe_n=32, device=device)
    else:
        lv, lf = sdf_mesh(p, low_grid, device=device)
    uv = grid_atlas(len(lf), W, H, 2)
    a = Asset(hv, hf, lv, lf, uv, W, H, 0.0, 2,
              f"sdf{n_prims}-s{seed}-high{len(hf)}-low{len(lf)}-{W}x{H}", {"seed": seed, "grids": dict(p.meta)})
    a.max_dist = max_dist_frac * a.diam
    return a


# --------------------------------------------------------------------------
# Cameras and generated-view stand-ins (UV-space backprojection)
# --------------------------------------------------------------------------

# the paper's view set (Sec. 7.4): azimuth / elevation in degrees and prior weight
PAPER_VIEWS = (("front", 0, 0, 1.0), ("rear", 180, 0, 1.0), ("top", 0, 90, 0.3), ("bottom", 0, -90, 0.3),
               ("front_left45", -45, 0, 0.1), ("front_right45", 45, 0, 0.1), ("left", -90, 0, 0.01),
               ("right", 90, 0, 0.01), ("rear_left45", -135, 0, 0.001), ("rear_right45", 135, 0, 0.001))


def look_at_camera(eye, target, up, fov_deg: float, w: int, h: int):
    """Pinhole camera [16] f32: R (rows right, down, forward) row-major, t,
    fx, fy, cx, cy, looking from ``eye`` at ``target``."""
    eye, target, up = (np.asarray(x, np.float64) for x in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, [1.0, 0.0, 0.0])
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    fy = 0.5 * h / math.tan(math.radians(fov_deg) / 2)
    return np.concatenate([R.ravel(), t, [fy, fy, 0.5 * w, 0.5 * h]]).astype(np.float32)


def paper_cameras(center, radius: float, w: int, h: int, fov_deg: float = 40.0):
    """The ten views of PAPER_VIEWS around a bounding sphere (centre, radius),
    framed so that the sphere fits the image; front looks along -z, up is +y.
    Returns (cams [10,16] f32, weights [10] f32, names)."""
    dist = radius / math.sin(math.radians(fov_deg) / 2) * 1.05
    cams, weights, names = [], [], []
    for name, az, el, wgt in PAPER_VIEWS:
        a, e = math.radians(az), math.radians(el)
        direction = np.array([math.sin(a) * math.cos(e), math.sin(e), math.cos(a) * math.cos(e)])
        up = [0.0, 1.0, 0.0] if abs(el) < 80 else [0.0, 0.0, -1.0 if el > 0 else 1.0]
        cams.append(look_at_camera(np.asarray(center) + dist * direction, center, up, fov_deg, w, h))
        weights.append(wgt)
        names.append(name)
    return np.stack(cams), np.asarray(weights, np.float32), names


def color_field(points):
    """Smooth seeded colour of world points [...,3] (numpy or torch), values in
    [0.05, 0.95] per channel: the stand-in for a generated texture."""
    mod = np
    try:
        import torch
        if isinstance(points, torch.Tensor):
            mod = torch
    except ImportError:
        pass
    x, y, z = points[..., 0], points[..., 1], points[..., 2]
    r = 0.5 + 0.45 * mod.sin(2.1 * x + 0.7 * y + 0.3)
    g = 0.5 + 0.45 * mod.sin(1.3 * y - 1.7 * z + 1.1)
    b = 0.5 + 0.45 * mod.cos(1.9 * z + 0.9 * x - 0.4)
    return mod.stack([r, g, b], -1)


def view_images(points, colors=color_field):
    """RGBA8 images [K,h,w,4] of world point maps [K,h,w,3] (NaN = background,
    coloured black, alpha 0)."""
    pts = np.asarray(points, np.float64)
    hit = np.isfinite(pts[..., 0])
    c = np.zeros(pts.shape[:-1] + (3,), np.float64)
    c[hit] = colors(pts[hit])
    img = np.zeros(pts.shape[:-1] + (4,), np.uint8)
    img[..., :3] = np.clip(np.round(c * 255), 0, 255).astype(np.uint8)
    img[..., 3] = np.where(hit, 255, 0)
    return img
