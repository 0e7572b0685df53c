"""Pins for the oracle's UV-space raster (Sec. 6.4, first stage).

* closed form on the trivial grid atlas (counts, owners, barycentrics);
* an independent exact-rational implementation of the ownership rule
  (Sutherland-Hodgman clipping for the positive-area overlap, exact point-to-
  segment distances) on tiny random atlases;
* brute force over all (texel, face) pairs equals the bounding-box version;
* snapping of UVs to 1/256 texel with ties away from zero.
"""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def test_snap_rounding():
    # u*W*256 exactly representable; halves round away from zero
    W = 128
    assert oracle.snap(0.0, W) == 0
    assert oracle.snap(1.0, W) == 128 * 256
    half = 0.5 / (W * 256)  # exactly half a snapped unit
    assert oracle.snap(np.float32(half), W) == 1
    assert oracle.snap(np.float32(-half), W) == -1
    assert oracle.snap(np.float32(3 * half), W) == 2
    assert oracle.snap(np.float32(2.5 / (W * 256) - 1e-12), W) in (2, 3)
    # non power-of-two width: u*W*256 computed exactly
    u = np.float32(0.1)
    assert oracle.snap(u, 1000) == math.floor(float(Fr(float(u)) * 1000 * 256) + Fr(1, 2))


@pytest.mark.parametrize("F,W,gutter", [(320, 128, 2), (100, 64, 2), (31, 64, 1)])
def test_grid_atlas_closed_form(F, W, gutter):
    """Quad k has corners on texel boundaries, L = cell - 2*gutter texels a side.
    Texel (x0+i, y0+j) belongs to face 2k iff j <= i (diagonal to the lower id),
    else to 2k+1; its barycentrics are those of the centre; nothing else is
    covered (conservative overlap needs positive area)."""
    H = W
    uv = synth.grid_atlas(F, W, H, gutter)
    face, bary, a2 = oracle.raster(uv, W, H)
    g, sx, sy = synth.grid_cells(F, W, H)
    L = sx - 2 * gutter
    expect = np.full((H, W), -1, np.int32)
    eb = np.zeros((H, W, 3))
    for f in range(F):
        k = f // 2
        x0, y0 = (k % g) * sx + gutter, (k // g) * sy + gutter
        for j in range(L):
            for i in range(L):
                a, b = i + 0.5, j + 0.5
                if f % 2 == 0 and j <= i:
                    expect[y0 + j, x0 + i] = f
                    eb[y0 + j, x0 + i] = (1 - a / L, (a - b) / L, b / L)
                elif f % 2 == 1 and j > i and (f - 1) // 2 == k:
                    expect[y0 + j, x0 + i] = f
                    # face 2k+1: corners (x0,y0) (x1,y1) (x0,y1)
                    eb[y0 + j, x0 + i] = (1 - b / L, a / L, (b - a) / L)
                elif f % 2 == 0 and j > i and f == F - 1:
                    pass  # last unpaired face: upper half stays empty
    assert np.array_equal(face, expect)
    m = face >= 0
    assert np.abs(bary[m] - eb[m]).max() < 1e-15
    n_pairs = F // 2
    n_ray = n_pairs * L * L + (F % 2) * (L * (L + 1) // 2)
    assert int(m.sum()) == n_ray
    assert np.all(np.abs(a2) == (L * 256) ** 2)


# ----------------------------------------------------------- exact reference

def _snap(u, W):
    x = Fr(float(np.float32(u))) * W * 256
    return math.floor(x + Fr(1, 2)) if x >= 0 else -math.floor(-x + Fr(1, 2))


def _clip_area(tri, sx, sy):
    """Area of triangle (exact points) clipped to the square [sx,sx+256]x[sy,sy+256]."""
    poly = list(tri)
    if (poly[1][0] - poly[0][0]) * (poly[2][1] - poly[0][1]) - (poly[1][1] - poly[0][1]) * (poly[2][0] - poly[0][0]) < 0:
        poly = poly[::-1]
    for axis, val, keep_ge in ((0, sx, True), (0, sx + 256, False), (1, sy, True), (1, sy + 256, False)):
        out = []
        n = len(poly)
        for i in range(n):
            p, q = poly[i], poly[(i + 1) % n]
            pin = p[axis] >= val if keep_ge else p[axis] <= val
            qin = q[axis] >= val if keep_ge else q[axis] <= val
            if pin:
                out.append(p)
            if pin != qin:
                t = Fr(val - p[axis]) / (q[axis] - p[axis])
                out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
        poly = out
        if not poly:
            return Fr(0)
    area = Fr(0)
    for i in range(len(poly)):
        p, q = poly[i], poly[(i + 1) % len(poly)]
        area += p[0] * q[1] - q[0] * p[1]
    return area / 2


def _seg_d2(c, a, b):
    dx, dy = b[0] - a[0], b[1] - a[1]
    wx, wy = c[0] - a[0], c[1] - a[1]
    dd = dx * dx + dy * dy
    t = Fr(0) if dd == 0 else max(Fr(0), min(Fr(1), Fr(wx * dx + wy * dy, dd)))
    px, py = a[0] + t * dx - c[0], a[1] + t * dy - c[1]
    return px * px + py * py, t


def exact_raster(uv, W, H):
    F = uv.shape[0]
    tris = [[(_snap(uv[f, k, 0], W), _snap(uv[f, k, 1], H)) for k in range(3)] for f in range(F)]
    face = np.full((H, W), -1, np.int32)
    bary = np.zeros((H, W, 3))
    n_cons = 0
    for y in range(H):
        for x in range(W):
            c = (256 * x + 128, 256 * y + 128)
            owner = None
            for f, t in enumerate(tris):
                a2 = (t[1][0] - t[0][0]) * (t[2][1] - t[0][1]) - (t[1][1] - t[0][1]) * (t[2][0] - t[0][0])
                if a2 == 0:
                    continue
                e = [(t[(k + 2) % 3][0] - t[(k + 1) % 3][0]) * (c[1] - t[(k + 1) % 3][1])
                     - (t[(k + 2) % 3][1] - t[(k + 1) % 3][1]) * (c[0] - t[(k + 1) % 3][0]) for k in range(3)]
                if all(v * a2 >= 0 for v in e):
                    owner = f
                    bary[y, x] = [Fr(v, a2) for v in e]
                    break
            if owner is None:
                best = None
                for f, t in enumerate(tris):
                    a2 = (t[1][0] - t[0][0]) * (t[2][1] - t[0][1]) - (t[1][1] - t[0][1]) * (t[2][0] - t[0][0])
                    if a2 == 0 or _clip_area(t, 256 * x, 256 * y) <= 0:
                        continue
                    qbest, eb = None, None
                    for k in range(3):
                        d2, tt = _seg_d2(c, t[k], t[(k + 1) % 3])
                        q = math.floor(d2 * 65536)
                        if qbest is None or q < qbest:
                            qbest, eb = q, (k, tt)
                    if best is None or qbest < best[0]:
                        best = (qbest, f, eb)
                if best is not None:
                    n_cons += 1
                    owner = best[1]
                    k, tt = best[2]
                    b = [0.0, 0.0, 0.0]
                    b[k] = float(1 - tt)
                    b[(k + 1) % 3] = float(tt)
                    bary[y, x] = b
            if owner is not None:
                face[y, x] = owner
    return face, bary, n_cons


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_raster_matches_exact_rational_definition(seed):
    W = H = 12
    uv = synth.jittered_atlas(6, W, H, seed, gutter=1)
    rng = np.random.default_rng(seed)
    # pull corners further off-lattice and let some triangles overlap their neighbours
    uv = (uv + rng.normal(0, 0.02, uv.shape)).astype(np.float32)
    face, bary, _ = oracle.raster(uv, W, H)
    ef, eb, n_cons = exact_raster(uv, W, H)
    assert np.array_equal(face, ef)
    m = face >= 0
    assert np.abs(bary[m] - eb[m]).max() < 1e-12
    # the conservative rule really was exercised
    assert n_cons > 0


@pytest.mark.parametrize("seed", [0, 5])
def test_raster_bbox_equals_brute_force(seed):
    W, H = 64, 48
    uv = synth.jittered_atlas(60, W, H, seed)
    f1, b1, _ = oracle.raster(uv, W, H, brute=False)
    f2, b2, _ = oracle.raster(uv, W, H, brute=True)
    assert np.array_equal(f1, f2)
    assert np.array_equal(b1, b2)


def test_degenerate_uv_flag():
    """|UV area| < 1e-4 texel^2 <=> |2*area| <= 13 in 1/256-texel units."""
    W = H = 32
    uv = synth.grid_atlas(8, W, H, 2).astype(np.float64)
    unit = 1.0 / (W * 256)
    uv[3, 2] = uv[3, 1]                              # zero area
    for f, h in ((5, 13), (6, 14)):
        uv[f, 1] = uv[f, 0] + (unit, 0.0)
        uv[f, 2] = uv[f, 0] + (0.0, h * unit)
    uv = uv.astype(np.float32)
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    F = np.array([[0, 1, 2]] * 8, np.int32)
    N = oracle.vertex_normals(V, F)
    _, _, dg = oracle.face_frames(V, F, uv, W, H, N)
    face, _, a2 = oracle.raster(uv, W, H)
    assert a2[3] == 0 and abs(a2[5]) == 13 and abs(a2[6]) == 14
    assert dg[3] == 1 and dg[5] == 1 and dg[6] == 0
    assert dg.sum() == 2
    assert not (face == 3).any()
