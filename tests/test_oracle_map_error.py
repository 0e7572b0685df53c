"""Pins for the oracle's "baked mean" measure (Sec. 6.1, the simplification
benchmark's baked-normal error): the angle at sample points of the low mesh
between the normal a baked RGBA8 map gives (decoded, taken to world space
through the bake's tangent frame) and the raw mesh's smooth normal at its
nearest point.

* identity: raw == low bakes to the neutral map and the angle is 0;
* a neutral map over a flat quad under a tilted plane gives the tilt angle;
* the baked map of that pair is exact up to the 8-bit rounding;
* a map of known per-texel values on an affine quad: decode, the texel read
  at the sample's UV point (x from u, y from v), the tangent along +dp/du and
  the bitangent along +dp/dv (mirrored UVs flip it), against a tilted raw
  plane, angle by angle;
* the BVH search equals brute force.
"""
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def _plane(n, x0, x1, y0, y1, h=0.0, s=0.0):
    xs, ys = np.linspace(x0, x1, n + 1), np.linspace(y0, y1, n + 1)
    X, Y = np.meshgrid(xs, ys)
    V = np.stack([X.ravel(), Y.ravel(), h - s * Y.ravel()], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.asarray(F, np.int32)


QUAD_V = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
QUAD_F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)


def _quad_uv(mirror=False):
    sgn = -1.0 if mirror else 1.0
    return np.array([[(0.1 + 0.4 * (QUAD_V[i, 0] + 1), 0.5 + sgn * 0.4 * QUAD_V[i, 1]) for i in f] for f in QUAD_F],
                    np.float32)


def test_identity_is_zero():
    V, F = synth.sh_displaced_sphere(2, 3)
    uv = synth.grid_atlas(len(F), 256, 256, 2)
    r = oracle.bake(V, F, V, F, uv, 256, 256, 0.05)
    sf, sb = synth.surface_samples(V, F, 3000, 1)
    ang, fl = oracle.normal_map_error(V, F, V, F, uv, 256, 256, r["rgba8"], sf, sb, 0.05)
    assert (ang >= 0).all() and ang.max() < 1e-5


@pytest.mark.parametrize("s", [0.1, 0.35])
def test_neutral_map_gives_the_tilt_and_baked_map_removes_it(s):
    hv, hf = _plane(16, -1.5, 1.5, -1.5, 1.5, 0.05, s)
    W = H = 64
    uv = _quad_uv()
    sf, sb = synth.surface_samples(QUAD_V, QUAD_F, 2000, 2)
    neutral = np.zeros((H, W, 4), np.uint8)
    neutral[...] = (128, 128, 255, 0)
    ang, _ = oracle.normal_map_error(hv, hf, QUAD_V, QUAD_F, uv, W, H, neutral, sf, sb, 1.0)
    assert np.abs(ang - np.degrees(np.arctan(s))).max() < 1e-4
    r = oracle.bake(hv, hf, QUAD_V, QUAD_F, uv, W, H, 1.0)
    ang, _ = oracle.normal_map_error(hv, hf, QUAD_V, QUAD_F, uv, W, H, r["rgba8"], sf, sb, 1.0)
    # each decoded component is within half a code (0.5/127) of the exact one
    assert ang.max() < np.degrees(np.sqrt(3) * 0.5 / 127) and ang.mean() < 0.2


@pytest.mark.parametrize("mirror", [False, True])
def test_known_map_values_angle_by_angle(mirror):
    """Tangent-space value per texel: c = (sin a cos b, sin a sin b, cos a)
    with a growing with x and b chosen by y, so a misread texel (x and y
    swapped, v flipped) or a wrong frame axis changes the angle.  The quad's
    UVs are affine in position: T = +x, B = +y (or -y mirrored), N = +z.  The
    raw plane is tilted about x, normal (0, s, 1)/sqrt(1 + s^2)."""
    W, H, s = 64, 48, 0.2
    hv, hf = _plane(8, -1.5, 1.5, -1.5, 1.5, 0.05, s)
    uv = _quad_uv(mirror)
    xs = np.arange(W)
    ys = np.arange(H)
    a = np.radians(5.0 + 50.0 * xs / W)[None, :] * np.ones((H, 1))
    b = np.where((ys % 2 == 0)[:, None], 0.0, np.pi / 2) * np.ones((1, W))
    c = np.stack([np.sin(a) * np.cos(b), np.sin(a) * np.sin(b), np.cos(a)], -1)
    rgba = np.zeros((H, W, 4), np.uint8)
    rgba[..., :3] = 128 + np.round(127 * c)
    rgba[..., 3] = 255
    # samples at texel centres, one per texel of the quad's interior
    pts = []
    for y in range(H):
        for x in range(W):
            u, v = (x + 0.5) / W, (y + 0.5) / H
            px = (u - 0.1) / 0.4 - 1
            py = ((v - 0.5) / 0.4) * (-1 if mirror else 1)
            if -0.98 < px < 0.98 and -0.98 < py < 0.98:
                pts.append((x, y, px, py))
    pts = np.array(pts)
    # barycentrics in face 0 (v0, v1, v2) or face 1 (v0, v2, v3) of the quad
    sf, sb = [], []
    for _, _, px, py in pts:
        P = np.array([px, py])
        for f in (0, 1):
            A, B, C = (QUAD_V[QUAD_F[f, k], :2].astype(np.float64) for k in range(3))
            M = np.stack([B - A, C - A], 1)
            b12 = np.linalg.solve(M, P - A)
            if b12.min() >= -1e-12 and b12.sum() <= 1 + 1e-12:
                sf.append(f)
                sb.append(b12)
                break
    sf, sb = np.array(sf, np.int32), np.array(sb)
    ang, _ = oracle.normal_map_error(hv, hf, QUAD_V, QUAD_F, uv, W, H, rgba, sf, sb, 1.0)
    q = rgba[pts[:, 1].astype(int), pts[:, 0].astype(int), :3].astype(np.float64)
    cd = (q - 128) / 127
    cd /= np.linalg.norm(cd, axis=1, keepdims=True)
    world = np.stack([cd[:, 0], (-1 if mirror else 1) * cd[:, 1], cd[:, 2]], -1)
    raw = np.array([0.0, s, 1.0]) / np.sqrt(1 + s * s)
    exp = np.degrees(np.arctan2(np.linalg.norm(np.cross(world, raw), axis=1), world @ raw))
    assert len(ang) > 1500
    assert np.abs(ang - exp).max() < 1e-4


def test_bvh_equals_brute_force():
    a = synth.sdf_asset(3, 20_000, 800, 128, 128, n_prims=8)
    r = oracle.bake_asset(a)
    sf, sb = synth.surface_samples(a.low_v, a.low_f, 1500, 4)
    g1, f1 = oracle.normal_map_error(a.high_v, a.high_f, a.low_v, a.low_f, a.low_uv, a.W, a.H, r["rgba8"], sf, sb,
                                     a.max_dist)
    g2, f2 = oracle.normal_map_error(a.high_v, a.high_f, a.low_v, a.low_f, a.low_uv, a.W, a.H, r["rgba8"], sf, sb,
                                     a.max_dist, use_bvh=False)
    assert np.array_equal(g1, g2) and np.array_equal(f1, f2)
    assert (g1 >= 0).mean() > 0.9


def test_degenerate_uv_face_uses_the_low_normal():
    """A face whose UVs are degenerate (the UV-reliability filter) does not
    read the map: its samples give the angle between the low normal and the
    raw normal (the tilt), while the other face's samples read the
    non-neutral map value."""
    s = 0.25
    hv, hf = _plane(8, -1.5, 1.5, -1.5, 1.5, 0.05, s)
    W = H = 64
    uv = _quad_uv()
    uv[1] = uv[1][0]                                   # face 1: all three corners at one UV point
    rgba = np.zeros((H, W, 4), np.uint8)
    rgba[...] = (128, 128 + 40, 128 + 119, 255)        # tilted away from +z in tangent space
    sf, sb = synth.surface_samples(QUAD_V, QUAD_F, 2000, 3)
    ang, _ = oracle.normal_map_error(hv, hf, QUAD_V, QUAD_F, uv, W, H, rgba, sf, sb, 1.0)
    tilt = np.degrees(np.arctan(s))
    assert np.abs(ang[sf == 1] - tilt).max() < 1e-4
    c = np.array([0.0, 40.0, 119.0]) / 127
    c /= np.linalg.norm(c)
    raw = np.array([0.0, s, 1.0]) / np.sqrt(1 + s * s)
    exp = np.degrees(np.arccos(c @ raw))
    assert np.abs(ang[sf == 0] - exp).max() < 1e-4
