"""Pins for the oracle's UV-space backprojection and incidence blending
(Sec. 7.4).

* a plane seen face-on through an image whose codes are affine in the pixel
  index: bilinear sampling reproduces the affine map, so the texture equals
  the closed form of the projection;
* occlusion: a plane behind another receives nothing where it is covered;
* blending: two constant-colour views of a tilted plane mix with weights
  w_k cos^alpha(theta_k) (closed form); a large alpha, where the powers
  underflow, still picks the better view (the log-space reduction);
* back-facing surfaces, points behind a camera and edge pixels (depth
  discontinuities) contribute nothing;
* the rendered depth of a plane is its distance along the view axis;
* anisotropic filtering: the Lanczos-2 pyramid against numpy's sinc (a ramp,
  a constant, one bright pixel), the taps of an oblique footprint against the
  exact derivative of the projection and numpy's SVD, and the trilinear level
  of a far face-on footprint against numpy bilinear samples of the pyramid.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def _plane(n, z=0.0, size=1.0, flip=False):
    xs = np.linspace(-size, size, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    F = np.asarray(F, np.int32)
    if flip:
        F = F[:, ::-1].copy()
    return V, F


def _front_camera(D, w, h, f=60.0):
    # at (0, 0, D) looking down -z: right = +x, down = -y, forward = -z
    R = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float64)
    t = -R @ np.array([0.0, 0.0, D])
    return np.concatenate([R.ravel(), t, [f, f, w / 2, h / 2]]).astype(np.float32)


def _texel_points(o, V, F):
    m = o["face"] >= 0
    p = (o["bary"][m][:, :, None] * V.astype(np.float64)[F[o["face"][m]]]).sum(1)
    return m, p


def test_render_depth_is_view_distance():
    V, F = _plane(4, z=0.25)
    cam = _front_camera(3.0, 32, 32)
    depth, point, near = oracle.render_views(V, F, cam[None], 32, 32)
    hit = np.isfinite(depth[0])
    assert hit.sum() > 100
    assert np.abs(depth[0][hit] - 2.75).max() < 1e-12
    assert np.abs(point[0][hit][:, 2] - 0.25).max() < 1e-12
    # a larger plane just behind the camera (nearer along the line than the
    # one in front) plays no part: the first hit is the smallest t > 0
    Vb, Fb = _plane(8, z=3.5, size=4.0)
    V2 = np.concatenate([V, Vb])
    F2 = np.concatenate([F, Fb + len(V)]).astype(np.int32)
    depth2, _, near2 = oracle.render_views(V2, F2, cam[None], 32, 32)
    assert np.array_equal(np.isfinite(depth2[0]), hit)
    assert np.abs(depth2[0][hit] - 2.75).max() < 1e-12
    assert not near2[0][hit].any()


def test_face_on_affine_image_closed_form():
    V, F = _plane(4)
    w = h = 64
    D, fx = 3.0, 60.0
    cam = _front_camera(D, w, h, fx)
    ii, jj = np.meshgrid(np.arange(w), np.arange(h))
    img = np.zeros((1, h, w, 4), np.uint8)
    img[0, ..., 0] = 2 * ii + 40
    img[0, ..., 1] = 3 * jj + 20
    img[0, ..., 2] = 128
    img[0, ..., 3] = 255
    W = H = 64
    uv = synth.grid_atlas(len(F), W, H, 2)
    o = oracle.backproject(V, F, uv, W, H, cam[None], img, np.ones(1, np.float32), alpha=1.0, eps=0.0,
                           depth_tol=1e-3, edge_tol=1.0)
    m, p = _texel_points(o, V, F)
    u = fx * p[:, 0] / D + w / 2
    v = -fx * p[:, 1] / D + h / 2
    # away from the plane's projected rim (edge pixels, two pixels wide with the bilinear footprint)
    margin = 1.0 - 2.5 * D / fx
    interior = (np.abs(p[:, 0]) < margin) & (np.abs(p[:, 1]) < margin) & (o["flags"][m] == 0)
    assert interior.sum() > 1000
    tex = o["texture"][m]
    assert o["filled"][m][interior].all()
    assert np.abs(tex[interior, 0] - (2 * (u[interior] - 0.5) + 40) / 255).max() < 1e-9
    assert np.abs(tex[interior, 1] - (3 * (v[interior] - 0.5) + 20) / 255).max() < 1e-9
    assert np.abs(tex[interior, 2] - 128 / 255).max() < 1e-12
    # incidence: cos of the angle between the plane normal (+z) and the direction to the camera
    I = o["incidence"][0][m]
    cos = D / np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2 + D ** 2)
    assert np.abs(I[interior] - cos[interior]).max() < 1e-12


def test_occluded_plane_receives_nothing():
    Vb, Fb = _plane(4, z=0.0)
    Vf, Ff = _plane(2, z=0.5, size=0.4)
    V = np.concatenate([Vb, Vf])
    F = np.concatenate([Fb, Ff + len(Vb)]).astype(np.int32)
    w = h = 64
    cam = _front_camera(3.0, w, h)
    img = np.full((1, h, w, 4), 200, np.uint8)
    W = H = 96
    uv = synth.grid_atlas(len(F), W, H, 2)
    # the pixel footprint is 0.05 world units here: edge_tol must exceed it (the planes are 0.5 apart)
    o = oracle.backproject(V, F, uv, W, H, cam[None], img, np.ones(1, np.float32), alpha=1.0, eps=1e-6,
                           depth_tol=1e-3, edge_tol=0.2)
    m, p = _texel_points(o, V, F)
    back = o["face"][m] < len(Fb)
    # behind the front plane's footprint, seen from the camera (with a margin of a few pixels)
    proj = p[:, :2] * 3.0 / (3.0 - p[:, 2:3])
    covered = back & (np.abs(proj).max(1) < 0.4 * 3.0 / 2.5 - 0.05)
    clear = (back & (np.abs(proj).max(1) > 0.4 * 3.0 / 2.5 + 0.15) & (np.abs(p[:, :2]).max(1) < 1 - 2.5 * 3.0 / 60)
             & (o["flags"][m] == 0))
    assert covered.sum() > 50 and clear.sum() > 200
    assert not o["filled"][m][covered].any()
    assert o["filled"][m][clear].all()


@pytest.mark.parametrize("alpha", [1.0, 4.0, 400.0])
def test_two_view_blend_closed_form(alpha):
    # the plane z = 0 seen from cameras at angles a1, a2 in the xz-plane; it
    # extends past both images (no silhouette, no edge pixels in view)
    V, F = _plane(8, size=1.5)
    w = h = 48
    cams, I_exp = [], []
    for ang in (10.0, 50.0):
        a = math.radians(ang)
        eye = np.array([4 * math.sin(a), 0.0, 4 * math.cos(a)])
        cams.append(synth.look_at_camera(eye, [0, 0, 0], [0, 1, 0], 30.0, w, h))
    img = np.zeros((2, h, w, 4), np.uint8)
    img[0, ..., 0] = 255
    img[1, ..., 2] = 255
    img[..., 3] = 255
    wts = np.array([0.3, 1.0], np.float32)
    W = H = 128
    uv = synth.grid_atlas(len(F), W, H, 2)
    # eps is absolute in the linear domain: at alpha = 400 the weights w I^alpha
    # are ~1e-60 and any eps > 0 would dominate, so that case takes eps = 0
    eps = 1e-6 if alpha < 100 else 0.0
    # depth_tol above the change of depth across one pixel of the oblique view
    # (the depth test reads the nearest pixel)
    o = oracle.backproject(V, F, uv, W, H, np.stack(cams), img, wts, alpha=alpha, eps=eps, depth_tol=0.1,
                           edge_tol=10.0)
    m, p = _texel_points(o, V, F)
    ok = (o["flags"][m] == 0) & (np.abs(p[:, :2]).max(1) < 0.5)      # inside both frusta
    assert ok.sum() > 100
    C = [np.array([4 * math.sin(math.radians(a)), 0.0, 4 * math.cos(math.radians(a))]) for a in (10.0, 50.0)]
    cos = np.stack([(c[None] - p)[:, 2] / np.linalg.norm(c[None] - p, axis=1) for c in C])   # normal +z
    L = np.log(wts.astype(np.float64))[:, None] + alpha * np.log(cos)
    mx = L.max(0)
    e = np.exp(L - mx)
    red = e[0] / (e.sum(0) + eps * np.exp(-mx))
    blue = e[1] / (e.sum(0) + eps * np.exp(-mx))
    tex = o["texture"][m]
    # 1e-6: the cameras are FP32 values, the closed form uses the exact positions
    assert np.abs(tex[ok, 0] - red[ok]).max() < 1e-6
    assert np.abs(tex[ok, 2] - blue[ok]).max() < 1e-6
    if alpha > 100:
        # the powers underflow; the log-space form still gives the better view's colour
        clear = ok & (np.abs(cos[0] - cos[1]) > 0.01)
        assert clear.sum() > 100
        assert (np.maximum(tex[clear, 0], tex[clear, 2]) > 0.999).all()
        assert np.array_equal(tex[clear, 0] > 0.5, (np.log(wts[0]) + alpha * np.log(cos[0]))[clear] >
                              (np.log(wts[1]) + alpha * np.log(cos[1]))[clear])


def test_backfacing_behind_camera_and_edges():
    # the plane's back side faces the camera: incidence 0, nothing filled
    V, F = _plane(4, flip=True)
    w = h = 48
    cam = _front_camera(3.0, w, h)
    img = np.full((1, h, w, 4), 90, np.uint8)
    W = H = 64
    uv = synth.grid_atlas(len(F), W, H, 2)
    o = oracle.backproject(V, F, uv, W, H, cam[None], img, np.ones(1, np.float32), alpha=1.0, eps=1e-6,
                           depth_tol=1e-3, edge_tol=0.2)
    assert not o["filled"].any()
    # a camera between the plane and ... looking away: every texel behind it
    Vp, Fp = _plane(4)
    R = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float64)     # forward = +z, away from the plane
    t = -R @ np.array([0.0, 0.0, 1.0])
    cam2 = np.concatenate([R.ravel(), t, [40, 40, w / 2, h / 2]]).astype(np.float32)
    o = oracle.backproject(Vp, Fp, uv, W, H, cam2[None], img, np.ones(1, np.float32), alpha=1.0, eps=1e-6,
                           depth_tol=1e-3, edge_tol=0.2)
    assert not o["filled"].any()
    # edge pixels: the silhouette of a small plane in front of the camera
    depth, point, near = oracle.render_views(Vp, Fp, _front_camera(3.0, w, h)[None], w, h)
    hit = np.isfinite(depth[0])
    rim = hit & ~(np.roll(hit, 1, 0) & np.roll(hit, -1, 0) & np.roll(hit, 1, 1) & np.roll(hit, -1, 1))
    # one flat sheet well inside the image: the edge pixels are exactly the hits beside a miss
    assert np.array_equal(oracle.edge_mask(depth, point, 0.2)[0].astype(bool), rim)
    o = oracle.backproject(Vp, Fp, uv, W, H, _front_camera(3.0, w, h)[None], img, np.ones(1, np.float32),
                           alpha=1.0, eps=1e-6, depth_tol=1e-3, edge_tol=0.2, views=(depth, point, near))
    m, p = _texel_points(o, Vp, Fp)
    u = np.floor(60 * p[:, 0] / 3.0 + w / 2).astype(int)
    v = np.floor(-60 * p[:, 1] / 3.0 + h / 2).astype(int)
    on_rim = rim[v.clip(0, h - 1), u.clip(0, w - 1)]
    assert on_rim.sum() > 20 and not o["filled"][m][on_rim].any()


# ---------------------------------------------------------------- anisotropic filtering

def _planar(n, size, s):
    """A flat grid in z = 0 with a planar atlas: uv = (x, y) * s + 1/2 per
    corner (one chart, similar to the surface, so texels are square on it)."""
    V, F = _plane(n, size=size)
    uv = (V[F][:, :, :2].astype(np.float64) * s + 0.5).astype(np.float32)
    return V, F, uv


def _bilinear(level, x, y):
    """Plain bilinear sample of an [h,w,3] array at continuous (x, y), pixel
    centres on the integer grid, clamped to the edge."""
    h, w = level.shape[:2]
    x0, y0 = np.floor(x).astype(int), np.floor(y).astype(int)
    ax, ay = x - x0, y - y0
    out = 0.0
    for dy in (0, 1):
        for dx in (0, 1):
            xx = np.clip(x0 + dx, 0, w - 1)
            yy = np.clip(y0 + dy, 0, h - 1)
            out = out + ((ax if dx else 1 - ax) * (ay if dy else 1 - ay))[..., None] * level[yy, xx]
    return out


def test_mip_pyramid_lanczos2():
    w, h = 100, 60
    img = np.zeros((h, w, 4), np.uint8)
    img[..., :3] = 77
    img[..., 3] = 255
    levels = oracle.mip_levels(img)
    assert [(P.shape[1], P.shape[0]) for P, _ in levels] == [(50, 30), (25, 15), (12, 7), (6, 3), (3, 1), (1, 1)]
    for P, S in levels:     # a constant stays constant, sharpened or not
        assert np.abs(P - 77 / 255).max() < 1e-12 and np.abs(S - 77 / 255).max() < 1e-12
    # a ramp in x: away from the border, level 1 is the ramp at the new pixel centres (X = 2j + 1)
    x = np.arange(w)
    img[..., 0] = 2 * x + 10
    P1, S1 = oracle.mip_levels(img)[0]
    j = np.arange(50)
    interior = (2 * j - 3 >= 0) & (2 * j + 4 <= w - 1)
    assert np.abs(P1[:, interior, 0] - (4 * j[interior] + 11) / 255).max() < 1e-12
    # the [1,2,1] unsharp mask leaves a ramp alone one pixel farther in
    inner = interior & np.roll(interior, 1) & np.roll(interior, -1)
    assert np.abs(S1[:, inner, 0] - P1[:, inner, 0]).max() < 1e-12
    # one brighter pixel on grey: level 1 holds the separable, normalised Lanczos-2 weights
    img[..., :3] = 128
    i0, j0 = 41, 27
    img[j0, i0, 0] = 228
    P1 = oracle.mip_levels(img)[0][0]
    t = np.arange(8)
    wt = np.sinc((t - 3.5) / 2) * np.sinc((t - 3.5) / 4)
    wt /= wt.sum()
    tx = i0 - 2 * np.arange(50) + 3
    ty = j0 - 2 * np.arange(30) + 3
    wx = np.where((tx >= 0) & (tx < 8), wt[np.clip(tx, 0, 7)], 0.0)
    wy = np.where((ty >= 0) & (ty < 8), wt[np.clip(ty, 0, 7)], 0.0)
    assert np.abs(P1[..., 0] - (128 + 100 * wy[:, None] * wx[None, :]) / 255).max() < 1e-12
    assert np.abs(P1[..., 1] - 128 / 255).max() < 1e-12


def test_aniso_taps_follow_the_footprint():
    """A plane seen 65 degrees off its normal through an image whose codes
    vary along u only: the colour is the mean of N equally spaced samples
    along the major axis of the texel's image footprint.  The expectation uses
    the exact derivative of the projection and numpy's SVD."""
    size, n, W = 10.0, 8, 512
    s = 0.45 / size
    V, F, uv = _planar(n, size, s)
    w = h = 48
    a = math.radians(65.0)
    eye = np.array([0.0, -4 * math.sin(a), 4 * math.cos(a)])
    cam = synth.look_at_camera(eye, [0, 0, 0], [0, 1, 0], 30.0, w, h)
    codes = (37 * np.arange(w) + 11) % 256
    img = np.zeros((1, h, w, 4), np.uint8)
    img[0, ..., 0] = codes[None, :]
    img[0, ..., 3] = 255
    kw = dict(alpha=1.0, eps=0.0, depth_tol=0.05, edge_tol=10.0)
    o = oracle.backproject(V, F, uv, W, W, cam[None], img, np.ones(1, np.float32), **kw)
    ob = oracle.backproject(V, F, uv, W, W, cam[None], img, np.ones(1, np.float32), filter="bilinear", **kw)
    m, p = _texel_points(o, V, F)
    R = cam[:9].astype(np.float64).reshape(3, 3)
    t = cam[9:12].astype(np.float64)
    fx, fy, cx, cy = (float(q) for q in cam[12:])
    c = p @ R.T + t
    u = fx * c[:, 0] / c[:, 2] + cx
    du = fx * (R[0][None] * c[:, 2:3] - c[:, 0:1] * R[2][None]) / c[:, 2:3] ** 2
    dv = fy * (R[1][None] * c[:, 2:3] - c[:, 1:2] * R[2][None]) / c[:, 2:3] ** 2
    dp = np.array([[1 / (s * W), 0.0], [0.0, 1 / (s * W)], [0.0, 0.0]])     # world per texel (x, y)
    J = np.stack([du @ dp, dv @ dp], 1)                                     # [n, 2 (u, v), 2 (x, y)]
    U, S, _ = np.linalg.svd(J)
    ratio = S[:, 0] / S[:, 1]
    N = np.clip(np.ceil(ratio - 0.05), 1, 8).astype(int)
    lam = np.log2(np.maximum(S[:, 1], S[:, 0] / 8)) - 0.5
    expect = np.zeros(len(p))
    for k in range(len(p)):
        taps = u[k] + U[k, 0, 0] * S[k, 0] * ((np.arange(N[k]) + 0.5) / N[k] - 0.5)
        expect[k] = np.mean(np.interp(taps - 0.5, np.arange(w), codes / 255))
    near = np.abs(ratio - 0.05 - np.round(ratio - 0.05)) < 1e-3
    ok = o["filled"][m].astype(bool) & (o["flags"][m] == 0) & ~near & (lam <= 0)
    assert ok.sum() > 2000 and (N[ok] >= 2).mean() > 0.9     # mostly two or three taps along u
    tex = o["texture"][m]
    assert np.abs(tex[ok, 0] - expect[ok]).max() < 1e-6
    # the single bilinear sample is a different (unfiltered) value
    assert np.abs(ob["texture"][m][ok, 0] - expect[ok]).max() > 0.05


def test_aniso_level_of_detail_trilinear():
    """A plane seen face-on from far away (an affine, isotropic footprint of
    4.5 pixels per texel): one tap, level log2(4.5) - 1/2 between pyramid
    levels 1 and 2, blended linearly."""
    size, n, W = 1.0, 4, 256
    s = 0.45 / size
    V, F, uv = _planar(n, size, s)
    w = h = 64
    D = 3.0
    sigma = 4.5
    f = sigma * s * W * D                 # pixels per texel = f / D * (1 / (s W))
    cam = _front_camera(D, w, h, f)
    rng = np.random.default_rng(5)
    img = np.zeros((1, h, w, 4), np.uint8)
    img[0, ..., :3] = rng.integers(0, 256, (h, w, 3))
    img[0, ..., 3] = 255
    o = oracle.backproject(V, F, uv, W, W, cam[None], img, np.ones(1, np.float32), alpha=1.0, eps=0.0,
                           depth_tol=0.05, edge_tol=10.0)
    m, p = _texel_points(o, V, F)
    u = f * p[:, 0] / D + w / 2
    v = -f * p[:, 1] / D + h / 2
    lam = math.log2(sigma) - 0.5
    fr = lam - 1
    S1 = oracle.mip_levels(img[0])[0][1]
    S2 = oracle.mip_levels(img[0])[1][1]
    expect = (1 - fr) * _bilinear(S1, u / 2 - 0.5, v / 2 - 0.5) + fr * _bilinear(S2, u / 4 - 0.5, v / 4 - 0.5)
    inside = (u > 0) & (u < w) & (v > 0) & (v < h)
    ok = o["filled"][m].astype(bool) & (o["flags"][m] == 0) & inside
    assert ok.sum() > 50
    assert np.abs(o["texture"][m][ok] - expect[ok]).max() < 1e-6


def test_variants_list_the_results_of_every_rounding_choice():
    """The set of correct results of a flagged texel (the set-valued check of
    the GPU parity tests).  Two constant-colour views (red, blue) of a plane
    with eps = 0: a blend of both is the closed form, of one view alone that
    view's colour exactly, of none an unfilled texel.  A texel whose
    projection lies within 1e-3 pixel of a pixel boundary in one view only
    has exactly two correct results, with that view and without it; in both
    views, four.  The texel's own result is always one of them."""
    V, F = _plane(8, size=1.5)
    w = h = 48
    cams = []
    for ang in (10.0, 50.0):
        a = math.radians(ang)
        cams.append(synth.look_at_camera([4 * math.sin(a), 0.0, 4 * math.cos(a)], [0, 0, 0], [0, 1, 0], 30.0, w, h))
    cams = np.stack(cams)
    img = np.zeros((2, h, w, 4), np.uint8)
    img[0, ..., 0] = 255
    img[1, ..., 2] = 255
    img[..., 3] = 255
    wts = np.array([0.3, 1.0], np.float32)
    W = H = 512
    uv = synth.grid_atlas(len(F), W, H, 2)
    for filt in ("bilinear", "aniso"):
        o = oracle.backproject(V, F, uv, W, H, cams, img, wts, alpha=6.0, eps=0.0, depth_tol=0.1, edge_tol=10.0,
                               filter=filt, variants=True)
        m, p = _texel_points(o, V, F)
        inner = np.abs(p[:, :2]).max(1) < 0.5                      # inside both frusta, away from the rims
        ids = np.flatnonzero(m.reshape(-1))
        # each view's pixel coordinates of the texel point, in FP64 from the FP32 cameras
        near_bd = []
        for k in range(2):
            c = cams[k].astype(np.float64)
            R, t, (fx, fy, cx, cy) = c[:9].reshape(3, 3), c[9:12], c[12:16]
            q = p @ R.T + t
            u, v = fx * q[:, 0] / q[:, 2] + cx, fy * q[:, 1] / q[:, 2] + cy
            fr = np.minimum(np.abs(u - np.round(u)), np.abs(v - np.round(v)))
            near_bd.append(fr < 1e-3)
        near_bd = np.stack(near_bd)
        C = [cams[k][:9].astype(np.float64).reshape(3, 3).T @ -cams[k][9:12].astype(np.float64) for k in range(2)]
        cos = np.stack([(c[None] - p)[:, 2] / np.linalg.norm(c[None] - p, axis=1) for c in C])
        L = np.log(wts.astype(np.float64))[:, None] + 6.0 * np.log(cos)
        e = np.exp(L - L.max(0))
        both = np.stack([e[0] / e.sum(0), np.zeros(len(p)), e[1] / e.sum(0)], -1)
        one = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])]
        n_single = n_double = 0
        for r, tex in enumerate(ids):
            if not inner[r]:
                continue
            fl = o["flags"].reshape(-1)[tex]
            assert fl == bool(near_bd[:, r].any()), (filt, tex)
            if not fl:
                continue
            var = o["variants"][int(tex)]
            own = np.concatenate([o["texture"].reshape(-1, 3)[tex], [o["filled"].reshape(-1)[tex]]])
            assert np.abs(var - own).max(1).min() < 1e-12
            def has(x, filled=1.0):
                return np.abs(var - np.concatenate([x, [filled]])).max(1).min() < 1e-9
            if near_bd[:, r].sum() == 1:
                k = int(np.flatnonzero(near_bd[:, r])[0])
                assert len(var) == 2 and has(both[r]) and has(one[1 - k])
                n_single += 1
            else:
                assert len(var) == 4 and has(both[r]) and has(one[0]) and has(one[1]) and has(np.zeros(3), 0.0)
                n_double += 1
        assert n_single > 50, (filt, n_single)
