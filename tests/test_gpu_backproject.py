"""GPU parity of UV-space backprojection and incidence blending (Sec. 7.4)
against the FP64 oracle through the C ABI (ag_render_views, ag_backproject).

The generated views are stand-ins made from the oracle's own renders (a smooth
colour field at each pixel's surface point), so no input comes from the CUDA
path.  The kernel renders its own depth buffers and edge masks.  Where the
oracle flags a texel (a pixel boundary, the depth limit, an edge decision or a
silhouette within rounding of the decision, or an anisotropic tap count or
fallback at its threshold), the oracle lists every correct result (each
rounding-dependent view counted or not, each threshold taken either way) and
the kernel's texel must be one of them."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_26137_b300 import synth

pytestmark = pytest.mark.gpu

TOL_TEX = 1e-4


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_both(lv, lf, uv, W, H, cams, weights, w, h, *, alpha, eps, depth_tol, edge_tol):
    import paper_2605_26137_b300 as pb
    depth_o, point_o, near_o = oracle.render_views(lv, lf, cams, w, h)
    images = synth.view_images(point_o)
    o = oracle.backproject(lv, lf, uv, W, H, cams, images, weights, alpha=alpha, eps=eps, depth_tol=depth_tol,
                           edge_tol=edge_tol, views=(depth_o, point_o, near_o), variants=True)
    bvh = pb.Bvh(_t(lv), _t(lf))
    depth, pts, edge = pb.render_views(bvh, cams, w, h, edge_tol=edge_tol)
    tex, inc = pb.backproject(_t(lv), _t(lf), _t(uv), W, H, cams, weights, _t(images), depth, edge, alpha=alpha,
                              eps=eps, depth_tol=depth_tol, incidence=True)
    pb.sync_status()
    bvh.free()
    g = dict(depth=depth.cpu().numpy(), points=pts.cpu().numpy(), edge=edge.cpu().numpy(),
             texture=tex.cpu().numpy(), incidence=inc.cpu().numpy())
    return g, o


def check_render(g, o, scale):
    near = o["near"].astype(bool)
    hit_o = np.isfinite(o["depth"])
    hit_g = np.isfinite(g["depth"])
    assert np.array_equal(hit_g[~near], hit_o[~near])
    both = hit_o & hit_g & ~near
    assert np.abs(g["depth"][both] - o["depth"][both]).max() <= 1e-5 * scale
    assert np.abs(g["points"][both] - o["point"][both]).max() <= 1e-5 * scale


def check_texture(g, o, sample=None):
    """Texels the oracle does not flag by value; flagged ones against the
    oracle's list of correct results.  Returns the fraction of compared
    texels checked either way (texels whose list was too long to write are
    the rest, at most 1 %)."""
    ray = o["face"] >= 0
    if sample is not None:
        sel = np.zeros(ray.size, bool)
        sel[np.asarray(sample)] = True
        sel = sel.reshape(ray.shape) & ray
    else:
        sel = ray
    ok = sel & (o["flags"] == 0)
    filled_g = g["texture"][..., 3] > 0.5
    assert np.array_equal(filled_g[ok], o["filled"][ok].astype(bool))
    both = ok & filled_g
    err = np.abs(g["texture"][..., :3][both] - o["texture"][both])
    assert err.max() <= TOL_TEX, err.max()
    if "incidence" in g:
        inc = np.abs(g["incidence"][:, ok] - o["incidence"][:, ok])
        assert inc.max() <= 1e-5
    # outside the ray texels nothing is written
    if sample is None:
        assert not g["texture"][~ray].any()
    gt = g["texture"].reshape(-1, 4)
    n_set = n_unlisted = 0
    for tex in np.flatnonzero((sel & (o["flags"] != 0)).reshape(-1)):
        var = o["variants"][int(tex)]
        if len(var) == 0:
            n_unlisted += 1
            continue
        fill = 1.0 if gt[tex, 3] > 0.5 else 0.0
        d = np.abs(var[:, :3] - gt[tex, :3]).max(1)
        assert ((var[:, 3] == fill) & (d <= TOL_TEX)).any(), (int(tex), gt[tex], var)
        n_set += 1
    assert n_unlisted <= 0.01 * sel.sum(), n_unlisted
    return float((ok.sum() + n_set) / sel.sum())


@pytest.mark.parametrize("seed", [0, 1])
def test_paper_views_tiny_asset(seed):
    a = synth.tiny_asset(seed)
    lv, lf = a.low_v, a.low_f
    c = (lv.max(0) + lv.min(0)) / 2
    r = float(np.linalg.norm(lv.max(0) - lv.min(0)) / 2)
    cams, weights, _ = synth.paper_cameras(c, r, 96, 80)
    scale = 2 * r
    g, o = run_both(lv, lf, a.low_uv, a.W, a.H, cams, weights, 96, 80, alpha=6.0, eps=1e-6, depth_tol=0.02 * scale,
                    edge_tol=0.05 * scale)
    check_render(g, o, scale)
    frac = check_texture(g, o)
    assert frac > 0.99
    assert o["filled"][o["face"] >= 0].mean() > 0.6


def test_sdf_asset_large_alpha_and_ragged_sizes():
    """A marching-grid low mesh (~6k faces), a 512 x 384 atlas, views of
    ragged sizes, alpha = 40 (the log-space blend)."""
    a = synth.sdf_asset(7, 60_000, 6_000, 512, 384, n_prims=16)
    lv, lf = a.low_v, a.low_f
    c = (lv.max(0) + lv.min(0)) / 2
    r = float(np.linalg.norm(lv.max(0) - lv.min(0)) / 2)
    # views dense enough that a pixel covers few texels (a flagged pixel flags them all)
    cams, weights, _ = synth.paper_cameras(c, r, 509, 383)
    scale = 2 * r
    g, o = run_both(lv, lf, a.low_uv, a.W, a.H, cams, weights, 509, 383, alpha=40.0, eps=1e-30,
                    depth_tol=0.01 * scale, edge_tol=0.03 * scale)
    check_render(g, o, scale)
    # a pixel whose render depends on rounding flags every texel that lands on
    # it or beside it in any view (on this marching-grid mesh about a fifth);
    # those are checked against the oracle's list of correct results
    assert check_texture(g, o) > 0.99


def test_render_modes_against_oracle():
    """Raster proposals and full tracing against the oracle's renders: the
    paper's ten views of a ~6k-face surface at a ragged size, and a camera
    inside the mesh's box (triangles behind the camera plane: that view is
    traced whole)."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(11, 60_000, 6_000, 512, 512, n_prims=16)
    lv, lf = a.low_v, a.low_f
    c = (lv.max(0) + lv.min(0)) / 2
    r = float(np.linalg.norm(lv.max(0) - lv.min(0)) / 2)
    w, h = 301, 217
    cams, _, _ = synth.paper_cameras(c, r, w, h)
    inside = synth.look_at_camera(c + np.array([0.05, 0.02, 0.03]) * r, c + np.array([1.0, 0.1, 0.0]) * r,
                                  [0, 1, 0], 70.0, w, h)
    cams = np.concatenate([cams, inside[None]])
    depth_o, point_o, near_o = oracle.render_views(lv, lf, cams, w, h)
    bvh = pb.Bvh(_t(lv), _t(lf))
    o = dict(depth=depth_o, point=point_o, near=near_o)
    outs = {}
    for mode in ("raster", "trace"):
        depth, pts, edge = pb.render_views(bvh, cams, w, h, edge_tol=0.03 * 2 * r, render=mode)
        pb.sync_status()
        g = dict(depth=depth.cpu().numpy(), points=pts.cpu().numpy(), edge=edge.cpu().numpy())
        check_render(g, o, 2 * r)
        outs[mode] = g
    # the modes differ at most where a pixel's render depends on rounding
    near = near_o.astype(bool)
    assert np.isfinite(depth_o[-1]).mean() > 0.1    # the inside view sees the surface
    same = outs["raster"]["depth"] == outs["trace"]["depth"]
    assert same[~near].mean() > 0.999
    bvh.free()


@pytest.mark.parametrize("alpha,eps,filt", [(6.0, 1e-6, "aniso"), (40.0, 1e-30, "aniso"), (6.0, 1e-6, "bilinear")])
def test_backproject_on_oracle_views(alpha, eps, filt):
    """The blend step alone: the kernel reads the oracle's depth buffers (as
    FP32) and edge masks, so a pixel whose render depends on rounding cannot
    change the comparison; only texels within rounding of a pixel boundary,
    the depth limit or the image border are skipped."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(3, 40_000, 4_000, 384, 256, n_prims=12)
    lv, lf = a.low_v, a.low_f
    c = (lv.max(0) + lv.min(0)) / 2
    r = float(np.linalg.norm(lv.max(0) - lv.min(0)) / 2)
    w, h = 333, 250
    cams, weights, _ = synth.paper_cameras(c, r, w, h)
    scale, edge_tol = 2 * r, 0.03 * 2 * r
    depth_o, point_o, near_o = oracle.render_views(lv, lf, cams, w, h)
    edge_o = oracle.edge_mask(depth_o, point_o, edge_tol)
    images = synth.view_images(point_o)
    o = oracle.backproject(lv, lf, a.low_uv, a.W, a.H, cams, images, weights, alpha=alpha, eps=eps,
                           depth_tol=0.01 * scale, edge_tol=edge_tol, views=(depth_o, point_o, np.zeros_like(near_o)),
                           filter=filt, variants=True)
    tex, inc = pb.backproject(_t(lv), _t(lf), _t(a.low_uv), a.W, a.H, cams, weights, _t(images),
                              _t(depth_o.astype(np.float32)), _t(edge_o), alpha=alpha, eps=eps,
                              depth_tol=0.01 * scale, incidence=True, filter=filt)
    pb.sync_status()
    g = dict(texture=tex.cpu().numpy(), incidence=inc.cpu().numpy())
    assert check_texture(g, o) > 0.99
    assert o["filled"][o["face"] >= 0].mean() > 0.8


def test_face_on_affine_image_closed_form():
    """The oracle's closed form, through the kernel: a plane seen face-on
    through an image whose codes are affine in the pixel index."""
    import paper_2605_26137_b300 as pb
    n = 4
    xs = np.linspace(-1, 1, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], -1).astype(np.float32)
    F = np.asarray([(j * (n + 1) + i, j * (n + 1) + i + 1, j * (n + 1) + i + n + 2) for j in range(n) for i in range(n)] +
                   [(j * (n + 1) + i, j * (n + 1) + i + n + 2, j * (n + 1) + i + n + 1) for j in range(n) for i in range(n)],
                   np.int32)
    w = h = 64
    D, f = 3.0, 60.0
    R = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float64)
    cam = np.concatenate([R.ravel(), -R @ [0, 0, D], [f, f, w / 2, h / 2]]).astype(np.float32)[None]
    ii, jj = np.meshgrid(np.arange(w), np.arange(h))
    img = np.zeros((1, h, w, 4), np.uint8)
    img[0, ..., 0] = 2 * ii + 40
    img[0, ..., 1] = 3 * jj + 20
    img[0, ..., 3] = 255
    W = H = 64
    uv = synth.grid_atlas(len(F), W, H, 2)
    bvh = pb.Bvh(_t(V), _t(F))
    depth, _, edge = pb.render_views(bvh, cam, w, h, edge_tol=1.0)
    tex = pb.backproject(_t(V), _t(F), _t(uv), W, H, cam, np.ones(1, np.float32), _t(img), depth, edge, alpha=1.0,
                         eps=0.0, depth_tol=1e-3)
    pb.sync_status()
    tex = tex.cpu().numpy()
    face, bary, _ = oracle.raster(uv, W, H)
    m = face >= 0
    p = (bary[m][:, :, None] * V.astype(np.float64)[F[face[m]]]).sum(1)
    u = f * p[:, 0] / D + w / 2
    v = -f * p[:, 1] / D + h / 2
    margin = 1.0 - 2.5 * D / f
    inner = (np.abs(p[:, 0]) < margin) & (np.abs(p[:, 1]) < margin) & (np.abs(u - np.round(u)) > 1e-3) & \
        (np.abs(v - np.round(v)) > 1e-3)
    t = tex[m]
    assert inner.sum() > 1000 and (t[inner, 3] == 1).all()
    assert np.abs(t[inner, 0] - (2 * (u[inner] - 0.5) + 40) / 255).max() < 2e-5
    assert np.abs(t[inner, 1] - (3 * (v[inner] - 0.5) + 20) / 255).max() < 2e-5
    bvh.free()


def test_argument_errors():
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(0)
    bvh = pb.Bvh(_t(a.low_v), _t(a.low_f))
    cams, weights, _ = synth.paper_cameras(np.zeros(3), 1.0, 32, 32)
    depth, _, edge = pb.render_views(bvh, cams, 32, 32, edge_tol=0.1)
    imgs = torch.zeros((10, 32, 32, 4), dtype=torch.uint8, device="cuda")
    bad = weights.copy()
    bad[3] = 0.0
    with pytest.raises(pb.AgError):
        pb.backproject(_t(a.low_v), _t(a.low_f), _t(a.low_uv), a.W, a.H, cams, bad, imgs, depth, edge, alpha=2.0,
                       eps=1e-6, depth_tol=0.01)
    with pytest.raises(pb.AgError):
        pb.render_views(bvh, cams, 0, 32, edge_tol=0.1)
    with pytest.raises(ValueError):
        pb.backproject(_t(a.low_v), _t(a.low_f), _t(a.low_uv), a.W, a.H, cams[:5], weights, imgs, depth, edge,
                       alpha=2.0, eps=1e-6, depth_tol=0.01)
    bvh.free()


def _planar(n, size, s):
    xs = np.linspace(-size, size, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], -1).astype(np.float32)
    F = np.asarray([(j * (n + 1) + i, j * (n + 1) + i + 1, j * (n + 1) + i + n + 2) for j in range(n) for i in range(n)] +
                   [(j * (n + 1) + i, j * (n + 1) + i + n + 2, j * (n + 1) + i + n + 1) for j in range(n) for i in range(n)],
                   np.int32)
    uv = (V[F][:, :, :2].astype(np.float64) * s + 0.5).astype(np.float32)
    return V, F, uv


@pytest.mark.parametrize("case", ["oblique", "far"])
def test_aniso_footprints(case):
    """The anisotropic filter against the oracle where it does most: a plane
    65 degrees off the view axis (two or three taps along the major axis) and
    a plane far away (footprints of several pixels: trilinear between pyramid
    levels), each filling a ragged-size view with a seeded random image."""
    import paper_2605_26137_b300 as pb
    import math
    rng = np.random.default_rng(9)
    if case == "oblique":
        size, n, W, w, h = 10.0, 8, 512, 61, 47
        a = math.radians(65.0)
        cam = synth.look_at_camera([0.0, -4 * math.sin(a), 4 * math.cos(a)], [0, 0, 0], [0, 1, 0], 30.0, w, h)
    else:
        size, n, W, w, h = 1.0, 4, 256, 70, 52
        D, f = 3.0, 4.5 * 0.45 * 256 * 3.0
        R = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float64)
        cam = np.concatenate([R.ravel(), -R @ [0, 0, D], [f, f, w / 2, h / 2]]).astype(np.float32)
    V, F, uv = _planar(n, size, 0.45 / size)
    img = np.zeros((1, h, w, 4), np.uint8)
    img[0, ..., :3] = rng.integers(0, 256, (h, w, 3))
    img[0, ..., 3] = 255
    depth_o, point_o, near_o = oracle.render_views(V, F, cam[None], w, h)
    edge_o = oracle.edge_mask(depth_o, point_o, 10.0)
    kw = dict(alpha=1.0, eps=0.0, depth_tol=0.05)
    o = oracle.backproject(V, F, uv, W, W, cam[None], img, np.ones(1, np.float32), edge_tol=10.0,
                           views=(depth_o, point_o, near_o), variants=True, **kw)
    tex = pb.backproject(_t(V), _t(F), _t(uv), W, W, cam[None], np.ones(1, np.float32), _t(img),
                         _t(depth_o.astype(np.float32)), _t(edge_o), **kw)
    pb.sync_status()
    g = tex.cpu().numpy()
    ok = (o["face"] >= 0) & (o["flags"] == 0) & o["filled"].astype(bool)
    assert ok.sum() > (2000 if case == "oblique" else 100)
    assert np.array_equal(g[..., 3][ok] > 0.5, np.ones(ok.sum(), bool))
    err = np.abs(g[..., :3][ok] - o["texture"][ok])
    assert err.max() <= TOL_TEX, err.max()
    assert check_texture(dict(texture=g), o) > 0.99


def test_bench_configuration_sampled():
    """The benchmark's backprojection workload: the paper's ten views at
    1024^2 of the headline asset's ~31.7k-face low mesh onto its 2048^2 grid
    atlas, alpha = 6, the bench's depth and edge tolerances.  The kernel
    renders its views and blends; 20k seeded ray texels are compared with the
    oracle (its own renders, its own colour images for both sides)."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(1, 2_000_000, 30_000, 2048, 2048, n_prims=32, device="cuda")
    lv, lf = a.low_v, a.low_f
    V = lv.astype(np.float64)
    c = (V.max(0) + V.min(0)) / 2
    r = float(np.linalg.norm(V.max(0) - V.min(0)) / 2)
    w = h = 1024
    cams, weights, _ = synth.paper_cameras(c, r, w, h)
    diam = 2 * r
    edge_tol, depth_tol = 0.01 * diam, 0.005 * diam
    depth_o, point_o, near_o = oracle.render_views(lv, lf, cams, w, h)
    images = synth.view_images(point_o)
    face, _, _ = oracle.raster(a.low_uv, a.W, a.H)
    rays = np.flatnonzero(face.reshape(-1) >= 0)
    sample = np.sort(np.random.default_rng(4).choice(rays, 20000, replace=False))
    o = oracle.backproject(lv, lf, a.low_uv, a.W, a.H, cams, images, weights, alpha=6.0, eps=1e-6,
                           depth_tol=depth_tol, edge_tol=edge_tol, views=(depth_o, point_o, near_o), sample=sample,
                           variants=True)
    bvh = pb.Bvh(_t(lv), _t(lf))
    depth, pts, edge = pb.render_views(bvh, cams, w, h, edge_tol=edge_tol)
    tex = pb.backproject(_t(lv), _t(lf), _t(a.low_uv), a.W, a.H, cams, weights, _t(images), depth, edge, alpha=6.0,
                         eps=1e-6, depth_tol=depth_tol)
    pb.sync_status()
    bvh.free()
    check_render(dict(depth=depth.cpu().numpy(), points=pts.cpu().numpy()),
                 dict(depth=depth_o, point=point_o, near=near_o), diam)
    frac = check_texture(dict(texture=tex.cpu().numpy()), o, sample=sample)
    print("compared by value or set:", frac, "flagged:", float((o["flags"].reshape(-1)[sample] != 0).mean()))
    assert frac > 0.99


def test_aniso_jittered_atlas_and_degenerate_uv():
    """Random off-lattice UV triangles (strongly anisotropic and varied
    footprints, some faces with zero or tiny UV area: the centre-sample
    fallback) on the paper's views of the tiny asset, on the oracle's views."""
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(3)
    lv, lf = a.low_v, a.low_f
    W = H = 256
    uv = synth.jittered_atlas(len(lf), W, H, seed=4)
    # a few faces shrunk to 0.02 x 0.006 texel (UV area 6e-5 texel^2, below the
    # footprint's 1e-4 limit): each still owns the texel it sits in
    tiny = np.arange(0, len(lf), 7)
    for f in tiny:
        p = uv[f].astype(np.float64) * [W, H]
        x0, y0 = np.floor(p[:, 0].mean()) + 0.4, np.floor(p[:, 1].mean()) + 0.4
        uv[f] = (np.array([[x0, y0], [x0 + 0.02, y0], [x0 + 0.02, y0 + 0.006]]) / [W, H]).astype(np.float32)
    c = (lv.max(0) + lv.min(0)) / 2
    r = float(np.linalg.norm(lv.max(0) - lv.min(0)) / 2)
    w, h = 161, 119
    cams, weights, _ = synth.paper_cameras(c, r, w, h)
    depth_o, point_o, near_o = oracle.render_views(lv, lf, cams, w, h)
    edge_o = oracle.edge_mask(depth_o, point_o, 0.05 * 2 * r)
    images = synth.view_images(point_o)
    kw = dict(alpha=6.0, eps=1e-6, depth_tol=0.02 * 2 * r)
    o = oracle.backproject(lv, lf, uv, W, H, cams, images, weights, edge_tol=0.05 * 2 * r,
                           views=(depth_o, point_o, np.zeros_like(near_o)), variants=True, **kw)
    tex = pb.backproject(_t(lv), _t(lf), _t(uv), W, H, cams, weights, _t(images), _t(depth_o.astype(np.float32)),
                         _t(edge_o), **kw)
    pb.sync_status()
    g = dict(texture=tex.cpu().numpy(), incidence=np.zeros((len(cams), H, W), np.float32))
    o2 = dict(o)
    o2["incidence"] = np.zeros_like(g["incidence"])
    assert check_texture(g, o2) > 0.99
    # the centre-sample fallback was compared on filled texels of the shrunk faces
    on_tiny = np.isin(o["face"], tiny) & (o["flags"] == 0) & o["filled"].astype(bool)
    assert on_tiny.sum() >= 5


def test_render_many_views_in_chunks():
    """130 views of 1024 x 1008 pixels: more than one chunk of z-buffer keys
    (1.5 GiB per chunk); the raster proposals give the traced buffers, and a
    sample of pixels matches the oracle's render."""
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(1)
    lv, lf = a.low_v, a.low_f
    c = (lv.max(0) + lv.min(0)) / 2
    r = float(np.linalg.norm(lv.max(0) - lv.min(0)) / 2)
    w, h, K = 1024, 1008, 130
    rng = np.random.default_rng(3)
    cams = []
    for k in range(K):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        cams.append(synth.look_at_camera(c + 3.2 * r * d, c, [0, 1, 0] if abs(d[1]) < 0.9 else [1, 0, 0], 40.0, w, h))
    cams = np.stack(cams)
    bvh = pb.Bvh(_t(lv), _t(lf))
    dr, _, er = pb.render_views(bvh, cams, w, h, edge_tol=0.05 * r, points=False)
    dt, _, et = pb.render_views(bvh, cams, w, h, edge_tol=0.05 * r, points=False, render="trace")
    pb.sync_status()
    bvh.free()
    dr, dt = dr.cpu().numpy(), dt.cpu().numpy()
    assert np.isfinite(dr).mean() > 0.1
    assert (dr == dt).mean() > 0.9999 and (np.isfinite(dr) == np.isfinite(dt)).mean() > 0.9999
    # the last chunk's views against the oracle on a sample of rows
    ks = [0, 64, 129]
    depth_o, point_o, near_o = oracle.render_views(lv, lf, cams[ks], w, h)
    # depth by value away from edge pixels: at a grazing hit the ray parameter
    # is ill-conditioned (rounding of the hit point divided by the grazing
    # angle's sine), and the blend never reads an edge pixel
    edge_o = oracle.edge_mask(depth_o, point_o, 0.05 * r).astype(bool)
    rows = rng.choice(h, 24, replace=False)
    for q, k in enumerate(ks):
        sel = ~near_o[q][rows].astype(bool)
        go, oo = dr[k][rows][sel], depth_o[q][rows][sel]
        assert np.array_equal(np.isfinite(go), np.isfinite(oo))
        fin = np.isfinite(oo) & ~edge_o[q][rows][sel]
        assert np.abs(go[fin] - oo[fin]).max() <= 1e-5 * 2 * r
