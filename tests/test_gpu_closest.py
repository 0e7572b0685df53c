"""GPU parity of the closest-point correspondence (Sec. 6.4 as worded: the
closest point of the high surface to each texel's position) against the FP64
oracle, through the C ABI, with the same tolerances as the ray query."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_26137_b300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


def _t(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dtype)


def gpu_bake(asset, layout="q8", bvh=None, **kw):
    import paper_2605_26137_b300 as pb
    if bvh is None:
        bvh = pb.Bvh(_t(asset.high_v), _t(asset.high_f), layout=layout)
    lv, lf, uv = _t(asset.low_v), _t(asset.low_f), _t(asset.low_uv)
    out = pb.bake(bvh, lv, lf, uv, asset.W, asset.H, asset.max_dist, gutter=asset.gutter, aux=True,
                  query="closest", **kw)
    pb.sync_status()
    return bvh, parity.to_numpy(out), out


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("layout", ["q8", "f32"])
def test_tiny_closest_matches_brute_force_oracle(seed, layout):
    a = synth.tiny_asset(seed)
    o = oracle.bake_asset(a, use_bvh=False, query="closest")
    _, g, _ = gpu_bake(a, layout)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a, query="closest")
    print(st)
    parity.check(st)
    assert st["n_ray"] == 4000


@pytest.mark.parametrize("W,H,seed", [(100, 77, 3), (129, 64, 4), (64, 200, 5)])
def test_closest_jittered_atlas_ragged_sizes(W, H, seed):
    lv, lf = synth.icosphere(2)
    hv, hf = synth.sh_displaced_sphere(4, seed)
    uv = synth.jittered_atlas(len(lf), W, H, seed)
    a = synth.Asset(hv, hf, lv, lf, uv, W, H, 0.15, 2)
    o = oracle.bake_asset(a, query="closest")
    _, g, _ = gpu_bake(a)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a, query="closest")
    print(st)
    parity.check(st)


def test_closest_sdf_asset_and_layouts_identical():
    """The pipeline-output shape (marching-grid union of primitives, ~120k
    high faces, 512x384 atlas); the Q8 and FP32 node layouts give the same
    bytes because box pruning never rejects the closest triangle."""
    a = synth.sdf_asset(7, 120_000, 6_000, 512, 384, n_prims=16)
    o = oracle.bake_asset(a, query="closest")
    _, g, _ = gpu_bake(a, "q8")
    st = parity.compare(g, o, a.diam, a.gutter, asset=a, query="closest")
    print(st)
    parity.check(st)
    _, g2, _ = gpu_bake(a, "f32")
    for k in ("normal_rgba8", "mask", "hit_tri"):
        assert np.array_equal(g[k], g2[k]), k
    assert np.array_equal(g["disp_f32"].view(np.uint32), g2["disp_f32"].view(np.uint32))


def _plane(n, z, size):
    xs = np.linspace(-size, size, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.asarray(F, np.int32)


def test_closest_plane_and_identity_closed_forms():
    """A flat high plane: (0,0,1) and the signed offset on every ray texel;
    identical meshes: (0,0,1) and zero displacement."""
    lv, lf = _plane(6, 0.0, 1.0)
    for z in (0.03, -0.02):
        hv, hf = _plane(20, z, 1.5)
        uv = synth.grid_atlas(len(lf), 64, 64, 2)
        a = synth.Asset(hv, hf, lv, lf, uv, 64, 64, 0.05, 2)
        _, g, _ = gpu_bake(a)
        m = g["face"] >= 0
        assert m.sum() > 0 and g["mask"][m].all()
        assert np.abs(g["normal_ts"][m] - [0, 0, 1]).max() < 1e-6
        assert np.abs(g["disp_f32"][m] - np.float32(z)).max() < 1e-7
    V, F = synth.sh_displaced_sphere(3, 11)
    uv = synth.grid_atlas(len(F), 256, 256, 2)
    a = synth.Asset(V, F, V, F, uv, 256, 256, 0.1, 2)
    _, g, _ = gpu_bake(a)
    m = g["face"] >= 0
    assert g["mask"][m].all()
    assert np.abs(g["disp_f32"][m]).max() < 1e-6 * a.diam
    assert np.abs(g["normal_ts"][m] - [0, 0, 1]).max() < 1e-5


def test_closest_batch_and_graph_equal_single_bakes():
    import paper_2605_26137_b300 as pb
    assets = [synth.tiny_asset(s, W=96 + 32 * s, H=128) for s in range(3)]
    singles, batch_in, plan_in = [], [], []
    for a in assets:
        bvh, g, _ = gpu_bake(a)
        singles.append(g)
        args = dict(bvh=bvh, low_verts=_t(a.low_v), low_faces=_t(a.low_f), low_uv=_t(a.low_uv), W=a.W, H=a.H,
                    max_dist=a.max_dist)
        batch_in.append(pb.Asset(**args))
        plan_in.append(pb.Asset(**args))
    outs = pb.bake_batch(batch_in, query="closest")
    plan = pb.BatchPlan(plan_in, query="closest")
    plan.launch()
    pb.sync_status()
    for g, ob, op in zip(singles, outs, [x.out for x in plan_in]):
        for out in (ob, op):
            assert np.array_equal(out.normal_rgba8.cpu().numpy(), g["normal_rgba8"])
            assert np.array_equal(out.mask.cpu().numpy(), g["mask"])
            assert np.array_equal(out.disp.cpu().numpy().view(np.uint16), g["disp"].view(np.uint16))
    plan.free()


def test_closest_launch_configurations_identical_and_step_cap():
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(5, 40_000, 2_000, 256, 192, n_prims=10)
    bvh = pb.Bvh(_t(a.high_v), _t(a.high_f))
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    ref = None
    for tile in ("8x8", "16x16", "32x8", "4x4"):
        for block in (64, 256):
            o = pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, ray_tile=tile, block_size=block, query="closest")
            pb.sync_status()
            got = (o.normal_rgba8.cpu().numpy(), o.mask.cpu().numpy(), o.disp.cpu().numpy().view(np.uint16))
            if ref is None:
                ref = got
            for x, y in zip(got, ref):
                assert np.array_equal(x, y), (tile, block)
    pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, max_steps=1, query="closest")
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 4
    # the backward pass is defined for the ray query only
    with pytest.raises(pb.AgError) as ei:
        from paper_2605_26137_b300 import _lib
        lib = _lib.load()
        import ctypes
        o = _lib.default_opts(query=_lib.AG_QUERY_CLOSEST)
        loss = torch.zeros(1, device="cuda")
        _lib.check(lib.ag_bake_backward(bvh.handle, lv.data_ptr(), uv.data_ptr(), lf.data_ptr(), lv.shape[0],
                                        lf.shape[0], a.W, a.H, float(a.max_dist), 0.1, ctypes.byref(o),
                                        torch.cuda.current_stream().cuda_stream, loss.data_ptr(), None))
    assert ei.value.status == 1


@pytest.mark.slow
def test_closest_full_size_sampled_parity():
    """The benchmark workload (~2M high-poly triangles, 2048^2 atlas): a seeded
    sample of texels against the oracle, unit normals everywhere."""
    a = synth.sdf_asset(1, 2_000_000, 30_000, 2048, 2048, n_prims=32)
    bvh, g, _ = gpu_bake(a)
    face = g["face"]
    rays = np.flatnonzero(face.reshape(-1) >= 0)
    rng = np.random.default_rng(1)
    sample = np.sort(rng.choice(rays, size=3000, replace=False))
    o = oracle.bake_asset(a, sample=sample, query="closest")
    assert np.array_equal(o["face"], face)
    st = parity.compare(g, o, a.diam, a.gutter, sample=sample, asset=a, query="closest")
    print(st)
    parity.check(st, small=0)
    n = g["normal_ts"]
    filled = g["normal_rgba8"][..., 3] == 255
    assert np.abs(np.linalg.norm(n[filled], axis=-1) - 1).max() < 1e-5
    bvh.free()


def test_point_distance_matches_oracle():
    """ag_point_distance: distances from random points near and far from a
    marching-grid surface against the oracle's closest point."""
    import paper_2605_26137_b300 as pb
    V, F = synth.sdf_mesh(synth.sdf_union_params(4, 12), 40, device="cpu")
    diam = float(np.linalg.norm(V.max(0) - V.min(0)))
    rng = np.random.default_rng(3)
    pts = np.concatenate([V[rng.integers(0, len(V), 3000)] + rng.normal(scale=0.02, size=(3000, 3)),
                          rng.uniform(-1.5, 1.5, size=(1000, 3))]).astype(np.float32)
    bvh = pb.Bvh(_t(V), _t(F))
    max_dist = 0.1
    d, tri = pb.point_distance(bvh, _t(pts), max_dist, tri=True)
    pb.sync_status()
    d, tri = d.cpu().numpy().astype(np.float64), tri.cpu().numpy()
    ob = oracle.Bvh(V, F)
    for k, p in enumerate(pts):
        t, d2, _, _ = oracle.closest_point(V, F, p.astype(np.float64), max_dist, bvh=ob)
        if t < 0:
            assert d[k] == -1.0 or abs(d[k] - max_dist) < 1e-6 * diam
            continue
        assert abs(d[k] - np.sqrt(d2)) <= 1e-6 * diam, k
        # the kernel's triangle is at the same distance (ties may pick another)
        _, d2k, _, _ = oracle.closest_point(V[F[tri[k]]], np.array([[0, 1, 2]], np.int32), p.astype(np.float64), 10.0)
        assert abs(np.sqrt(d2k) - np.sqrt(d2)) <= 1e-6 * diam
    bvh.free()


@pytest.mark.parametrize("collapse", ["sah", "area"])
def test_point_distance_unbounded_radius_deep_tree(collapse):
    """A radius as large as the mesh (the Chamfer and Hausdorff measurements)
    keeps every box in range while the first descent runs: the stack must hold
    7 entries per level of a deep tree without overflowing.  The ~1M-face
    surface of the QEM workload; a sample of the distances against the
    oracle."""
    import paper_2605_26137_b300 as pb
    V, F = synth.sdf_mesh_target(synth.sdf_union_params(1, 32), 1_000_000)
    diam = float(np.linalg.norm(V.max(0) - V.min(0)))
    rng = np.random.default_rng(8)
    pts = np.concatenate([V[rng.integers(0, len(V), 20000)] + rng.normal(scale=0.01, size=(20000, 3)),
                          rng.uniform(-2.0, 2.0, size=(4000, 3))]).astype(np.float32)
    bvh = pb.Bvh(_t(V), _t(F), collapse=collapse)
    assert bvh.info()["max_depth"] >= 9
    d = pb.point_distance(bvh, _t(pts), diam)
    pb.sync_status()    # raises on a stack overflow
    d = d.cpu().numpy().astype(np.float64)
    ob = oracle.Bvh(V, F)
    for k in rng.choice(len(pts), 300, replace=False):
        t, d2, _, _ = oracle.closest_point(V, F, pts[k].astype(np.float64), diam, bvh=ob)
        assert t >= 0 and abs(d[k] - np.sqrt(d2)) <= 1e-6 * diam, k
    bvh.free()
