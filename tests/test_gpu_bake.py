"""GPU parity: the CUDA bake against the FP64 oracle on the same seeded inputs,
through the C ABI (libagbake.so)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_26137_b300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


def _t(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dtype)


def gpu_bake(asset, layout="q8", **kw):
    import paper_2605_26137_b300 as pb
    hv, hf = _t(asset.high_v), _t(asset.high_f)
    bvh = pb.Bvh(hv, hf, layout=layout)
    lv, lf, uv = _t(asset.low_v), _t(asset.low_f), _t(asset.low_uv)
    out = pb.bake(bvh, lv, lf, uv, asset.W, asset.H, asset.max_dist, gutter=asset.gutter, aux=True, **kw)
    pb.sync_status()
    return bvh, parity.to_numpy(out), out


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("layout", ["q8", "f32"])
def test_tiny_bake_matches_oracle(seed, layout):
    a = synth.tiny_asset(seed)
    o = oracle.bake_asset(a, use_bvh=False)  # brute-force oracle
    _, g, _ = gpu_bake(a, layout)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a)
    print(st)
    parity.check(st)
    assert st["n_ray"] == 4000


@pytest.mark.parametrize("W,H,seed", [(100, 77, 3), (129, 64, 4), (64, 200, 5)])
def test_jittered_atlas_ragged_sizes(W, H, seed):
    """Off-lattice UVs (conservative coverage), degenerate UV faces, image
    sizes that are not multiples of the raster or dilation tiles."""
    lv, lf = synth.icosphere(2)
    hv, hf = synth.sh_displaced_sphere(4, seed)
    uv = synth.jittered_atlas(len(lf), W, H, seed)
    a = synth.Asset(hv, hf, lv, lf, uv, W, H, 0.15, 2)
    o = oracle.bake_asset(a)
    _, g, _ = gpu_bake(a)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a)
    print(st)
    parity.check(st)
    assert o["degen"].sum() > 0


def test_sdf_asset_matches_oracle():
    """A small asset of the pipeline-output shape: marching-grid union of
    primitives, ~120k high faces, ~6k low faces, 512x384 atlas."""
    a = synth.sdf_asset(7, 120_000, 6_000, 512, 384, n_prims=16)
    o = oracle.bake_asset(a)
    _, g, _ = gpu_bake(a)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a)
    print(st)
    parity.check(st)


@pytest.mark.parametrize("collapse,grid_levels", [("area", None), ("sah", None), ("sah", "1")])
def test_bvh_structure_invariants(collapse, grid_levels, monkeypatch):
    """grid_levels "1": every collapse level after the first runs on the
    one-CTA path that otherwise only trees deeper than 16 levels reach."""
    import struct
    if grid_levels is not None:
        monkeypatch.setenv("AG_TEST_GRID_LEVELS", grid_levels)
    a = synth.sdf_asset(3, 60_000, 2_000, 256, 256, n_prims=12)
    hv, hf = _t(a.high_v), _t(a.high_f)
    import paper_2605_26137_b300 as pb
    for layout in ("q8", "f32"):
        bvh = pb.Bvh(hv, hf, layout=layout, collapse=collapse)
        info = bvh.info()
        nodes, tris, ids, vn = bvh.copy_out()
        n = len(a.high_f)
        # every triangle exactly once, records carry its vertices
        assert np.array_equal(np.sort(ids), np.arange(n))
        vid = tris[..., 3].view(np.int32)
        assert np.array_equal(vid, a.high_f[ids])
        assert np.array_equal(tris[..., :3], a.high_v[a.high_f[ids]])
        # exact FP32 box of every record range vs the node's child boxes
        ns = info["node_size"]
        raw = nodes.reshape(-1, ns)
        seen = np.zeros(n, np.int32)
        reach = np.zeros(len(raw), np.int32)
        reach[0] = 1

        def child_boxes(r):
            if layout == "q8":
                o = np.frombuffer(r[:12].tobytes(), np.float32).astype(np.float32)
                e = r[12:15].astype(np.int64)
                s = (np.uint32(1) * (e.astype(np.uint32) << 23)).view(np.float32)
                q = r[32:80].reshape(6, 8).astype(np.float32)
                lo = np.stack([np.float32(q[a_] * s[a_]) + o[a_] for a_ in range(3)], 1)
                hi = np.stack([np.float32(q[3 + a_] * s[a_]) + o[a_] for a_ in range(3)], 1)
                meta = r[24:32]
                cb, tb = struct.unpack("<II", r[16:24].tobytes())
            else:
                cb, tb = struct.unpack("<II", r[:8].tobytes())
                meta = r[8:16]
                f = np.frombuffer(r[16:208].tobytes(), np.float32).reshape(6, 8)
                lo, hi = f[:3].T, f[3:].T
            return cb, tb, meta, lo, hi

        for i, r in enumerate(raw):
            cb, tb, meta, lo, hi = child_boxes(r)
            for c in range(8):
                m = int(meta[c])
                if m == 0:
                    continue
                if m & 0x80:
                    k = cb + (m & 0x7F)
                    reach[k] += 1
                    _, _, cm, clo, chi = child_boxes(raw[k])
                    valid = cm != 0
                    # the child node's own children lie inside this child box
                    assert np.all(clo[valid] >= lo[c] - 0) or layout == "q8"
                else:
                    cnt, off = (m >> 5) & 3, m & 31
                    recs = np.arange(tb + off, tb + off + cnt)
                    seen[recs] += 1
                    v = tris[recs, :, :3].reshape(-1, 3)
                    assert np.all(v >= lo[c]) and np.all(v <= hi[c]), "child box does not contain its triangles"
        assert np.all(seen == 1), "record not referenced exactly once"
        assert np.all(reach == 1), "node not referenced exactly once"
        # smooth normals are unit and area weighted
        on = oracle.vertex_normals(a.high_v, a.high_f)
        assert np.abs(vn[:, :3] - on).max() < 1e-6
        bvh.free()


def test_batch_and_graph_equal_single_bakes():
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
    outs = pb.bake_batch(batch_in)
    plan = pb.BatchPlan(plan_in)
    plan.launch()
    plan.launch()
    pb.sync_status()
    for g, ob, op in zip(singles, outs, [x.out for x in plan_in]):
        for out in (ob, op):
            assert np.array_equal(out.normal_rgba8.cpu().numpy(), g["normal_rgba8"])
            assert np.array_equal(out.mask.cpu().numpy(), g["mask"])
            assert np.array_equal(out.disp.cpu().numpy().view(np.uint16), g["disp"].view(np.uint16))
    plan.free()



@pytest.mark.parametrize("query,layout", [("ray", "q8"), ("closest", "q8"), ("ray", "f32"), ("closest", "f32")])
def test_batch_warps_spanning_small_and_empty_assets(query, layout):
    """A batch whose ray lists are shorter than a warp (one or two faces left
    on the atlas) or empty, between ordinary assets: the batched traversal's
    warps span several assets and skip empty ones.  Every asset's maps equal
    its single bake byte for byte, for both node layouts."""
    import paper_2605_26137_b300 as pb
    base = [synth.tiny_asset(s, W=96 + 32 * s, H=128) for s in range(3)]

    def few(a, keep):   # all faces but the first `keep` moved off the atlas
        uv = (a.low_uv * 0.4 + 1.5).astype(np.float32)
        uv[:keep] = a.low_uv[:keep]
        return uv

    specs = [(base[0], base[0].low_uv), (base[1], few(base[1], 1)), (base[1], few(base[1], 0)),
             (base[2], few(base[2], 2)), (base[0], few(base[0], 1)), (base[2], base[2].low_uv)]
    handles, singles, assets = [], [], []
    for a, uv in specs:
        bvh = pb.Bvh(_t(a.high_v), _t(a.high_f), layout=layout)
        handles.append(bvh)
        lv, lf, tuv = _t(a.low_v), _t(a.low_f), _t(uv)
        o = pb.bake(bvh, lv, lf, tuv, a.W, a.H, a.max_dist, query=query, aux=True)
        pb.sync_status()
        singles.append((o.normal_rgba8.cpu().numpy(), o.mask.cpu().numpy(), o.disp.cpu().numpy().view(np.uint16),
                        int(o.n_rays.item())))
        assets.append(pb.Asset(bvh, lv, lf, tuv, a.W, a.H, a.max_dist))
    n_rays = [x[3] for x in singles]
    assert n_rays[2] == 0 and 0 < n_rays[1] < 32 and 0 < n_rays[4] < 32 and n_rays[0] > 1000, n_rays
    outs = pb.bake_batch(assets, query=query)
    pb.sync_status()
    for (rgba, mask, disp, _), out in zip(singles, outs):
        assert np.array_equal(out.normal_rgba8.cpu().numpy(), rgba)
        assert np.array_equal(out.mask.cpu().numpy(), mask)
        assert np.array_equal(out.disp.cpu().numpy().view(np.uint16), disp)
    for h in handles:
        h.free()

def test_step_cap_sets_status_and_clears():
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(0)
    hv, hf = _t(a.high_v), _t(a.high_f)
    bvh = pb.Bvh(hv, hf)
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, max_steps=1)
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 4
    pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist)
    pb.sync_status()  # cleared, and a normal bake sets nothing


@pytest.mark.parametrize("schedule", ["batch", "refill", "coop2", "coop8"])
def test_stack_overflow_sets_status_and_clears(schedule):
    """A traversal stack capped at one entry (the counting build's test hook)
    must overflow on the tiny asset; the overflow is reported as
    AG_ERR_TRAVERSAL_LIMIT, and the next bake (full stack) is clean and
    equal to a bake that never overflowed."""
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(0)
    bvh = pb.Bvh(_t(a.high_v), _t(a.high_f))
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    md = 0.6   # a long ray crosses many boxes, so a one-entry stack cannot hold them
    clean = pb.bake(bvh, lv, lf, uv, a.W, a.H, md, schedule=schedule)
    pb.sync_status()
    ref = clean.normal_rgba8.cpu().numpy()
    pb.bake(bvh, lv, lf, uv, a.W, a.H, md, schedule=schedule, counters=True, aux=True, stack_limit=1)
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 4
    again = pb.bake(bvh, lv, lf, uv, a.W, a.H, md, schedule=schedule, counters=True, aux=True)
    pb.sync_status()
    assert np.array_equal(again.normal_rgba8.cpu().numpy(), ref)


def test_device_argument_errors():
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(0)
    hv, hf = _t(a.high_v), _t(a.high_f)
    bad = hf.clone()
    bad[5, 1] = len(a.high_v) + 3
    with pytest.raises(pb.AgError) as ei:
        pb.Bvh(hv, bad)
    assert ei.value.status == 1
    # an asynchronous build returns before the check: the bad index reaches
    # the status word, and the handle stays safe to use and free
    pb.sync_status()
    abvh = pb.Bvh(hv, bad, async_build=True)
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 1
    assert abvh.info()["n_tris"] == len(a.high_f)
    abvh.free()
    pb.sync_status()
    bvh = pb.Bvh(hv, hf)
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    with pytest.raises(pb.AgError):
        pb.bake(bvh, lv, lf, uv, 0, a.H, a.max_dist)
    with pytest.raises(pb.AgError):
        pb.bake(bvh, lv, lf, uv, a.W, a.H, -1.0)
    uv_bad = uv.clone()
    uv_bad[3, 1, 0] = float("nan")
    pb.bake(bvh, lv, lf, uv_bad, a.W, a.H, a.max_dist)
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 1
    pb.sync_status()


@pytest.mark.parametrize("rotate", [False, True])
def test_backward_matches_oracle_gradient_and_fd(rotate):
    """The 320-face icosphere over the displaced 5,120-face icosphere.  Their
    edges line up radially, so ~8% of the rays hit a high-poly edge where the
    piecewise-smooth gradient has a kink and either side is correct; with the
    high mesh rotated off that alignment the agreement is much tighter."""
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(0)
    tol = 1e-3
    if rotate:
        rng = np.random.default_rng(11)
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        a.high_v = (a.high_v.astype(np.float64) @ q.T).astype(np.float32)
        tol = 1e-4
    o = oracle.bake_asset(a)
    lam = 0.1
    lv64 = a.low_v.astype(np.float64)
    L_o, g_o = oracle.loss_grad(a.high_v, a.high_f, o["high_normals"], lv64, a.low_f, o["face"], o["bary"],
                                o["hit_tri"], lam)
    fd = oracle.fd_grad(a.high_v, a.high_f, o["high_normals"], lv64, a.low_f, o["face"], o["bary"], o["hit_tri"],
                        lam, h=1e-4)
    bvh = pb.Bvh(_t(a.high_v), _t(a.high_f))
    lv = _t(a.low_v)
    loss, grad = pb.bake_backward(bvh, lv, _t(a.low_f), _t(a.low_uv), a.W, a.H, a.max_dist, lam)
    pb.sync_status()
    L_g = float(loss.item())
    g_g = grad.cpu().numpy().astype(np.float64)
    assert abs(L_g - L_o) <= 1e-4 * abs(L_o)
    rel_o = np.linalg.norm(g_g - g_o) / np.linalg.norm(g_o)
    rel_fd = np.linalg.norm(g_g - fd) / np.linalg.norm(fd)
    print("loss", L_g, L_o, "rel vs analytic", rel_o, "rel vs fd", rel_fd)
    assert rel_fd <= tol
    assert rel_o <= tol
    # autograd wrapper gives the same gradient
    x = lv.clone().requires_grad_(True)
    L = pb.bake_loss(bvh, x, _t(a.low_f), _t(a.low_uv), a.W, a.H, a.max_dist, lam)
    L.backward()
    assert (x.grad - grad).norm() <= 1e-4 * grad.norm()


@pytest.mark.slow
def test_full_size_asset_sampled_parity():
    """The benchmark workload at full size (~2M high-poly triangles, 2048^2
    atlas, bench launch configuration): the whole raster map bit-exact, a
    seeded sample of ray texels against the oracle, and properties that hold
    at any size on every texel (unit normals, alpha/filled, dilation = the
    renormalised mean of the filled neighbours)."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(1, 2_000_000, 30_000, 2048, 2048, n_prims=32)
    bvh, g, out = gpu_bake(a)
    face, bary, _ = oracle.raster(a.low_uv, a.W, a.H)
    assert np.array_equal(g["face"], face)
    assert np.abs(g["bary"][face >= 0] - bary[face >= 0]).max() < 2e-6
    rays = np.flatnonzero(face.reshape(-1) >= 0)
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(rays, size=3000, replace=False))
    o = oracle.bake_asset(a, sample=sample)
    st = parity.compare(g, o, a.diam, a.gutter, sample=sample, asset=a)
    print(st)
    parity.check(st, small=0)
    # properties on every texel
    n = g["normal_ts"]
    filled = g["normal_rgba8"][..., 3] == 255
    assert np.abs(np.linalg.norm(n[filled], axis=-1) - 1).max() < 1e-5
    ray = face >= 0
    assert np.array_equal(filled[ray], np.ones(ray.sum(), bool))
    # one dilation pass reproduced from the GPU's own ray texels (first ring)
    H, W = face.shape
    ring = np.zeros_like(ray)
    ring[1:-1, 1:-1] = ~ray[1:-1, 1:-1] & (
        ray[:-2, :-2] | ray[:-2, 1:-1] | ray[:-2, 2:] | ray[1:-1, :-2] | ray[1:-1, 2:] | ray[2:, :-2] | ray[2:, 1:-1] | ray[2:, 2:])
    ys, xs = np.nonzero(ring)
    pick = rng.choice(len(ys), size=min(2000, len(ys)), replace=False)
    for y, x in zip(ys[pick], xs[pick]):
        acc, cnt = np.zeros(3), 0
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dy or dx) and ray[y + dy, x + dx]:
                    acc += n[y + dy, x + dx]
                    cnt += 1
        m = acc / cnt
        assert np.abs(n[y, x] - m / np.linalg.norm(m)).max() < 1e-5
    bvh.free()


def test_large_asset_sampled_parity_both_layouts():
    """The 8M-triangle, 4096^2 precision-study workload: the whole raster map
    bit-exact, and a seeded sample of ray texels against the oracle for the
    8-bit and the FP32 node layouts."""
    a = synth.sdf_asset(1, 8_000_000, 30_000, 4096, 4096, n_prims=32)
    face, _, _ = oracle.raster(a.low_uv, a.W, a.H)
    rays = np.flatnonzero(face.reshape(-1) >= 0)
    sample = np.sort(np.random.default_rng(2).choice(rays, size=1500, replace=False))
    o = oracle.bake_asset(a, sample=sample)
    for layout in ("q8", "f32"):
        bvh, g, _ = gpu_bake(a, layout=layout)
        assert np.array_equal(g["face"], face)
        st = parity.compare(g, o, a.diam, a.gutter, sample=sample, asset=a)
        print(layout, len(a.high_f), st)
        parity.check(st, small=0)
        bvh.free()


def test_launch_configurations_give_identical_bakes_and_autotune(tmp_path, monkeypatch):
    """Schedules, block sizes and ray tiles change only the speed: every
    configuration produces the same bytes; the autotuner picks one of them
    and caches it."""
    import paper_2605_26137_b300 as pb
    from paper_2605_26137_b300 import autotune
    a = synth.sdf_asset(5, 40_000, 2_000, 256, 192, n_prims=10)
    bvh = pb.Bvh(_t(a.high_v), _t(a.high_f))
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    ref = None
    for sched in ("batch", "refill", "coop2", "coop4", "coop8"):
        for tile in ("8x8", "16x16", "32x8", "4x4"):
            for block in (64, 256):
                o = pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, schedule=sched, ray_tile=tile, block_size=block,
                            aux=True)
                pb.sync_status()
                got = (o.normal_rgba8.cpu().numpy(), o.mask.cpu().numpy(), o.disp.cpu().numpy().view(np.uint16),
                       o.hit_tri.cpu().numpy(), o.normal_ts.cpu().numpy().view(np.uint32))
                if ref is None:
                    ref = got
                for x, y in zip(got, ref):
                    assert np.array_equal(x, y), (sched, tile, block)
    monkeypatch.setenv("AGBAKE_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    e = autotune.tune(bvh, lv, lf, uv, a.W, a.H, a.max_dist)
    assert not e["cached"] and e["ms"] > 0
    assert e["schedule"] in (0, 1, 2, 3, 4) and e["block_size"] in (0, 64, 128, 256) and e["ray_tile"] in (0, 1, 2, 3)
    e2 = autotune.tune(bvh, lv, lf, uv, a.W, a.H, a.max_dist)
    assert e2["cached"] and e2["schedule"] == e["schedule"]
    o = pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, **autotune.launch_kwargs(e))
    assert np.array_equal(o.normal_rgba8.cpu().numpy(), ref[0])


def test_empty_and_degenerate_atlases():
    """No covered texel: UVs outside the atlas, or every face with zero UV
    area.  The bake still writes every output (neutral normal, alpha 0)."""
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(0)
    bvh = pb.Bvh(_t(a.high_v), _t(a.high_f))
    lv, lf = _t(a.low_v), _t(a.low_f)
    outside = (a.low_uv * 0.4 + 1.5).astype(np.float32)            # in [1.5, 1.9]: valid, off the atlas
    flat = np.repeat(a.low_uv[:, :1, :], 3, axis=1).copy()          # zero UV area everywhere
    for uv in (outside, flat):
        o = pb.bake(bvh, lv, lf, _t(uv), a.W, a.H, a.max_dist, aux=True)
        pb.sync_status()
        rgba = o.normal_rgba8.cpu().numpy()
        assert (rgba == np.array([128, 128, 255, 0], np.uint8)).all()
        assert not o.mask.cpu().numpy().any() and not o.disp.cpu().numpy().any()
        assert int(o.n_rays.item()) == 0 and (o.face.cpu().numpy() == -1).all()


@pytest.mark.parametrize("W,H", [(16384, 64), (64, 16384)])
def test_maximum_atlas_width_and_height(W, H):
    """The largest atlas dimension the ABI accepts, on a thin atlas."""
    lv, lf = synth.icosphere(2)
    hv, hf = synth.sh_displaced_sphere(4, 9)
    uv = synth.grid_atlas(len(lf), W, H, gutter=1)
    a = synth.Asset(hv, hf, lv, lf, uv, W, H, 0.15, 2)
    o = oracle.bake_asset(a)
    _, g, _ = gpu_bake(a)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a)
    print(st)
    parity.check(st)
    assert st["n_ray"] > 10_000


@pytest.mark.parametrize("n_high", [1, 2, 3, 4, 9])
def test_tiny_high_meshes(n_high):
    """BVHs of one to a few triangles (a root that is itself a leaf)."""
    lv = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    lf = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    rng = np.random.default_rng(n_high)
    hv = (rng.uniform(-1.2, 1.2, size=(3 * n_high, 3)) * [1, 1, 0.05]).astype(np.float32)
    hf = np.arange(3 * n_high, dtype=np.int32).reshape(-1, 3)
    uv = synth.grid_atlas(2, 32, 32, 2)
    a = synth.Asset(hv, hf, lv, lf, uv, 32, 32, 0.5, 2)
    o = oracle.bake_asset(a, use_bvh=False)
    _, g, _ = gpu_bake(a)
    st = parity.compare(g, o, a.diam, a.gutter, asset=a)
    parity.check(st)


def test_stream_pipeline_with_stream_ordered_free():
    """Two bakes in flight on two streams, each handle freed in its stream's
    order (ag_bvh_free_async): the maps equal a plain synchronous bake."""
    import paper_2605_26137_b300 as pb
    a = synth.tiny_asset(2)
    _, ref, _ = gpu_bake(a)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i in range(4):
        st = streams[i % 2]
        with torch.cuda.stream(st):
            bvh = pb.Bvh(_t(a.high_v), _t(a.high_f))
            out = pb.bake(bvh, _t(a.low_v), _t(a.low_f), _t(a.low_uv), a.W, a.H, a.max_dist, gutter=a.gutter)
            host = torch.empty_like(out.normal_rgba8, device="cpu").pin_memory()
            host.copy_(out.normal_rgba8, non_blocking=True)
            bvh.free(stream=st)
            outs.append((host, out))
    for st in streams:
        st.synchronize()
    pb.sync_status()
    for host, _ in outs:
        assert np.array_equal(host.numpy(), ref["normal_rgba8"])


@pytest.mark.parametrize("collapse", ["area_count", "count", "sah"])
def test_collapse_rules_give_identical_bakes(collapse):
    """Every collapse rule builds a different tree over the same triangles; the
    closest hit does not depend on the tree, so the maps are byte-identical."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(5, 120_000, 6_000, 512, 384, n_prims=16)
    hv, hf = _t(a.high_v), _t(a.high_f)
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    outs = []
    for rule in ("area", collapse):
        bvh = pb.Bvh(hv, hf, collapse=rule)
        o = pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, aux=True)
        pb.sync_status()
        outs.append(parity.to_numpy(o))
        bvh.free()
    for k in ("normal_rgba8", "mask", "disp", "hit_tri"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def _wide_tree_cost(nodes, node_size):
    """Surface-area cost of an FP32-layout wide tree, the root excluded: every
    wide child costs its box's half area, every leaf 0.3 x half area x count."""
    import struct
    raw = nodes.reshape(-1, node_size)
    total = 0.0
    for r in raw:
        meta = r[8:16]
        f = np.frombuffer(r[16:208].tobytes(), np.float32).reshape(6, 8).astype(np.float64)
        d = f[3:] - f[:3]
        ha = d[0] * d[1] + d[1] * d[2] + d[2] * d[0]
        for c in range(8):
            m = int(meta[c])
            if m == 0:
                continue
            total += ha[c] if m & 0x80 else 0.3 * ha[c] * ((m >> 5) & 3)
    return total


def test_sah_collapse_costs_no_more_than_greedy_rules():
    """The SAH collapse minimises the surface-area cost over every way of
    cutting the same binary tree into 8-wide nodes, and each greedy rule makes
    one such cut: its tree costs at least as much (to float rounding)."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(6, 40_000, 2_000, 256, 256, n_prims=10)
    hv, hf = _t(a.high_v), _t(a.high_f)
    cost = {}
    for rule in ("sah", "area", "area_count", "count"):
        bvh = pb.Bvh(hv, hf, layout="f32", collapse=rule)
        nodes, _, _, _ = bvh.copy_out()
        cost[rule] = _wide_tree_cost(nodes, bvh.info()["node_size"])
        bvh.free()
    print(cost)
    for rule in ("area", "area_count", "count"):
        assert cost["sah"] <= cost[rule] * (1 + 1e-5), rule


def test_async_build_on_another_stream():
    """A handle built asynchronously on one stream and baked on another with
    no ordering by the caller: the bake orders its traversal after the build
    (its raster and frames may run beside it) and gives the maps of a bake
    on the build's own stream."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(6, 200_000, 6_000, 512, 512, n_prims=16)
    hv, hf = _t(a.high_v), _t(a.high_f)
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)
    ref_bvh = pb.Bvh(hv, hf)
    ref = parity.to_numpy(pb.bake(ref_bvh, lv, lf, uv, a.W, a.H, a.max_dist, aux=True))
    ref_bvh.free()
    torch.cuda.synchronize()
    sb, sk = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(sb):
        bvh = pb.Bvh(hv, hf, async_build=True, stream=sb)
    with torch.cuda.stream(sk):
        o = pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, aux=True, stream=sk)
    sk.synchronize()
    sb.synchronize()
    pb.sync_status()
    out = parity.to_numpy(o)
    for k in ("normal_rgba8", "mask", "disp", "hit_tri"):
        assert np.array_equal(out[k], ref[k]), k
    bvh.free()


@pytest.mark.parametrize("layout", ["q8", "f32"])
def test_async_build_and_one_cta_collapse_give_identical_bakes(layout, monkeypatch):
    """A build that returns without a host round trip (the bake is enqueued
    before anything waits for the build), and builds whose collapse hands every
    level after the second to the one-CTA path, give the default build's tree
    summary and byte-identical maps."""
    import paper_2605_26137_b300 as pb
    a = synth.sdf_asset(5, 120_000, 6_000, 512, 384, n_prims=16)
    hv, hf = _t(a.high_v), _t(a.high_f)
    lv, lf, uv = _t(a.low_v), _t(a.low_f), _t(a.low_uv)

    def run(**kw):
        bvh = pb.Bvh(hv, hf, layout=layout, **kw)
        o = pb.bake(bvh, lv, lf, uv, a.W, a.H, a.max_dist, aux=True)
        pb.sync_status()
        out = parity.to_numpy(o)
        inf = bvh.info()
        bvh.free()
        return out, inf

    ref, ri = run()
    cases = [run(async_build=True)]
    monkeypatch.setenv("AG_TEST_GRID_LEVELS", "2")
    cases += [run(), run(async_build=True)]
    for out, inf in cases:
        for k in ("normal_rgba8", "mask", "disp", "hit_tri"):
            assert np.array_equal(out[k], ref[k]), k
        for k in ("n_nodes", "max_depth", "scene_lo", "scene_hi", "diam", "n_tris"):
            assert inf[k] == ri[k], k
        assert inf["build_ms"] > 0
