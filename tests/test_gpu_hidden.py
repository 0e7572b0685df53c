"""GPU parity of hidden-face removal (Sec. 6.2) against the FP64 oracle,
through the C ABI (ag_visibility, ag_exterior_fill).

Per ray, the kernel's first-hit face must equal the oracle's where the oracle
finds exactly one face within 1e-5 R of the ray and the hit point lies farther
than that from the face's boundary; elsewhere it must be one of the oracle's
candidate faces (or a miss).  The per-face mask must be the union of the
kernel's own hits and lie between the oracle's certain and candidate sets.
The flood fill is integer graph work with the gate decided in FP64 in the same
order on both sides: bit-exact.  Both renders are checked: z-buffer proposals
confirmed by the ray test (the default) and every ray traced."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_26137_b300 import synth

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_vis(V, F, n_views, res, layout="q8", render="raster", **kw):
    """Visibility through the kernel; the counting build (tracing every ray)
    with render="trace"."""
    import paper_2605_26137_b300 as pb
    bvh = pb.Bvh(_t(V), _t(F), layout=layout)
    trace = render == "trace"
    vis, hits, cnt = pb.visibility(bvh, n_views, res, hit_ids=True, counters=trace, render=render, **kw)
    pb.sync_status()
    out = vis.cpu().numpy(), hits.cpu().numpy(), cnt.cpu().numpy() if trace else None
    bvh.free()
    return out


def check_rays(g, o):
    """Per-ray agreement; returns the fraction of rays that were certain."""
    g = g.reshape(-1)
    h, nc = o["hit"].reshape(-1), o["ncand"].reshape(-1)
    cand, near = o["cand"].reshape(-1, oracle.MAX_CAND), o["edge_near"].reshape(-1)
    certain = (nc <= 1) & (near == 0)
    bad = certain & (g != h)
    assert not bad.any(), f"{bad.sum()} certain rays differ, e.g. ray {np.flatnonzero(bad)[:5]}"
    unc = ~certain & (nc <= oracle.MAX_CAND)
    ok = (g[unc] == -1) | (cand[unc] == g[unc][:, None]).any(1)
    assert ok.all(), f"{(~ok).sum()} uncertain rays outside their candidate sets"
    return float(certain.mean())


def mask_bounds(o, nf):
    h, nc = o["hit"].reshape(-1), o["ncand"].reshape(-1)
    cand, near = o["cand"].reshape(-1, oracle.MAX_CAND), o["edge_near"].reshape(-1)
    certain = (nc <= 1) & (near == 0)
    strict = np.zeros(nf, bool)
    strict[h[certain & (h >= 0)]] = True
    loose = np.zeros(nf, bool)
    loose[h[h >= 0]] = True
    c = cand[~certain]
    loose[c[c >= 0]] = True
    return strict, loose


def _meshes():
    Vs, Fs = synth.sh_displaced_sphere(3, 4, amp=0.1)
    Vo, Fo = synth.icosphere(3, 1.0)
    Vi, Fi = synth.icosphere(2, 0.5)
    nested = (np.concatenate([Vo, Vi]), np.concatenate([Fo, Fi + len(Vo)]).astype(np.int32))
    Vh, Fh, _ = synth.hidden_face_mesh(2, target_faces=22000, device="cpu")
    return {"sphere": (Vs, Fs), "nested": nested, "generated": (Vh, Fh)}


MESHES = _meshes()


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("layout", ["q8", "f32"])
@pytest.mark.parametrize("n_views,res", [(16, 64), (7, 37)])
@pytest.mark.parametrize("render", ["raster", "trace"])
def test_visibility_matches_oracle(name, layout, n_views, res, render):
    V, F = MESHES[name]
    o = oracle.visibility(V, F, n_views, res)
    vis, hits, cnt = gpu_vis(V, F, n_views, res, layout, render)
    frac = check_rays(hits, o)
    assert frac > 0.98
    # the mask is the union of the kernel's own hits, between the oracle's bounds
    own = np.zeros(len(F), np.uint8)
    own[hits[hits >= 0]] = 1
    assert np.array_equal(vis, own)
    strict, loose = mask_bounds(o, len(F))
    assert np.all(vis[strict] == 1) and not np.any(vis[~loose])
    if cnt is not None:
        assert cnt[0] == n_views * res * res and cnt[3] == (hits >= 0).sum()


def test_exterior_fill_bit_exact_and_generated_mesh_cleanup():
    import paper_2605_26137_b300 as pb
    V, F, inner = synth.hidden_face_mesh(7, target_faces=22000, device="cpu")
    assert inner.sum() == 8 * 320
    vis, _, _ = gpu_vis(V, F, 24, 96)
    ext = pb.exterior_fill(_t(V), _t(F), _t(vis))
    pb.sync_status()
    ext = ext.cpu().numpy()
    assert np.array_equal(ext, oracle.exterior_fill(V, F, vis))
    # the oracle's own mask through the kernel as well
    ov = oracle.visibility(V, F, 24, 96, candidates=False)["visible"]
    assert np.array_equal(pb.exterior_fill(_t(V), _t(F), _t(ov)).cpu().numpy(), oracle.exterior_fill(V, F, ov))
    # interior shells removed, the outer surface kept (a marching-grid face folded
    # against all its neighbours and seen by no ray is, by the method, removed)
    assert not ext[inner].any() and ext[~inner].mean() > 0.999
    assert not vis[inner].any()
    # random masks and flipped faces: still bit-exact
    rng = np.random.default_rng(0)
    G = F.copy()
    flip = rng.random(len(G)) < 0.2
    G[flip] = G[flip][:, ::-1]
    for p in (0.001, 0.05, 0.5):
        m = (rng.random(len(G)) < p).astype(np.uint8)
        got = pb.exterior_fill(_t(V), _t(G), _t(m)).cpu().numpy()
        assert np.array_equal(got, oracle.exterior_fill(V, G, m)), p


def test_hidden_faces_one_call_and_argument_errors():
    import paper_2605_26137_b300 as pb
    V, F, inner = synth.hidden_face_mesh(1, target_faces=22000, device="cpu")
    assert inner.sum() > 0
    ext, vis = pb.hidden_faces(_t(V), _t(F), n_views=32, res=64)
    pb.sync_status()
    ext = ext.cpu().numpy()
    assert not ext[inner].any() and ext[~inner].mean() > 0.999
    bvh = pb.Bvh(_t(V), _t(F))
    for nv, res in ((0, 64), (4, 0), (4, 16385)):
        with pytest.raises(pb.AgError) as ei:
            pb.visibility(bvh, nv, res)
        assert ei.value.status == 1
    # one view of one pixel: the centre ray
    v1, h1, _ = pb.visibility(bvh, 1, 1, hit_ids=True)
    pb.sync_status()
    o1 = oracle.visibility(V, F, 1, 1)
    check_rays(h1.cpu().numpy(), o1)
    # step cap (of the traversal: every ray traced)
    pb.visibility(bvh, 2, 16, max_steps=1, render="trace")
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 4
    bvh.free()
    # an out-of-range face index: never exterior, reported by the status word
    Fb = F.copy()
    Fb[7, 2] = len(V) + 5
    m = np.ones(len(F), np.uint8)
    got = pb.exterior_fill(_t(V), _t(Fb), _t(m))
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 1
    assert got.cpu().numpy()[7] == 0


@pytest.mark.slow
def test_full_size_sampled():
    """The paper's configuration: 512 views x 1024^2 rays on a ~22k-face mesh
    with interior shells; 20k sampled rays against the oracle, the mask equal
    to the union of all 537M hits, interior shells removed."""
    import paper_2605_26137_b300 as pb
    V, F, inner = synth.hidden_face_mesh(0, target_faces=22000, device="cpu")
    n_views, res = 512, 1024
    vis, hits, _ = gpu_vis(V, F, n_views, res)
    own = np.zeros(len(F), np.uint8)
    flat = hits.reshape(-1)
    own[np.unique(flat[flat >= 0])] = 1
    assert np.array_equal(vis, own)
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(flat.size, 20000, replace=False))
    o = oracle.visibility(V, F, n_views, res, sample=sample)
    assert check_rays(flat[sample], o) > 0.98
    ext = pb.exterior_fill(_t(V), _t(F), _t(vis)).cpu().numpy()
    assert np.array_equal(ext, oracle.exterior_fill(V, F, vis))
    assert not vis[inner].any() and not ext[inner].any() and ext[~inner].mean() > 0.999
