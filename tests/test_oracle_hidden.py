"""Pins for the oracle's hidden-face removal (Sec. 6.2): the view lattice and
image geometry, per-face visibility and the normal-gated exterior flood fill.

* view basis: the closed form for one lattice point, orthonormal and
  right-handed frames, equally spaced heights;
* a square seen face-on: the exact set of pixels whose rays land on it;
* a convex mesh is entirely visible; a shell inside another is entirely
  hidden and not exterior; the BVH equals brute force ray by ray;
* candidate lists: rays through the middle of a face have exactly that face,
  rays through a shared edge have both faces;
* flood fill: hand-built strips and folds (coplanar links, a flipped face and
  a right-angle fold block, a 60-degree fold passes, a non-manifold edge
  links all its faces), and connected components computed by networkx on
  random meshes with flipped faces.
"""
import networkx as nx
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def test_view_basis_closed_form_and_frames():
    u, e1, e2 = oracle.view_basis(0, 2)
    assert np.allclose(u, [np.sqrt(0.75), 0, 0.5], atol=1e-15)
    assert np.allclose(e1, [0, 1, 0], atol=1e-15)
    assert np.allclose(e2, [-0.5, 0, np.sqrt(0.75)], atol=1e-15)
    n = 37
    zs = []
    for k in range(n):
        u, e1, e2 = oracle.view_basis(k, n)
        M = np.stack([e1, e2, u])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(M) == pytest.approx(1.0, abs=1e-14)
        zs.append(u[2])
    assert np.allclose(np.diff(zs), -2.0 / n, atol=1e-14)
    # successive lattice points turn by the golden angle about z
    u0, _, _ = oracle.view_basis(5, n)
    u1, _, _ = oracle.view_basis(6, n)
    dphi = (np.arctan2(u1[1], u1[0]) - np.arctan2(u0[1], u0[0])) % (2 * np.pi)
    assert dphi == pytest.approx(np.pi * (3 - np.sqrt(5)), abs=1e-12)


def _square_x0():
    # the square x = 0, |y|, |z| <= 1 (two triangles facing +x)
    V = np.array([[0, -1, -1], [0, 1, -1], [0, 1, 1], [0, -1, 1]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return V, F


@pytest.mark.parametrize("res", [8, 33, 64])
def test_square_face_on_hit_pattern(res):
    V, F = _square_x0()
    r = oracle.visibility(V, F, 1, res, use_bvh=False)   # one view: u = +x, e1 = +y, e2 = +z
    c, R = r["frame"]
    assert np.allclose(c, 0) and R == pytest.approx(np.sqrt(2))
    coord = (2 * (np.arange(res) + 0.5) / res - 1) * R
    inside = np.abs(coord) <= 1
    expect = inside[:, None] & inside[None, :]          # [j (e2), i (e1)]
    got = r["hit"][0] >= 0
    certain = r["ncand"][0] <= 1
    assert np.array_equal(got[certain], expect[certain])
    assert certain.sum() >= expect.size - 4 * res       # only the rim and the diagonal can be uncertain
    assert r["visible"].all()


def test_convex_mesh_fully_visible_and_bvh_equals_brute_force():
    V, F = synth.sh_displaced_sphere(3, 2, amp=0.02)
    a = oracle.visibility(V, F, 24, 48)
    b = oracle.visibility(V, F, 24, 48, use_bvh=False)
    assert np.array_equal(a["hit"], b["hit"])
    assert np.array_equal(a["ncand"], b["ncand"])
    assert np.array_equal(np.sort(a["cand"], -1), np.sort(b["cand"], -1))
    full = oracle.visibility(V, F, 64, 64, candidates=False)
    assert full["visible"].all()
    assert oracle.exterior_fill(V, F, full["visible"]).all()


def test_nested_shells():
    Vo, Fo = synth.icosphere(3, 1.0)
    Vi, Fi = synth.icosphere(2, 0.5)
    V = np.concatenate([Vo, Vi])
    F = np.concatenate([Fo, Fi + len(Vo)])
    r = oracle.visibility(V, F, 48, 48, candidates=False)
    assert r["visible"][:len(Fo)].all() and not r["visible"][len(Fo):].any()
    ext = oracle.exterior_fill(V, F, r["visible"])
    assert ext[:len(Fo)].all() and not ext[len(Fo):].any()


def test_candidates_face_interior_and_shared_edge():
    V, F = _square_x0()
    res = 64
    r = oracle.visibility(V, F, 1, res, use_bvh=False)
    R = r["frame"][1]
    coord = (2 * (np.arange(res) + 0.5) / res - 1) * R
    # a pixel well inside triangle 1 (z > y) and far from every edge
    j = int(np.argmin(np.abs(coord - 0.6)))
    i = int(np.argmin(np.abs(coord + 0.4)))
    assert r["hit"][0, j, i] == 1 and r["ncand"][0, j, i] == 1 and not r["edge_near"][0, j, i]
    # a pixel exactly on the shared diagonal y = z (odd resolution puts one there)
    r = oracle.visibility(V, F, 1, 33, use_bvh=False)
    mid = 16
    assert r["ncand"][0, mid, mid] == 2 and set(r["cand"][0, mid, mid, :2]) == {0, 1}
    assert r["edge_near"][0, mid, mid]


# ------------------------------------------------------------------ flood fill

def _normals(V, F):
    A, B, C = V[F[:, 0]].astype(np.float64), V[F[:, 1]].astype(np.float64), V[F[:, 2]].astype(np.float64)
    return np.cross(B - A, C - A)


def test_fill_coplanar_strip_and_flipped_face():
    # quads of two triangles along x, all facing +z
    V = np.array([[x, y, 0] for x in range(4) for y in (0, 1)], np.float32)
    idx = lambda x, y: 2 * x + y
    F = []
    for x in range(3):
        F += [(idx(x, 0), idx(x + 1, 0), idx(x + 1, 1)), (idx(x, 0), idx(x + 1, 1), idx(x, 1))]
    F = np.array(F, np.int32)
    assert (_normals(V, F)[:, 2] > 0).all()
    vis = np.zeros(len(F), np.uint8)
    vis[0] = 1
    assert oracle.exterior_fill(V, F, vis).all()
    # edge adjacency of this triangulation is the chain 1 - 0 - 3 - 2 - 5 - 4;
    # flipping face 3 cuts the chain there
    G = F.copy()
    G[3] = G[3][::-1]
    ext = oracle.exterior_fill(V, G, vis)
    assert ext.tolist() == [1, 1, 0, 0, 0, 0]
    # seeded beyond the flip instead: 2, 4 and 5
    vis2 = np.zeros(len(F), np.uint8)
    vis2[5] = 1
    assert oracle.exterior_fill(V, G, vis2).tolist() == [0, 0, 1, 0, 1, 1]


@pytest.mark.parametrize("angle,linked", [(60, True), (89, True), (90, False), (120, False)])
def test_fill_fold_angle(angle, linked):
    # two triangles sharing the edge (0,0,0)-(0,1,0), both facing +z when flat;
    # the second folded about that edge by `angle`, so n0 . n1 = cos(angle)
    # (at 90 degrees exactly perpendicular: n0 . n1 = 0, and the gate is strict)
    a = np.radians(angle)
    tip = [0.0, 0.0, 1.0] if angle == 90 else [np.cos(a), 0.0, np.sin(a)]
    V = np.array([[0, 0, 0], [0, 1, 0], [-1, 0, 0], tip], np.float32)
    F = np.array([[0, 1, 2], [1, 0, 3]], np.int32)
    n = _normals(V, F)
    assert (n[0] @ n[1] > 0) == linked
    ext = oracle.exterior_fill(V, F, np.array([1, 0], np.uint8))
    assert bool(ext[1]) == linked


def test_fill_non_manifold_edge_and_degenerate_face():
    # three triangles on the edge (0,1), all within 90 degrees of each other; a zero-area face
    V = np.array([[0, 0, 0], [1, 0, 0], [0.5, 1, 0], [0.5, 1, 0.3], [0.5, 1, -0.3], [2, 0, 0]], np.float32)
    F = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4], [0, 1, 5]], np.int32)
    vis = np.array([1, 0, 0, 0], np.uint8)
    assert oracle.exterior_fill(V, F, vis).tolist() == [1, 1, 1, 0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fill_matches_networkx_components(seed):
    rng = np.random.default_rng(seed)
    V, F = synth.sh_displaced_sphere(2, seed, amp=0.2)
    F = F.copy()
    flip = rng.random(len(F)) < 0.15
    F[flip] = F[flip][:, ::-1]
    vis = (rng.random(len(F)) < 0.05).astype(np.uint8)
    n = _normals(V, F)
    G = nx.Graph()
    G.add_nodes_from(range(len(F)))
    edges = {}
    for f, tri in enumerate(F):
        for k in range(3):
            e = tuple(sorted((int(tri[k]), int(tri[(k + 1) % 3]))))
            edges.setdefault(e, []).append(f)
    for fs in edges.values():
        for i in range(len(fs)):
            for j in range(i + 1, len(fs)):
                if n[fs[i]] @ n[fs[j]] > 0:
                    G.add_edge(fs[i], fs[j])
    expect = np.zeros(len(F), np.uint8)
    for comp in nx.connected_components(G):
        comp = list(comp)
        if vis[comp].any():
            expect[comp] = 1
    assert np.array_equal(oracle.exterior_fill(V, F, vis), expect)
    assert 0 < expect.sum() < len(F)
