"""Pins for the oracle's QEM simplification (Sec. 6.1).

* a face quadric evaluates to the squared distance to the face's plane
  (closed forms for axis-aligned and oblique planes; sums add);
* placement: three orthogonal planes through X make X the unconstrained
  optimum, and the paper's projection onto the edge follows in closed form;
  one or two planes are singular and fall back to the midpoint;
* a closed sphere simplifies to exactly the target, stays a closed
  consistently oriented manifold of genus 0 near the sphere;
* an open flat grid: every boundary vertex of the result is an original
  boundary vertex at its original position, every vertex stays in the plane;
* a tetrahedron does not collapse;
* one round's collapses touch no two adjacent vertices of the input;
* a simplified SDF surface stays within a small distance of the original.
"""
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def test_face_quadric_is_squared_plane_distance():
    rng = np.random.default_rng(0)
    P = np.array([[0, 0, 0.3], [1, 0, 0.3], [0, 1, 0.3]])
    q = oracle.qem_face_quadric(P)
    for v in rng.normal(size=(20, 3)):
        assert oracle.qem_eval(q, v) == pytest.approx((v[2] - 0.3) ** 2, rel=1e-12, abs=1e-15)
    # the plane x + y + z = 1, corners in either orientation
    P = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    for Pk in (P, P[::-1]):
        q = oracle.qem_face_quadric(Pk)
        for v in rng.normal(size=(20, 3)):
            assert oracle.qem_eval(q, v) == pytest.approx((v.sum() - 1) ** 2 / 3, rel=1e-12, abs=1e-15)
    # sums of quadrics are sums of squared distances
    q2 = oracle.qem_face_quadric(np.array([[0, 0, 0], [0, 1, 0], [0, 0, 1.0]]))   # the plane x = 0
    v = np.array([0.2, -0.4, 0.7])
    assert oracle.qem_eval(q + q2, v) == pytest.approx((v.sum() - 1) ** 2 / 3 + 0.04, rel=1e-12)
    # a zero-area face has no plane
    assert not oracle.qem_face_quadric(np.array([[0, 0, 0], [1, 1, 1], [2, 2, 2.0]])).any()


def _planes_through(X, normals):
    q = np.zeros(10)
    for n in normals:
        n = np.asarray(n, float)
        u = np.cross(n, [1, 0, 0] if abs(n[0]) < 0.9 else [0, 1, 0])
        w = np.cross(n, u)
        q += oracle.qem_face_quadric(np.array([X, X + u, X + w]))
    return q


def test_placement_closed_form_and_singular_fallback():
    X = np.array([0.3, -0.2, 0.5])
    q = _planes_through(X, [[1, 0, 0], [0, 1, 0], [0, 0, 1]])
    assert oracle.qem_eval(q, X) == pytest.approx(0.0, abs=1e-24)
    rng = np.random.default_rng(1)
    for _ in range(50):
        v0, v1 = rng.normal(size=3), rng.normal(size=3)
        t, sing = oracle.qem_place(q, v0, v1)
        e = v1 - v0
        expect = np.clip((X - v0) @ e / (e @ e), 0, 1)
        assert not sing and t == pytest.approx(expect, abs=1e-12)
    # an edge through X: the optimum itself
    t, _ = oracle.qem_place(q, X - [0.1, 0.2, 0.0], X + [0.3, 0.6, 0.0])
    assert t == pytest.approx(0.25, abs=1e-12)
    # one plane or two (a line of optima): singular, midpoint
    for normals in ([[0, 0, 1]], [[1, 0, 0], [0, 1, 1]]):
        t, sing = oracle.qem_place(_planes_through(X, normals), np.zeros(3), np.ones(3))
        assert sing and t == 0.5


def _edges(F):
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    u, c = np.unique(e, axis=0, return_counts=True)
    return u, c


def test_closed_sphere_simplification():
    V, F = synth.icosphere(4)
    r = oracle.qem_simplify(V, F, 500)
    Vo, Fo = r["V"], r["F"]
    assert len(Fo) == 500
    u, c = _edges(Fo)
    assert (c == 2).all()                                   # closed 2-manifold
    assert len(Vo) - len(u) + len(Fo) == 2                  # genus 0
    A, B, C = Vo[Fo[:, 0]], Vo[Fo[:, 1]], Vo[Fo[:, 2]]
    n = np.cross(B - A, C - A)
    assert (np.linalg.norm(n, axis=1) > 0).all()
    assert ((n * (A + B + C)).sum(1) > 0).all()             # still facing outward
    rad = np.linalg.norm(Vo, axis=1)
    assert rad.max() <= 1.0 + 1e-6 and rad.min() > 0.985
    assert r["alive"][-1] == 500 and (np.diff(r["alive"]) < 0).all()


def test_open_grid_keeps_boundary_and_plane():
    n = 20
    xs = np.linspace(-1, 1, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    F = np.asarray(F, np.int32)
    u, c = _edges(F)
    bnd = np.zeros(len(V), bool)
    bnd[u[c == 1].ravel()] = True
    r = oracle.qem_simplify(V, F, 200)
    assert len(r["F"]) <= 200
    assert (r["V"][:, 2] == 0).all()
    kept_bnd = bnd[r["keep_v"]]
    assert np.array_equal(r["V"][kept_bnd], V[r["keep_v"][kept_bnd]].astype(np.float64))
    # boundary edges collapse onto one of their endpoints: every boundary vertex
    # of the result is an original boundary vertex, where it was
    uo, co = _edges(r["F"])
    assert kept_bnd[np.unique(uo[co == 1])].all()
    n_out = np.cross(r["V"][r["F"][:, 1]] - r["V"][r["F"][:, 0]], r["V"][r["F"][:, 2]] - r["V"][r["F"][:, 0]])
    assert (n_out[:, 2] > 0).all()


def test_tetrahedron_does_not_collapse():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    F = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    r = oracle.qem_simplify(V, F, 2)
    assert len(r["F"]) == 4 and r["rounds"] == 0


def test_one_round_collapses_are_independent():
    V, F = synth.sh_displaced_sphere(3, 5, amp=0.08)
    r = oracle.qem_simplify(V, F, 10, max_rounds=1)
    assert r["rounds"] == 1 and r["collapses"][0] > 10
    dead = np.setdiff1d(np.arange(len(V)), r["keep_v"])
    # partner of each removed vertex: the vertex that took its place in its faces
    Fo_orig = r["keep_v"][r["F"]]
    partner = {}
    keep_f = r["keep_f"]
    for k, f in enumerate(keep_f):
        for j in range(3):
            if F[f, j] in set(dead):
                partner[int(F[f, j])] = int(Fo_orig[k, j])
    assert set(partner) == set(dead.tolist())
    u, _ = _edges(F)
    adj = {tuple(e) for e in u.tolist()}
    ends = sorted(set(partner) | set(partner.values()))
    pair = {**partner, **{a: b for b, a in partner.items()}}
    for i, x in enumerate(ends):
        for y in ends[i + 1:]:
            if pair.get(x) == y:
                assert (min(x, y), max(x, y)) in adj          # a collapsed edge
            else:
                assert (min(x, y), max(x, y)) not in adj, (x, y)


def test_sdf_surface_stays_close():
    V, F = synth.sdf_mesh(synth.sdf_union_params(3, 12), 48, device="cpu")
    diam = float(np.linalg.norm(V.max(0) - V.min(0)))
    r = oracle.qem_simplify(V, F, len(F) // 8)
    assert len(r["F"]) == len(F) // 8
    bvh = oracle.Bvh(V, F)
    d = np.array([np.sqrt(oracle.closest_point(V, F, v, diam, bvh=bvh)[1]) for v in r["V"]]) / diam
    # an 8x reduction: vertices stay on the surface but for thin features
    assert d.mean() < 5e-4 and np.percentile(d, 99) < 2e-3 and d.max() < 2e-2
    u, c = _edges(r["F"])
    assert (c == 2).all()
