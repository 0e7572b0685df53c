"""Pins for the oracle's closest-hit query (Sec. 6.4, correspondence step).

* the median-split BVH returns exactly what brute force returns;
* analytic ray/plane and ray/sphere distances;
* watertightness: rays aimed at vertices and edge midpoints of a closed mesh
  from inside it always hit;
* the tie rules (|t| ties prefer t >= 0, t ties prefer the lower id);
* hit point consistency: o + t d equals the barycentric point of the hit.
"""
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def _plane(n, z, size=2.0):
    xs = np.linspace(-size, size, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.asarray(F, np.int32)


def test_bvh_equals_brute_force_random_rays():
    V, F = synth.sh_displaced_sphere(4, 3)
    bvh = oracle.Bvh(V, F)
    rng = np.random.default_rng(0)
    for _ in range(300):
        o = rng.uniform(-1.2, 1.2, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        tmax = rng.uniform(0.05, 2.0)
        a = oracle.closest_hit(V, F, o, d, tmax)
        b = oracle.closest_hit(V, F, o, d, tmax, bvh=bvh)
        assert a[0] == b[0]
        assert a[1] == b[1]
        assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("z", [0.03, -0.07, 0.0])
def test_plane_distance(z):
    V, F = _plane(8, z)
    rng = np.random.default_rng(1)
    for _ in range(50):
        o = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), 0.0])
        d = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 1.0])
        d /= np.linalg.norm(d)
        tri, t, b = oracle.closest_hit(V, F, o, d, 0.5)
        assert tri >= 0
        assert abs(t - float(np.float32(z)) / d[2]) < 1e-14
        assert np.all(b >= -1e-15) and abs(b.sum() - 1) < 1e-14


def test_sphere_distance_within_tessellation_bound():
    R = 1.0
    V, F = synth.icosphere(5, R)
    Vd = V.astype(np.float64)
    # inscribed polyhedron: every face plane lies between R*cos(a) and R
    cosa = min(np.dot(Vd[f].mean(0) / np.linalg.norm(Vd[f].mean(0)), Vd[f[0]]) / R for f in F)
    rng = np.random.default_rng(2)
    for _ in range(100):
        o = rng.uniform(-0.3, 0.3, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        tri, t, b = oracle.closest_hit(V, F, o, d, 3.0)
        assert tri >= 0
        # analytic: |o + t d| = R  ->  t = -o.d + sqrt((o.d)^2 - |o|^2 + R^2)  (or the negative root)
        od = o @ d
        disc = np.sqrt(od * od - o @ o + R * R)
        t_exact = min((-od + disc, -od - disc), key=abs)
        x = o + t * d
        r = np.linalg.norm(x)
        assert R * cosa - 1e-12 <= r <= R + 1e-12
        assert abs(abs(t) - abs(t_exact)) < R * (1 - cosa) * 4 / abs(d @ (x / r)) + 1e-9
        # the returned barycentrics reproduce the hit point
        assert np.abs(b @ Vd[F[tri]] - x).max() < 1e-12


def test_watertight_vertices_and_edges():
    V, F = synth.sh_displaced_sphere(3, 7)
    Vd = V.astype(np.float64)
    targets = list(Vd)
    for f in F[:400]:
        for k in range(3):
            targets.append(0.5 * (Vd[f[k]] + Vd[f[(k + 1) % 3]]))
    for x in targets:
        # from just inside, straight through the vertex / edge midpoint
        d = x / np.linalg.norm(x)
        o = 0.9 * x
        tri, t, _ = oracle.closest_hit(V, F, o, d, 0.5)
        assert tri >= 0, "ray through a vertex/edge escaped"
        assert abs(t - 0.1 * np.linalg.norm(x)) < 1e-12


def test_tie_rules():
    # two planes at +c and -c: equal |t|, the positive one wins
    V1, F1 = _plane(2, 0.05)
    V2, F2 = _plane(2, -0.05)
    V = np.concatenate([V2, V1])
    F = np.concatenate([F2, F1 + len(V2)])
    o = np.array([0.1, 0.2, 0.0])
    d = np.array([0.0, 0.0, 1.0])
    tri, t, _ = oracle.closest_hit(V, F, o, d, 1.0)
    assert t == pytest.approx(0.05) and tri >= len(F2)
    # duplicated triangle: equal t, the lower id wins
    Vp, Fp = _plane(2, 0.02)
    F = np.concatenate([Fp[::-1], Fp])
    tri, t, _ = oracle.closest_hit(Vp, F, o, d, 1.0)
    dup = len(Fp) + (len(Fp) - 1 - tri) if tri < len(Fp) else tri
    assert tri < len(Fp) and np.array_equal(F[tri], F[dup])
    # tmax is inclusive
    tri, t, _ = oracle.closest_hit(Vp, Fp, o, d, 0.02)
    assert tri >= 0 and t == pytest.approx(0.02)
    tri, _, _ = oracle.closest_hit(Vp, Fp, o, d, np.nextafter(np.float32(0.02), 0) * 0.999)
    assert tri == -1


@pytest.mark.parametrize("query", ["ray", "closest"])
def test_shade_given_triangle(query):
    """The evaluation of one given triangle per texel (used to check answers
    where two triangles are within rounding of the closest one): with the
    oracle's own closest triangle it reproduces the search's normal,
    displacement and barycentrics; on a flat plane z = c any triangle gives
    t = c (the plane's crossing) and the normal (0, 0, 1); a triangle beside
    the texel's ray shows a negative barycentric (ray) or lies farther than
    the plane's distance (closest point)."""
    a = synth.tiny_asset(4)
    r = oracle.bake_asset(a, query=query)
    tex = np.flatnonzero((r["mask"] == 1).reshape(-1))[::7]
    tris = r["hit_tri"].reshape(-1)[tex]
    nts, t, b, valid = oracle.shade_given(a, tex, tris, query)
    assert valid.all()
    assert np.abs(nts - r["nts"].reshape(-1, 3)[tex]).max() < 1e-12
    assert np.abs(t - r["hit_t"].reshape(-1)[tex]).max() < 1e-12
    assert np.abs(b - r["hit_b"].reshape(-1, 3)[tex]).max() < 1e-9 and b.min() >= 0.0

    lv = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    lf = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    uv = synth.grid_atlas(2, 32, 32, 2)
    c = 0.0625
    hv, hf = _plane(8, c, 1.5)
    p = synth.Asset(hv, hf, lv, lf, uv, 32, 32, 0.5, 2)
    rp = oracle.bake_asset(p, query=query)
    tex = np.flatnonzero((rp["mask"] == 1).reshape(-1))
    own = rp["hit_tri"].reshape(-1)[tex]
    other = (own + 37) % len(hf)
    nts, t, b, valid = oracle.shade_given(p, tex, other, query)
    assert valid.all()
    assert np.abs(nts - [0.0, 0.0, 1.0]).max() < 1e-12
    if query == "ray":
        assert np.abs(t - c).max() < 1e-12
        assert (b.min(1) < -1e-3).all()
    else:
        assert (np.abs(t) > c + 1e-3).all()
