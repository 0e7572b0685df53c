"""Pins for the oracle's closest-point query (Sec. 6.4 words the
correspondence as the nearest point of the high-poly surface to each texel's
world-space position).

* one triangle: hand-computed interior, edge and vertex cases; on random
  triangles (slivers and a zero-area one included) the returned point lies in
  the triangle, reproduces the returned distance, and no point of a dense
  sampling of the triangle is closer;
* the median-split BVH returns exactly what brute force returns;
* a sphere: the distance lies between the inscribed polyhedron's bounds;
* the distance filter is inclusive; ties prefer the lower triangle id;
* whole bakes: a flat high plane gives (0,0,1) and the signed offset, the
  same as the ray query; identical meshes give (0,0,1) and zero; a fine
  sphere gives the radial normal; a ridge seen from below flags the texels
  above its crease as ambiguous and no others.
"""
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth

ONE = np.array([[0, 1, 2]], np.int32)


def _tri(A, B, C):
    return np.array([A, B, C], np.float32)


def _cp1(V, p, rmax=100.0):
    return oracle.closest_point(V, ONE, np.asarray(p, np.float64), rmax)


def test_single_triangle_hand_cases():
    V = _tri((0, 0, 0), (1, 0, 0), (0, 1, 0))
    # above the interior: the foot of the perpendicular
    tri, d2, x, b = _cp1(V, (0.25, 0.5, 3.0))
    assert tri == 0 and d2 == 9.0 and np.array_equal(x, [0.25, 0.5, 0.0])
    assert np.allclose(b, [0.25, 0.25, 0.5], atol=1e-15)
    # vertex region of A
    tri, d2, x, b = _cp1(V, (-1.0, -2.0, 0.0))
    assert d2 == 5.0 and np.array_equal(x, [0, 0, 0]) and np.array_equal(b, [1, 0, 0])
    # edge AB region: projection onto the x axis
    tri, d2, x, b = _cp1(V, (0.75, -2.0, 1.0))
    assert d2 == 5.0 and np.array_equal(x, [0.75, 0, 0]) and np.allclose(b, [0.25, 0.75, 0])
    # hypotenuse BC: (1,1,0) projects to its midpoint
    tri, d2, x, b = _cp1(V, (1.0, 1.0, 0.0))
    assert d2 == pytest.approx(0.5, rel=1e-15) and np.allclose(x, [0.5, 0.5, 0]) and np.allclose(b, [0, 0.5, 0.5])
    # a point on the triangle is its own closest point
    tri, d2, x, b = _cp1(V, (0.125, 0.25, 0.0))
    assert d2 == 0.0 and np.array_equal(x, [0.125, 0.25, 0.0])


def _samples(Vd, n=60, rng=None):
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1))
    keep = i + j <= n
    bb = np.stack([i[keep], j[keep]], -1) / n
    pts = [Vd[0] + bb[:, :1] * (Vd[1] - Vd[0]) + bb[:, 1:] * (Vd[2] - Vd[0])]
    s = np.linspace(0, 1, 2001)[:, None]
    for k in range(3):
        pts.append(Vd[k] + s * (Vd[(k + 1) % 3] - Vd[k]))
    if rng is not None:
        r = rng.dirichlet((1, 1, 1), 4000)
        pts.append(r @ Vd)
    return np.concatenate(pts)


def test_random_triangles_against_dense_sampling():
    rng = np.random.default_rng(7)
    tris = [rng.normal(size=(3, 3)) for _ in range(60)]
    tris.append(np.array([[0, 0, 0], [1, 1e-4, 0], [2, 0, 1e-4]]))      # sliver
    tris.append(np.array([[0, 0, 0], [1, 1, 1], [3, 3, 3]]))            # zero area
    tris.append(np.array([[0, 0, 0], [0, 0, 0], [1, 2, 0]]))            # repeated vertex
    for T in tris:
        V = T.astype(np.float32)
        Vd = V.astype(np.float64)
        S = _samples(Vd, rng=rng)
        for _ in range(15):
            p = rng.normal(size=3) * rng.choice([0.1, 1.0, 3.0])
            tri, d2, x, b = _cp1(V, p)
            assert tri == 0
            # a point of the closed triangle ...
            assert b.min() >= -1e-12 and abs(b.sum() - 1) < 1e-12
            assert np.abs(b @ Vd - x).max() < 1e-12 * (1 + np.abs(Vd).max())
            # ... at the returned distance ...
            assert abs(np.sum((p - x) ** 2) - d2) <= 1e-12 * max(d2, 1e-300) + 1e-28
            # ... and no sample of the triangle is closer
            ds = np.sum((S - p) ** 2, 1)
            assert ds.min() >= d2 * (1 - 1e-12) - 1e-28
            # near-optimal against the sampling resolution
            h = np.abs(Vd[1:] - Vd[0]).max() * 2 / 60 + 1e-12
            assert np.sqrt(ds.min()) <= np.sqrt(d2) + h


def test_bvh_equals_brute_force():
    V, F = synth.sh_displaced_sphere(4, 3)
    bvh = oracle.Bvh(V, F)
    rng = np.random.default_rng(0)
    for _ in range(300):
        p = rng.normal(size=3)
        p *= rng.uniform(0.7, 1.3) / np.linalg.norm(p)
        rmax = rng.uniform(0.01, 0.5)
        a = oracle.closest_point(V, F, p, rmax)
        b = oracle.closest_point(V, F, p, rmax, bvh=bvh)
        assert a[0] == b[0] and a[1] == b[1]
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    # points on vertices and edge midpoints: exact ties between neighbours
    Vd = V.astype(np.float64)
    for f in F[:200]:
        for p in (Vd[f[0]], 0.5 * (Vd[f[0]] + Vd[f[1]])):
            a = oracle.closest_point(V, F, p, 0.1)
            b = oracle.closest_point(V, F, p, 0.1, bvh=bvh)
            assert a[0] == b[0] and a[1] == b[1] and a[1] < 1e-30


def test_sphere_distance_bounds():
    V, F = synth.icosphere(5, 1.0)
    Vd = V.astype(np.float64)
    # the FP32 polyhedron lies between the sphere through its farthest vertex
    # and the sphere tangent to its nearest face plane
    R = np.linalg.norm(Vd, axis=1).max()
    n = np.cross(Vd[F[:, 1]] - Vd[F[:, 0]], Vd[F[:, 2]] - Vd[F[:, 0]])
    rin = (np.abs((n * Vd[F[:, 0]]).sum(1)) / np.linalg.norm(n, axis=1)).min()
    bvh = oracle.Bvh(V, F)
    rng = np.random.default_rng(2)
    for _ in range(200):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        rho = rng.uniform(0.8, 1.2)
        tri, d2, x, b = oracle.closest_point(V, F, rho * u, 1.0, bvh=bvh)
        d = np.sqrt(d2)
        assert tri >= 0
        if rho >= R:
            assert rho - R - 1e-12 <= d <= rho - rin + 1e-12
        elif rho <= rin:
            assert rin - rho - 1e-12 <= d <= R - rho + 1e-12
        r = np.linalg.norm(x)
        assert rin - 1e-12 <= r <= R + 1e-12
        # the closest point of a convex surface from outside lies along the
        # face normal: x is where the radial direction meets the polyhedron
        if rho > R:
            assert np.degrees(np.arccos(np.clip(u @ (x / r), -1, 1))) < 2.0


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


def test_filter_inclusive_and_ties():
    Vp, Fp = _plane(2, 0.02)
    p = np.array([0.1, 0.2, 0.0])
    z = float(np.float32(0.02))
    tri, d2, x, b = oracle.closest_point(Vp, Fp, p, z)
    assert tri >= 0 and d2 == z * z
    tri, _, _, _ = oracle.closest_point(Vp, Fp, p, np.nextafter(z, 0))
    assert tri == -1
    # duplicated triangles: the lower id wins
    F = np.concatenate([Fp[::-1], Fp])
    tri, d2, x, b = oracle.closest_point(Vp, F, p, 1.0)
    assert tri < len(Fp) and d2 == z * z
    # two planes at +c and -c: equal distance, the lower id wins (no sign preference)
    V1, F1 = _plane(2, 0.05)
    V2, F2 = _plane(2, -0.05)
    V = np.concatenate([V1, V2])
    F = np.concatenate([F1, F2 + len(V1)])
    tri, d2, x, b = oracle.closest_point(V, F, p, 1.0)
    assert tri < len(F1) and x[2] == pytest.approx(0.05)
    F = np.concatenate([F2 + len(V1), F1])
    tri, d2, x, b = oracle.closest_point(V, F, p, 1.0)
    assert tri < len(F2) and x[2] == pytest.approx(-0.05)


# ------------------------------------------------------------- whole bakes

@pytest.mark.parametrize("z", [0.04, -0.03])
def test_bake_flat_plane_matches_ray(z):
    lv, lf = _plane(6, 0.0, 1.0)
    hv, hf = _plane(20, z, 1.5)
    uv = synth.grid_atlas(len(lf), 64, 64, 2)
    c = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.05, query="closest")
    r = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.05)
    m = c["face"] >= 0
    assert m.sum() > 0 and c["mask"][m].all()
    assert np.abs(c["nts"][m] - [0, 0, 1]).max() < 1e-12
    assert np.abs(c["disp"][m] - np.float32(z)).max() < 1e-12     # signed by the texel normal (+z)
    assert np.abs(c["disp"] - r["disp"]).max() < 1e-12
    assert not (c["flags"][m] & 0b1010).any()
    c2 = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.02, query="closest")
    assert not c2["mask"].any()


def test_bake_identity():
    V, F = synth.sh_displaced_sphere(3, 11)
    uv = synth.grid_atlas(len(F), 256, 256, 2)
    c = oracle.bake(V, F, V, F, uv, 256, 256, 0.1, query="closest")
    m = c["face"] >= 0
    assert c["mask"][m].all()
    assert np.abs(c["disp"][m]).max() < 1e-12
    assert np.abs(c["nts"][m] - [0, 0, 1]).max() < 1e-9
    assert not (c["flags"][m] & 0b1000).any()


def test_bake_sphere_radial_normal():
    lv, lf = synth.icosphere(2)
    hv, hf = synth.icosphere(6)
    uv = synth.grid_atlas(len(lf), 256, 256, 2)
    c = oracle.bake(hv, hf, lv, lf, uv, 256, 256, 0.2, query="closest")
    m = (c["face"] >= 0) & ((c["flags"] & 0b1000) == 0)
    assert c["mask"][c["face"] >= 0].all()
    face, bary = c["face"][m], c["bary"][m]
    p = (bary[:, :, None] * lv.astype(np.float64)[lf[face]]).sum(1)
    rho = np.linalg.norm(p, axis=1)
    # the low mesh lies inside the unit sphere: positive offset along the
    # (outward) texel normal, about 1 - |p|
    assert (c["disp"][m] > 0).all()
    assert np.abs(c["disp"][m] - (1 - rho)).max() < 1.5e-4
    # world normal from the tangent frame equals the radial direction at the hit
    ln = c["low_normals"]
    N = (bary[:, :, None] * ln[lf[face]]).sum(1)
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    T = (bary[:, :, None] * c["tangents"][face]).sum(1)
    T -= (T * N).sum(1, keepdims=True) * N
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    B = np.cross(N, T) * c["wsign"][face][:, None]
    n = c["nts"][m]
    nw = n[:, :1] * T + n[:, 1:2] * B + n[:, 2:3] * N
    x = p / rho[:, None]
    err = np.degrees(np.arccos(np.clip((nw * x).sum(1), -1, 1)))
    assert err.max() < 0.2 and err.mean() < 0.05


def test_bake_ridge_flags_crease():
    # low: the plane z = 0; high: the ridge z = 0.05 - 0.2 |x - x0| above it,
    # built from two sheets with separate vertices (each slope keeps its own
    # constant normal), its crease x0 placed on a column of texel centres
    lv, lf = _plane(4, 0.0, 1.0)
    W = H = 128
    uv = synth.grid_atlas(len(lf), W, H, 2)
    face, bary, _ = oracle.raster(uv, W, H)
    m = face >= 0
    px = (bary[m][:, :, None] * lv.astype(np.float64)[lf[face[m]]]).sum(1)[:, 0]
    x0 = float(np.float32(px[np.argmin(np.abs(px - 0.1))]))
    n = 20
    X, Y = np.meshgrid(np.linspace(0.0, 1.5, n + 1), np.linspace(-1.5, 1.5, n + 1))
    right = np.stack([x0 + X.ravel(), Y.ravel(), (0.05 - 0.2 * X).ravel()], -1)
    left = np.stack([x0 - X.ravel(), Y.ravel(), (0.05 - 0.2 * X).ravel()], -1)
    hv = np.concatenate([right, left]).astype(np.float32)
    _, f1 = _plane(n, 0.0)
    hf = np.concatenate([f1, f1[:, ::-1] + (n + 1) ** 2]).astype(np.int32)
    c = oracle.bake(hv, hf, lv, lf, uv, W, H, 0.2, query="closest")
    amb = (c["flags"][m] & 0b1000) != 0
    off = np.abs(px - x0)
    # under the crease both slopes are equally close
    on = off < 1e-7
    assert on.sum() >= 10 and amb[on].all()
    # away from it the gap 2 * 0.2 |x - x0| / sqrt(1.04) exceeds the 1e-7*diam tolerance
    away = off > 1e-5
    assert not amb[away].any()
    # the closest point lies on the slope facing the texel: distance and normal
    dexp = (0.05 - 0.2 * off[away]) / np.sqrt(1.04)
    assert np.abs(c["disp"][m][away] - dexp).max() < 1e-7
    nts = c["nts"][m][away]
    assert np.abs(nts[:, 2] - 1 / np.sqrt(1.04)).max() < 1e-6   # FP32 vertex rounding
    assert np.abs(np.hypot(nts[:, 0], nts[:, 1]) - 0.2 / np.sqrt(1.04)).max() < 1e-6


def test_bake_signed_permutation_invariance():
    a = synth.tiny_asset(4)
    r0 = oracle.bake_asset(a, query="closest")
    P = np.array([[0, 0, -1], [1, 0, 0], [0, -1, 0]], np.float32)  # det +1, exact in FP32
    r1 = oracle.bake(a.high_v @ P.T, a.high_f, a.low_v @ P.T, a.low_f, a.low_uv, a.W, a.H, a.max_dist, a.gutter,
                     query="closest")
    assert np.array_equal(r0["mask"], r1["mask"])
    assert np.array_equal(r0["flags"], r1["flags"])
    assert np.abs(r0["nts"] - r1["nts"]).max() < 1e-9
    assert np.abs(r0["disp"] - r1["disp"]).max() < 1e-12
