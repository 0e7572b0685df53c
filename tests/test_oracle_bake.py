"""Pins for the oracle's full bake (Sec. 6.4): closed forms and invariants.

* a flat low plane over a flat high plane bakes to (0,0,1) with displacement
  equal to the plane offset (and misses beyond max_dist);
* identical high and low meshes bake to (0,0,1) with zero displacement;
* a fine sphere over a coarse icosphere gives the analytic sphere normal;
* signed axis permutations of both meshes leave the bake unchanged, general
  rotations change it by no more than the FP32 input rounding;
* tangent-space normals have unit length;
* the UV-gradient tangent of an affinely mapped plane is dp/du;
* the RGB8 encoding and the dilation rule on hand-checked maps.
"""
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def _grid_plane(n, z=0.0, size=1.0):
    xs = np.linspace(-size, size, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.asarray(F, np.int32)


def _frame_world(r, lv, lf):
    """World-space normal from the tangent-space one, using the oracle's frames."""
    face, bary = r["face"], r["bary"]
    m = face >= 0
    f = face[m]
    b = bary[m]
    ln = r["low_normals"]
    N = (b[:, :, None] * ln[lf[f]]).sum(1)
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    T = (b[:, :, None] * r["tangents"][f]).sum(1)
    T -= (T * N).sum(1, keepdims=True) * N
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    B = np.cross(N, T) * r["wsign"][f][:, None]
    n = r["nts"][m]
    return n[:, :1] * T + n[:, 1:2] * B + n[:, 2:3] * N, m


@pytest.mark.parametrize("z", [0.04, -0.03])
def test_flat_plane(z):
    lv, lf = _grid_plane(6)
    hv, hf = _grid_plane(20, z, 1.5)
    uv = synth.grid_atlas(len(lf), 64, 64, 2)
    r = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.05)
    m = r["face"] >= 0
    assert m.sum() > 0 and r["mask"][m].all()
    assert np.abs(r["nts"][m] - [0, 0, 1]).max() < 1e-12
    assert np.abs(r["disp"][m] - np.float32(z)).max() < 1e-12
    r2 = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.02)
    assert not r2["mask"].any()
    assert np.array_equal(r2["rgba8"][m][:, :3], np.tile([128, 128, 255], (m.sum(), 1)))


def test_identity_high_equals_low():
    V, F = synth.sh_displaced_sphere(3, 11)
    uv = synth.grid_atlas(len(F), 256, 256, 2)
    r = oracle.bake(V, F, V, F, uv, 256, 256, 0.1)
    m = r["face"] >= 0
    assert r["mask"][m].all()
    assert np.abs(r["disp"][m]).max() < 1e-12
    assert np.abs(r["nts"][m] - [0, 0, 1]).max() < 1e-9


def test_sphere_analytic_normal():
    lv, lf = synth.icosphere(2)
    hv, hf = synth.icosphere(6)
    uv = synth.grid_atlas(len(lf), 256, 256, 2)
    r = oracle.bake(hv, hf, lv, lf, uv, 256, 256, 0.2)
    nw, m = _frame_world(r, lv, lf)
    assert r["mask"][m].all()
    # hit point and its exact sphere normal
    face, bary = r["face"][m], r["bary"][m]
    p = (bary[:, :, None] * lv.astype(np.float64)[lf[face]]).sum(1)
    d = (bary[:, :, None] * r["low_normals"][lf[face]]).sum(1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = p + r["hit_t"][m][:, None] * d
    exact = x / np.linalg.norm(x, axis=1, keepdims=True)
    err = np.arccos(np.clip((nw * exact).sum(1), -1, 1))
    # bound: the high vertex normals' own deviation from radial plus the
    # angular sag of linear interpolation across one edge (edge angle^2)
    hn = r["high_normals"]
    hd = hv.astype(np.float64) / np.linalg.norm(hv.astype(np.float64), axis=1, keepdims=True)
    vdev = np.arccos(np.clip((hn * hd).sum(1), -1, 1)).max()
    e = np.concatenate([hf[:, [0, 1]], hf[:, [1, 2]], hf[:, [2, 0]]])
    edge_ang = np.arccos(np.clip((hd[e[:, 0]] * hd[e[:, 1]]).sum(1), -1, 1)).max()
    assert err.max() <= vdev + edge_ang ** 2 + 1e-9
    assert np.degrees(err.max()) < 0.1 and np.degrees(err.mean()) < 0.03
    # the coarse sphere's own (face) normal is far off: the bake really transfers detail
    assert np.abs(r["nts"][m][:, :2]).max() > 1e-3


def test_signed_permutation_invariance():
    a = synth.tiny_asset(4)
    r0 = oracle.bake_asset(a)
    P = np.array([[0, 0, -1], [1, 0, 0], [0, -1, 0]], np.float32)  # det +1, exact in FP32
    hv = a.high_v @ P.T
    lv = a.low_v @ P.T
    r1 = oracle.bake(hv, a.high_f, lv, a.low_f, a.low_uv, a.W, a.H, a.max_dist, a.gutter)
    assert np.array_equal(r0["mask"], r1["mask"])
    assert np.abs(r0["nts"] - r1["nts"]).max() < 1e-9
    assert np.abs(r0["disp"] - r1["disp"]).max() < 1e-12


def test_rigid_invariance_general():
    a = synth.tiny_asset(5)
    r0 = oracle.bake_asset(a)
    rng = np.random.default_rng(0)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    tr = np.array([0.3, -0.2, 0.5])
    hv = (a.high_v.astype(np.float64) @ q.T + tr).astype(np.float32)
    lv = (a.low_v.astype(np.float64) @ q.T + tr).astype(np.float32)
    r1 = oracle.bake(hv, a.high_f, lv, a.low_f, a.low_uv, a.W, a.H, a.max_dist, a.gutter)
    both = (r0["mask"] == 1) & (r1["mask"] == 1) & ((r0["flags"] & 0b1011) == 0)
    assert both.sum() > 0.9 * (r0["face"] >= 0).sum()
    assert np.abs(r0["nts"][both] - r1["nts"][both]).max() < 1e-4
    assert np.abs(r0["disp"][both] - r1["disp"][both]).max() < 1e-5


def test_unit_length_and_encoding():
    a = synth.tiny_asset(1)
    r = oracle.bake_asset(a)
    assert np.abs(np.linalg.norm(r["nts"], axis=-1) - 1).max() < 1e-12
    filled = r["filled"] > 0
    dec = (r["rgba8"][..., :3].astype(np.float64) - 128) / 127
    assert np.abs(dec - r["nts"]).max() <= 0.5 / 127 + 1e-6
    assert np.all(r["rgba8"][..., 3][filled] == 255) and np.all(r["rgba8"][..., 3][~filled] == 0)


def test_encode_exact_values():
    vals = np.array([-1.0, 1.0, 0.0, -2.0, 2.0, 1 / 255, -1 / 255, 0.5])
    nts = np.stack([vals, vals, vals], -1)
    rgba = oracle.encode(nts, np.ones(len(vals), np.uint8))
    # 128 + round_half_away(127 * clamp(c, -1, 1))
    assert rgba[:, 0].tolist() == [1, 255, 128, 1, 255, 128, 128, 192]
    # zero lies in the middle of code 128: noise of either sign keeps the code
    tiny = np.array([[1e-7, -1e-7, 3e-3], [-3e-3, 0.0, -0.0]])
    assert oracle.encode(tiny, np.ones(2, np.uint8))[:, :3].tolist() == [[128, 128, 128], [128, 128, 128]]
    # half-way cases round away from zero
    half = np.array([[0.5 / 127, -0.5 / 127, 1.5 / 127]])
    assert oracle.encode(half, np.ones(1, np.uint8))[0, :3].tolist() == [129, 127, 130]


def test_tangent_is_dp_du_on_affine_plane():
    V = np.array([[0, 0, 0], [2, 0, 0], [0, 1, 0], [2, 1, 0]], np.float32)
    F = np.array([[0, 1, 3], [0, 3, 2]], np.int32)
    # u = 0.1 + 0.2 y + 0.1 x, v = 0.2 + 0.3 x ; p(u,v) affine
    def uvmap(p):
        return (0.1 + 0.2 * p[1] + 0.1 * p[0], 0.2 + 0.3 * p[0])
    uv = np.array([[uvmap(V[i]) for i in f] for f in F], np.float32)
    W = H = 1024
    N = oracle.vertex_normals(V, F)
    T, w, dg = oracle.face_frames(V, F, uv, W, H, N)
    # [du dv] = J [dx dy]; dp/du = first column of J^-1 (in xy), embedded in z=0
    J = np.array([[0.1, 0.2], [0.3, 0.0]])
    Ji = np.linalg.inv(J)
    dpdu = np.array([Ji[0, 0], Ji[1, 0], 0.0])
    dpdv = np.array([Ji[0, 1], Ji[1, 1], 0.0])
    dpdu /= np.linalg.norm(dpdu)
    assert not dg.any()
    assert np.abs(T - dpdu).max() < 1e-4  # UV snapping to 1/256 texel perturbs the map
    hand = np.sign(np.cross(N[0], dpdu) @ dpdv)
    assert np.all(w == hand)


def test_dilation_hand_checked():
    W, H = 5, 4
    filled = np.zeros((H, W), np.uint8)
    nts = np.zeros((H, W, 3))
    nts[..., 2] = 1
    disp = np.zeros((H, W))
    filled[1, 0] = 1
    nts[1, 0] = (1, 0, 0)
    disp[1, 0] = 0.2
    filled[1, 2] = 1
    nts[1, 2] = (0, 1, 0)
    disp[1, 2] = 0.4
    f1, n1, d1 = oracle.dilate(W, H, 1, filled, nts, disp)
    s = np.sqrt(0.5)
    assert np.allclose(n1[1, 1], (s, s, 0)) and np.isclose(d1[1, 1], 0.3)
    assert np.allclose(n1[0, 0], (1, 0, 0)) and np.isclose(d1[0, 0], 0.2)
    assert np.allclose(n1[2, 3], (0, 1, 0)) and np.isclose(d1[2, 3], 0.4)
    assert f1[3].sum() == 0 and f1[:, 4].sum() == 0  # only one ring after one pass
    assert f1[1, 1] == 2 and f1[1, 0] == 1
    f2, n2, d2 = oracle.dilate(W, H, 2, filled, nts, disp)
    # second pass: (3,1) sees (2,0) (2,1) (2,2) from pass one
    exp = n1[2, 0] + n1[2, 1] + n1[2, 2]
    assert np.allclose(n2[3, 1], exp / np.linalg.norm(exp))
    assert np.isclose(d2[3, 1], (d1[2, 0] + d1[2, 1] + d1[2, 2]) / 3)
    assert f2[3, 4] == 0 or f2[3, 4] == 2


@pytest.mark.parametrize("mirror", [False, True])
def test_bitangent_follows_dp_dv(mirror):
    """A tilted high plane z = h - s y over the flat low quad, with UVs an
    affine function of position (v increasing or, mirrored, decreasing with
    y): the texel frame is T = dp/du = +x, B along +dp/dv (so -y when
    mirrored), N = +z, and the hit normal (0, s, 1) / sqrt(1 + s^2) has
    tangent-space components (0, +-s, 1) / sqrt(1 + s^2)."""
    h, s = 0.05, 0.02
    lv = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    lf = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    sgn = -1.0 if mirror else 1.0

    def uvmap(p):
        return (0.1 + 0.4 * (p[0] + 1), 0.5 + sgn * 0.4 * p[1])
    uv = np.array([[uvmap(lv[i]) for i in f] for f in lf], np.float32)
    hv, hf = _grid_plane(24, 0.0, 1.5)
    hv[:, 2] = (h - s * hv[:, 1].astype(np.float64)).astype(np.float32)
    r = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.1)
    m = r["face"] >= 0
    assert m.sum() > 1000 and r["mask"][m].all()
    k = 1.0 / np.sqrt(1 + s * s)
    exp = np.array([0.0, sgn * s * k, k])
    assert np.abs(r["nts"][m] - exp).max() < 2e-4
