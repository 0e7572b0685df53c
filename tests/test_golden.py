"""The oracle against the stored fixtures of tests/golden/: hand-derived closed
forms (RGB8 encoding, one dilation pass, a flat plane over a flat plane) and
the oracle's own earlier bake of the seeded tiny asset (a guard against
unintended change of its arithmetic; see make_oracle_regression.py)."""
import hashlib
import os

import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_encode_fixture():
    rows = _rows("encode_rgb8.txt")
    c = np.array([float(r[0]) for r in rows])
    code = [int(r[1]) for r in rows]
    rgba = oracle.encode(np.stack([c, c, c], -1), np.ones(len(c), np.uint8))
    assert rgba[:, 0].tolist() == code and rgba[:, 2].tolist() == code
    assert np.all(rgba[:, 3] == 255)


def test_dilation_fixture():
    W, H = 5, 4
    filled = np.zeros((H, W), np.uint8)
    nts = np.zeros((H, W, 3))
    nts[..., 2] = 1
    disp = np.zeros((H, W))
    filled[1, 0], nts[1, 0], disp[1, 0] = 1, (1, 0, 0), 0.2
    filled[1, 2], nts[1, 2], disp[1, 2] = 1, (0, 1, 0), 0.4
    f1, n1, d1 = oracle.dilate(W, H, 1, filled, nts, disp)
    seen = np.zeros((H, W), bool)
    for r in _rows("dilation_5x4.txt"):
        x, y = int(r[0]), int(r[1])
        seen[y, x] = True
        assert np.allclose(n1[y, x], [float(v) for v in r[2:5]], atol=1e-15), (x, y)
        assert abs(d1[y, x] - float(r[5])) < 1e-15, (x, y)
        assert f1[y, x] == int(r[6]), (x, y)
    assert f1[1, 0] == 1 and f1[1, 2] == 1
    seen[1, 0] = seen[1, 2] = True
    assert np.all(f1[~seen] == 0)   # row 3 and column 4


def _grid_plane(n, z, size):
    xs = np.linspace(-size, size, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.asarray(F, np.int32)


@pytest.mark.parametrize("row", range(3))
def test_flat_plane_fixture(row):
    r = _rows("flat_plane.txt")[row]
    h, max_dist, hit = float(r[0]), float(r[1]), int(r[2])
    lv, lf = _grid_plane(6, 0.0, 1.0)
    hv, hf = _grid_plane(20, h, 1.5)
    uv = synth.grid_atlas(len(lf), 64, 64, 2)
    o = oracle.bake(hv, hf, lv, lf, uv, 64, 64, max_dist)
    m = o["face"] >= 0
    assert m.sum() > 0
    if not hit:
        assert not o["mask"].any()
        return
    assert o["mask"][m].all()
    assert np.abs(o["nts"][m] - [float(v) for v in r[3:6]]).max() < 1e-12
    assert np.all(o["rgba8"][m] == [int(v) for v in r[6:9]] + [255])
    assert np.abs(o["disp"][m] - np.float32(float(r[9]))).max() < 1e-12


def test_oracle_regression_tiny_asset():
    rows = _rows("oracle_tiny_asset.txt")
    kv = {r[0]: r[1] for r in rows if len(r) == 2}
    a = synth.tiny_asset(1)
    o = oracle.bake_asset(a)

    def digest(x):
        return hashlib.sha256(np.ascontiguousarray(x).tobytes()).hexdigest()

    assert digest(o["face"].astype(np.int32)) == kv["face_map_sha256"]
    assert digest(o["rgba8"].astype(np.uint8)) == kv["rgba8_sha256"]
    assert digest(o["mask"].astype(np.uint8)) == kv["mask_sha256"]
    assert int((o["face"] >= 0).sum()) == int(kv["ray_texels"])
    assert int(o["mask"].sum()) == int(kv["hits"])
    for r in (r for r in rows if len(r) == 7):
        x, y, f = int(r[0]), int(r[1]), int(r[2])
        assert o["face"][y, x] == f
        assert np.abs(o["nts"][y, x] - [float(v) for v in r[3:6]]).max() < 1e-12
        assert abs(o["disp"][y, x] - float(r[6])) < 1e-12
