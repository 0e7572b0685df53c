"""Pins for the oracle's baking loss and its analytic gradient.

L = mean over hit texels of t^2 + lambda * mean of (1 - n_hit . d), with the
hit triangles held fixed.  The analytic gradient is checked against FP64
central finite differences (h = 1e-4) of the same loss on the 320-face
icosphere over the 5,120-face displaced sphere; the identity (high == low)
is a minimum with L = 0 and zero gradient.
"""
import numpy as np
import pytest

import oracle
from paper_2605_26137_b300 import synth


def _setup(seed=0):
    a = synth.tiny_asset(seed)
    r = oracle.bake_asset(a)
    return a, r


@pytest.mark.slow
def test_analytic_gradient_matches_finite_differences():
    a, r = _setup(0)
    lv = a.low_v.astype(np.float64)
    L, g = oracle.loss_grad(a.high_v, a.high_f, r["high_normals"], lv, a.low_f, r["face"], r["bary"], r["hit_tri"], 0.1)
    # the loss reproduces the forward bake's hit distances
    m = r["mask"] == 1
    n_hit = m.sum()
    assert n_hit > 0
    assert L >= np.mean(r["disp"][m] ** 2) - 1e-12
    fd = oracle.fd_grad(a.high_v, a.high_f, r["high_normals"], lv, a.low_f, r["face"], r["bary"], r["hit_tri"], 0.1, h=1e-4)
    rel = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert rel < 1e-6
    # per-coordinate agreement where the gradient is not tiny
    big = np.abs(fd) > 1e-3 * np.abs(fd).max()
    assert np.abs((g[big] - fd[big]) / fd[big]).max() < 1e-4


def test_loss_terms_without_normal_term():
    a, r = _setup(2)
    lv = a.low_v.astype(np.float64)
    L, _ = oracle.loss_grad(a.high_v, a.high_f, r["high_normals"], lv, a.low_f, r["face"], r["bary"], r["hit_tri"], 0.0, False)
    m = r["mask"] == 1
    assert L == pytest.approx(np.mean(r["disp"][m] ** 2), rel=1e-10)


def test_identity_is_a_minimum():
    V, F = synth.sh_displaced_sphere(2, 5)
    uv = synth.grid_atlas(len(F), 128, 128, 2)
    r = oracle.bake(V, F, V, F, uv, 128, 128, 0.1)
    L, g = oracle.loss_grad(V, F, r["high_normals"], V.astype(np.float64), F, r["face"], r["bary"], r["hit_tri"], 0.1)
    assert abs(L) < 1e-14
    assert np.abs(g).max() < 1e-9


def test_gradient_coordinate_subset_sign():
    """Moving a vertex along its own gradient direction raises the loss."""
    a, r = _setup(3)
    lv = a.low_v.astype(np.float64)
    args = (a.high_v, a.high_f, r["high_normals"])
    L0, g = oracle.loss_grad(*args, lv, a.low_f, r["face"], r["bary"], r["hit_tri"], 0.1)
    step = 1e-4 * g / np.abs(g).max()
    L1, _ = oracle.loss_grad(*args, lv + step, a.low_f, r["face"], r["bary"], r["hit_tri"], 0.1, False)
    L2, _ = oracle.loss_grad(*args, lv - step, a.low_f, r["face"], r["bary"], r["hit_tri"], 0.1, False)
    assert L1 > L0 > L2


def test_normal_term_closed_form_on_tilted_plane():
    """The lambda term in closed form.  A flat low quad (normal +z) under a
    high plane z = h - s y that covers only part of it: every hit texel sees
    the plane's normal (0, s, 1)/sqrt(1 + s^2), so n_hit . d = 1/sqrt(1 + s^2)
    and L(lambda) - L(0) = lambda (1 - 1/sqrt(1 + s^2)), with the mean taken
    over the hit texels only.  Texels the plane does not cover miss, so a
    mean over all ray texels would scale the term by the hit fraction."""
    h, s = 0.05, 0.3
    lv = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0]], np.float32)
    lf = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    uv = np.array([[(0.1 + 0.4 * (lv[i, 0] + 1), 0.1 + 0.4 * (lv[i, 1] + 1)) for i in f] for f in lf], np.float32)
    n = 24
    xs, ys = np.linspace(-1.5, 0.2, n + 1), np.linspace(-1.5, 1.5, n + 1)
    X, Y = np.meshgrid(xs, ys)
    hv = np.stack([X.ravel(), Y.ravel(), h - s * Y.ravel()], -1).astype(np.float32)
    hf = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            hf += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    hf = np.asarray(hf, np.int32)
    r = oracle.bake(hv, hf, lv, lf, uv, 64, 64, 0.5)
    ray = r["face"] >= 0
    hit = ray & (r["mask"] == 1)
    frac = hit.sum() / ray.sum()
    assert 0.4 < frac < 0.8, frac
    args = (hv, hf, r["high_normals"], lv.astype(np.float64), lf, r["face"], r["bary"], r["hit_tri"])
    L0, _ = oracle.loss_grad(*args, 0.0, False)
    for lam in (0.1, 0.7):
        L, _ = oracle.loss_grad(*args, lam, False)
        assert (L - L0) / lam == pytest.approx(1.0 - 1.0 / np.sqrt(1.0 + s * s), abs=1e-6)
