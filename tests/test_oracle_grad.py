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
