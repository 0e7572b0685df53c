"""GPU-vs-oracle comparison of one bake, with the tolerances the build is
held to (tangent-space components 1e-4 absolute, displacement 1e-5 of the
high-mesh bbox diagonal, hit masks equal except where several answers are
equally correct, 8-bit maps off by at most one code on at most 0.01% of
texels, exact integer raster).
"""
from __future__ import annotations

import numpy as np

TOL_NTS = 1e-4
TOL_DISP_REL = 1e-5
RGBA_FRAC = 1e-4
# texels compared by nothing at all (a hit on one side, a miss on the other,
# where the oracle marks the texel as one with several correct answers)
SKIP_FRAC = 1e-3
# a triangle the GPU hit must lie under the ray up to this barycentric slack
BARY_SLACK = 1e-5


def to_numpy(out) -> dict:
    d = {}
    for k in ("normal_rgba8", "mask", "disp", "normal_ts", "disp_f32", "face", "bary", "hit_tri", "hit_t"):
        v = getattr(out, k, None)
        if v is not None:
            d[k] = v.detach().cpu().numpy()
    return d


def _dilate_ring(m: np.ndarray, r: int) -> np.ndarray:
    out = m.copy()
    for _ in range(r):
        p = np.pad(out, 1)
        acc = np.zeros_like(out)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                acc |= p[1 + dy:1 + dy + out.shape[0], 1 + dx:1 + dx + out.shape[1]]
        out = acc
    return out


def compare(g: dict, o: dict, diam: float, gutter: int = 2, sample=None, asset=None, query="ray") -> dict:
    """Statistics of the comparison; ``check`` asserts them.  With ``asset``,
    texels where two triangles lie within rounding of the closest answer
    (oracle flag 8, values otherwise not compared) are checked against the
    set of correct answers: the oracle evaluates the GPU's own triangle in
    FP64, which must lie under the ray (or be as near as the closest point),
    and the GPU's normal and displacement must be that triangle's."""
    H, W = o["face"].shape
    st = {}
    st["face_equal"] = bool(np.array_equal(g["face"], o["face"]))
    ray = o["face"] >= 0
    if sample is not None:
        sel = np.zeros(H * W, bool)
        sel[np.asarray(sample)] = True
        sel = sel.reshape(H, W) & ray
    else:
        sel = ray
    st["n_ray"] = int(ray.sum())
    st["n_compared"] = int(sel.sum())
    st["bary_max"] = float(np.abs(g["bary"][ray] - o["bary"][ray]).max()) if ray.any() else 0.0
    flags = o["flags"]
    exc = (flags & 0b1111) != 0
    gm, om = g["mask"].astype(bool), o["mask"].astype(bool)
    mism = sel & (gm != om)
    st["n_except"] = int((sel & exc).sum())
    st["mask_mismatch"] = int(mism.sum())
    st["mask_mismatch_unexcused"] = int((mism & ~exc).sum())
    same = sel & (gm == om) & ((flags & 0b1000) == 0)
    dn = np.abs(g["normal_ts"] - o["nts"])
    st["nts_max"] = float(dn[same].max()) if same.any() else 0.0
    dd = np.abs(g["disp_f32"] - o["disp"])
    st["disp_max_rel"] = float(dd[same].max() / diam) if same.any() else 0.0
    ht = g["hit_tri"] == o["hit_tri"]
    st["hit_tri_equal_frac"] = float(ht[same & om].mean()) if (same & om).any() else 1.0
    # ambiguous closest answers: |displacement| is unique even there
    amb = sel & gm & om & ((flags & 0b1000) != 0)
    st["n_amb"] = int(amb.sum())
    st["amb_absdisp_max_rel"] = float(np.abs(np.abs(g["disp_f32"][amb]) - np.abs(o["disp"][amb])).max() / diam) \
        if amb.any() else 0.0
    if asset is not None and amb.any():
        import oracle
        tex = np.flatnonzero(amb.reshape(-1))
        tris = g["hit_tri"].reshape(-1)[tex]
        nts_f, t_f, b_f, valid = oracle.shade_given(asset, tex, tris, query)
        st["amb_given_valid"] = bool(valid.all() and (tris >= 0).all())
        st["amb_bary_min"] = float(b_f.min()) if len(tex) else 0.0
        # the GPU's triangle is as close as the closest one, up to the displacement tolerance
        st["amb_excess_rel"] = float((np.abs(t_f) - np.abs(o["disp"].reshape(-1)[tex])).max() / diam)
        st["amb_nts_max"] = float(np.abs(g["normal_ts"].reshape(-1, 3)[tex] - nts_f).max())
        gd = g["disp_f32"].reshape(-1)[tex]
        # closest-point query: the sign of a distance at right angles to the
        # texel normal is a rounding decision, so its magnitude is compared
        dd_f = np.abs(gd - t_f) if query == "ray" else np.abs(np.abs(gd) - np.abs(t_f))
        st["amb_disp_max_rel"] = float(dd_f.max() / diam)
    # encoded maps: texels whose value legitimately differs (mask mismatch or
    # ambiguous closest hit) and, for dilated texels, their neighbourhoods
    bad = mism | (sel & ((flags & 0b1000) != 0))
    if sample is None:
        excl = _dilate_ring(bad, gutter) & ~ray | bad
        filled = o["filled"] > 0
        dil = (o["filled"] == 2) & ~excl
        st["dil_nts_max"] = float(dn[dil].max()) if dil.any() else 0.0
        st["dil_disp_max_rel"] = float(dd[dil].max() / diam) if dil.any() else 0.0
        region = ~excl
        st["alpha_equal"] = bool(np.array_equal(g["normal_rgba8"][..., 3], o["rgba8"][..., 3]))
        st["filled_equal"] = bool(np.array_equal(g["normal_rgba8"][..., 3] == 255, filled))
    else:
        region = sel & ~bad
    d8 = np.abs(g["normal_rgba8"][..., :3].astype(np.int32) - o["rgba8"][..., :3].astype(np.int32))
    diff_tex = (d8.max(-1) > 0) & region
    st["rgba_max"] = int(d8[region].max()) if region.any() else 0
    st["rgba_diff_texels"] = int(diff_tex.sum())
    st["rgba_region"] = int(region.sum())
    st["rgba_diff_frac"] = float(diff_tex.sum() / max(1, region.sum()))
    g16 = g["disp"].astype(np.float64)
    o16 = o["disp16"].astype(np.float64)
    ulp = np.spacing(np.abs(o16).astype(np.float16)).astype(np.float64)
    dd16 = np.abs(g16 - o16)
    st["disp16_max_ulps"] = float((dd16[region] / np.maximum(ulp[region], 1e-30)).max()) if region.any() else 0.0
    return st


def allowed_code_flips(region: int, rgba_frac=RGBA_FRAC, small=100_000) -> float:
    """The 8-bit bar is a rate (at most 0.01% of texels one code off).  On a
    map of fewer than `small` texels the expected count is below ten and its
    Poisson noise dominates, so the count may reach the rate plus three
    standard deviations there."""
    lam = rgba_frac * region
    if region >= small:
        return lam
    return max(1.0, lam + 3.0 * lam ** 0.5)


def check(st: dict, *, rgba_frac=RGBA_FRAC, small=100_000):
    assert st["face_equal"], "raster face map differs"
    skipped = st["mask_mismatch"]
    assert skipped <= max(3, SKIP_FRAC * st["n_compared"]), \
        f"{skipped} of {st['n_compared']} texels have a hit on one side only"
    assert st["amb_absdisp_max_rel"] <= TOL_DISP_REL, f"|displacement| off by {st['amb_absdisp_max_rel']} on ambiguous texels"
    if "amb_given_valid" in st:
        assert st["amb_given_valid"], "the GPU's triangle on an ambiguous texel is not hit by the ray"
        assert st["amb_bary_min"] >= -BARY_SLACK, f"the GPU's triangle lies {st['amb_bary_min']} outside the ray"
        assert st["amb_excess_rel"] <= TOL_DISP_REL, f"the GPU's triangle is {st['amb_excess_rel']} of diam farther"
        assert st["amb_nts_max"] <= TOL_NTS, f"normal off by {st['amb_nts_max']} from the GPU triangle's own"
        assert st["amb_disp_max_rel"] <= TOL_DISP_REL, f"displacement off by {st['amb_disp_max_rel']} from its triangle's"
    assert st["bary_max"] < 2e-6, f"raster barycentrics off by {st['bary_max']}"
    assert st["mask_mismatch_unexcused"] == 0, f"{st['mask_mismatch_unexcused']} hit-mask mismatches outside the exceptions"
    assert st["nts_max"] <= TOL_NTS, f"tangent-space normal off by {st['nts_max']}"
    assert st["disp_max_rel"] <= TOL_DISP_REL, f"displacement off by {st['disp_max_rel']} of diam"
    if "dil_nts_max" in st:
        assert st["dil_nts_max"] <= TOL_NTS, f"dilated normal off by {st['dil_nts_max']}"
        assert st["dil_disp_max_rel"] <= TOL_DISP_REL, f"dilated displacement off by {st['dil_disp_max_rel']}"
    assert st["rgba_max"] <= 1, f"8-bit map off by {st['rgba_max']} codes"
    allowed = allowed_code_flips(st["rgba_region"], rgba_frac, small)
    assert st["rgba_diff_texels"] <= allowed, f"{st['rgba_diff_texels']} texels off by one code (allowed {allowed})"
    assert st["disp16_max_ulps"] <= 1.0, f"fp16 displacement off by {st['disp16_max_ulps']} ulp"
