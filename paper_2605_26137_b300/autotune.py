"""Autotuner front end.

The measurement is native (ag_autotune times whole bakes of the caller's
asset for every schedule x block size x ray tile on the GPU); this module
persists the choice in a JSON cache keyed by GPU name, BVH layout and
power-of-two buckets of the atlas texel count and the high-mesh triangle
count, so later bakes of similar assets reuse it without timing.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import tempfile

import torch

from . import _lib
from ._lib import check

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "agbake", "autotune.json")


def cache_path() -> str:
    return os.environ.get("AGBAKE_AUTOTUNE_CACHE", DEFAULT_CACHE)


def bucket_key(bvh, W: int, H: int, query: str = "ray") -> str:
    info = bvh.info()
    layout = "q8" if info["layout"] == _lib.AG_BVH_Q8 else "f32"
    q = "" if query == "ray" else f"|{query}"
    return (f"{torch.cuda.get_device_name()}|{layout}|texels~2^{round(math.log2(max(1, W * H)))}"
            f"|tris~2^{round(math.log2(max(1, info['n_tris'])))}{q}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(bvh, low_verts, low_faces, low_uv, W: int, H: int, max_dist: float, *, low_normals=None,
         force: bool = False, path: str | None = None, stream=None, query: str = "ray") -> dict:
    """Launch configuration for bake()/BatchPlan: {"schedule", "block_size",
    "blocks_per_sm", "ray_tile", "ms", "cached"}, for the given query
    ("ray" or "closest")."""
    from .torch_api import _QUERY, _check_low, _ptr, _stream
    path = path or cache_path()
    key = bucket_key(bvh, W, H, query)
    data = _load(path)
    if key in data and not force:
        return dict(data[key], cached=True)
    _check_low(low_verts, low_faces, low_uv, low_normals)
    lib = _lib.load()
    o = _lib.default_opts(query=_QUERY[query])
    best = ctypes.c_float()
    check(lib.ag_autotune(bvh.handle, low_verts.data_ptr(), _ptr(low_normals), low_uv.data_ptr(),
                          low_faces.data_ptr(), low_verts.shape[0], low_faces.shape[0], W, H, float(max_dist),
                          _stream(stream), ctypes.byref(o), ctypes.byref(best)))
    entry = {"schedule": int(o.schedule), "block_size": int(o.block_size), "blocks_per_sm": int(o.blocks_per_sm),
             "ray_tile": int(o.ray_tile), "ms": float(best.value)}
    data[key] = entry
    try:
        _store(path, data)
    except OSError:
        pass  # a read-only cache location only costs a re-tune next time
    return dict(entry, cached=False)


def launch_kwargs(entry: dict) -> dict:
    return {k: entry[k] for k in ("schedule", "block_size", "blocks_per_sm", "ray_tile")}
