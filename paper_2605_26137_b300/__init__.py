"""B300-native tangent-space normal baker (AssetGen, Sec. 6.4, normal-map baking),
with the hidden-face removal pass of Sec. 6.2 on the same BVH and the QEM
simplification of Sec. 6.1.

The compute path is the CUDA library ``libagbake.so`` behind the C ABI of
``include/ag.h``; this package only marshals torch tensors into it.
"""
import importlib

from ._lib import EXPORTS, AgError, load as load_library  # noqa: F401

_TORCH_API = ("Bvh", "BakeOutputs", "Asset", "BatchPlan", "BakeLoss", "bake", "bake_batch", "bake_backward",
              "bake_loss", "alloc_outputs", "sync_status", "visibility", "exterior_fill", "hidden_faces", "qem_simplify",
              "point_distance", "render_views", "backproject", "normal_map_error")


def __getattr__(name):
    # torch-facing API, imported lazily so that host-only users (tests of the
    # ABI, the input generators) do not import torch
    if name in _TORCH_API:
        return getattr(importlib.import_module(".torch_api", __name__), name)
    raise AttributeError(name)
