"""Writes oracle_tiny_asset.txt: the FP64 oracle's bake of the seeded tiny
asset (a 320-face icosphere over a 5,120-face displaced sphere, 128^2 atlas).

Uses only the oracle and the seeded input generators. The stored values pin
the oracle against unintended change: any later change of its arithmetic must
regenerate this file and say, in its commit message, which passage of the
paper (or which reading of it) justifies the change.

    python tests/golden/make_oracle_regression.py
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2605_26137_b300 import synth  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main():
    a = synth.tiny_asset(1)
    r = oracle.bake_asset(a)
    face, rgba, mask = r["face"], r["rgba8"], r["mask"]
    ys, xs = np.nonzero(face >= 0)
    pick = np.random.default_rng(7).choice(len(ys), size=40, replace=False)
    lines = ["# Oracle bake of synth.tiny_asset(1): 128 x 128 atlas, max_dist 0.15, gutter 2.",
             "# Written by make_oracle_regression.py (oracle and seeded generators only).",
             f"face_map_sha256 {digest(face.astype(np.int32))}",
             f"rgba8_sha256 {digest(rgba.astype(np.uint8))}",
             f"mask_sha256 {digest(mask.astype(np.uint8))}",
             f"ray_texels {int((face >= 0).sum())}",
             f"hits {int(mask.sum())}",
             "# x y face nx ny nz disp (ray texels, %.17g)"]
    for i in sorted(pick):
        y, x = int(ys[i]), int(xs[i])
        n = r["nts"][y, x]
        lines.append(f"{x} {y} {int(face[y, x])} {n[0]:.17g} {n[1]:.17g} {n[2]:.17g} {r['disp'][y, x]:.17g}")
    with open(os.path.join(HERE, "oracle_tiny_asset.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
