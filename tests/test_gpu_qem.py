"""GPU parity of QEM simplification (Sec. 6.1) against the FP64 oracle through
the C ABI (ag_qem_simplify).  Both evaluate every quadric expression in FP64
with the same operation order and take the same decisions, so the simplified
meshes must be identical: the same surviving vertices with bit-identical
positions, the same faces, the same number of rounds."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_26137_b300 import synth

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_simplify(V, F, target, **kw):
    import paper_2605_26137_b300 as pb
    vo, fo, keep, rounds = pb.qem_simplify(_t(V), _t(F), target, **kw)
    pb.sync_status()
    return vo.cpu().numpy(), fo.cpu().numpy(), keep.cpu().numpy(), rounds


def assert_identical(V, F, target, **kw):
    o = oracle.qem_simplify(V, F, target, **({"max_rounds": kw["max_rounds"]} if "max_rounds" in kw else {}))
    vo, fo, keep, rounds = gpu_simplify(V, F, target, **kw)
    assert rounds == o["rounds"]
    assert np.array_equal(keep, o["keep_v"])
    assert np.array_equal(fo, o["F"])
    assert np.array_equal(vo.view(np.uint64), o["V"].view(np.uint64))
    return o


def _grid(n):
    xs = np.linspace(-1, 1, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), 0.1 * np.sin(3 * X.ravel()) * np.cos(2 * Y.ravel())], -1).astype(np.float32)
    F = []
    for j in range(n):
        for i in range(n):
            a = j * (n + 1) + i
            F += [(a, a + 1, a + n + 2), (a, a + n + 2, a + n + 1)]
    return V, np.asarray(F, np.int32)


CASES = {
    "icosphere": lambda: (*synth.icosphere(4), 500),
    "displaced_sphere": lambda: (*synth.sh_displaced_sphere(4, 3, amp=0.1), 1000),
    "open_wavy_grid": lambda: (*_grid(40), 600),
    "sdf_32k": lambda: (*synth.sdf_mesh(synth.sdf_union_params(3, 12), 48, device="cpu"), 4000),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_identical_to_oracle(name):
    V, F, target = CASES[name]()
    o = assert_identical(V, F, target)
    assert len(o["F"]) <= target


def test_round_limit_and_unreachable_target():
    V, F = synth.sh_displaced_sphere(3, 8, amp=0.1)
    assert_identical(V, F, 10, max_rounds=3)
    # a tetrahedron cannot be reduced: no round runs
    Vt = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    Ft = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32)
    vo, fo, keep, rounds = gpu_simplify(Vt, Ft, 2)
    assert rounds == 0 and len(fo) == 4 and len(vo) == 4


@pytest.mark.parametrize("max_rounds", [7, 8, 9, 16, 17, 41])
def test_round_caps_across_enqueued_batches(max_rounds):
    """The rounds are enqueued eight at a time and stop on the device: a cap
    that falls inside, at the end of, or just past a batch (and one well past
    the renumbering of the working mesh, when its alive faces fall to a
    quarter) leaves the same mesh and round count as the oracle."""
    V, F = synth.sdf_mesh(synth.sdf_union_params(3, 12), 48, device="cpu")
    assert_identical(V, F, 500, max_rounds=max_rounds)


def test_degenerate_input_faces_and_errors():
    import paper_2605_26137_b300 as pb
    V, F = synth.icosphere(3)
    G = np.concatenate([F, np.array([[0, 0, 5], [7, 8, 7]], np.int32)])   # repeated indices: dropped
    o = assert_identical(V, G, 300)
    assert len(o["F"]) == 300
    bad = F.copy()
    bad[3, 1] = len(V) + 2
    pb.qem_simplify(_t(V), _t(bad), 300)
    with pytest.raises(pb.AgError) as ei:
        pb.sync_status()
    assert ei.value.status == 1
    with pytest.raises(pb.AgError):
        pb.qem_simplify(_t(V), _t(F), -1)


@pytest.mark.slow
def test_identical_to_oracle_250k():
    """A marching-grid SDF surface of ~250k faces reduced to 10k faces: some
    200 rounds, every one identical."""
    V, F = synth.sdf_mesh(synth.sdf_union_params(5, 24), 128, device="cpu")
    assert len(F) > 150_000
    assert_identical(V, F, 10_000)


def test_midpoint_placement_identical_and_worse_than_optimal():
    """The baseline placement (every interior edge at its midpoint) through the
    same rounds: identical to the oracle's baseline; on a curved surface the
    paper's projected optimum keeps the vertices closer to the original."""
    V, F = synth.sdf_mesh(synth.sdf_union_params(3, 12), 48, device="cpu")
    o = oracle.qem_simplify(V, F, 4000, midpoint=True)
    vo, fo, keep, rounds = gpu_simplify(V, F, 4000, placement="midpoint")
    assert rounds == o["rounds"] and np.array_equal(fo, o["F"]) and np.array_equal(keep, o["keep_v"])
    assert np.array_equal(vo.view(np.uint64), o["V"].view(np.uint64))
    opt = oracle.qem_simplify(V, F, 4000)
    bvh = oracle.Bvh(V, F)
    diam = float(np.linalg.norm(V.max(0) - V.min(0)))

    def mean_dist(Vs):
        return np.mean([np.sqrt(oracle.closest_point(V, F, v, diam, bvh=bvh)[1]) for v in Vs])
    assert mean_dist(opt["V"]) < mean_dist(o["V"])
