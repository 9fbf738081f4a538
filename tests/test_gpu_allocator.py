"""relo_set_allocator: with a caller's allocator (torch's caching allocator behind a counting
wrapper) every device block of a scene, a forest and a regressor comes from it and goes back to it,
also after the allocator was reset; results equal those under cudaMalloc; an allocator that
fails, or returns a pointer that is not 256-byte aligned, makes creation return RELO_ENOMEM and
gets the pointer back."""
import gc

import numpy as np
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


class Counting:
    def __init__(self, shift=0):
        self.live, self.allocs, self.frees, self.shift = {}, 0, 0, shift

    def alloc(self, n):
        p = torch.cuda.caching_allocator_alloc(n + self.shift)
        self.live[p + self.shift] = (p, n)
        self.allocs += 1
        return p + self.shift

    def free(self, q):
        p, _ = self.live.pop(q)
        self.frees += 1
        torch.cuda.caching_allocator_delete(p)


@pytest.fixture(autouse=True)
def _default_allocator():
    yield
    B.set_allocator()


def _attempts(room, room_training, scene, forest):
    world, _ = room
    intr = synth.Intrinsics.for_size(96, 72)
    qs = synth.query_poses(world, [f[1] for f in room_training], 3, seed=31)
    items = [dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=P, seed=7 + i)
             for i, P in enumerate(qs)]
    prm = B.ransac_params(n_hyps=32, batch=64, max_tries=2000)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    return B.relocalise_batch(att, prm, ws)


def test_handles_live_in_the_callers_allocator(room, room_training, room_forest):
    _, blocks = room
    ref = _attempts(room, room_training, B.Scene(blocks, 16),
                    B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10))
    a = Counting()
    gc.collect()  # garbage of earlier tests may hold torch memory: free it before the baseline
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    B.set_allocator(a.alloc, a.free)
    scene = B.Scene(blocks, 16)
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    reg = B.Regressor(seed=3)
    held = sum(n for _, n in a.live.values())
    assert a.allocs >= 9 and held > 0
    assert torch.cuda.memory_allocated() - before >= held
    got = _attempts(room, room_training, scene, forest)
    for r, g in zip(ref, got):
        for k in ("status", "hypothesis", "n_inliers", "omega", "omega_a", "omega_ab", "verified"):
            assert r[k] == g[k], k
        assert np.array_equal(r["pose"], g["pose"])
    # back to cudaMalloc: the handles' blocks still go back to the counting allocator
    B.set_allocator()
    n = a.allocs
    other = B.Scene(blocks, 16)
    assert a.allocs == n
    del scene, forest, reg, other
    gc.collect()
    assert not a.live and a.frees == a.allocs


def test_a_failing_or_misaligned_allocator_gives_enomem(room, room_forest):
    _, blocks = room
    B.set_allocator(lambda n: 0, lambda p: None)
    with pytest.raises(B.ReloError) as e:
        B.Scene(blocks, 16)
    assert e.value.status == B.ENOMEM
    a = Counting(shift=16)
    B.set_allocator(a.alloc, a.free)
    with pytest.raises(B.ReloError) as e:
        B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    assert e.value.status == B.ENOMEM
    assert a.allocs == 1 and a.frees == 1 and not a.live
