"""Error paths, with every failure made on the host or caught by a bounded loop (nothing here
faults, traps or hangs the GPU): injected allocation failures make every creation call return
RELO_ENOMEM and the next call succeeds; a scene whose hash chains were turned into cycles makes
the attempts that raycast it report RELO_EDEVICE, and the context stays usable; a forest with
empty leaves finds no hypothesis (RELO_ENOTFOUND); non-finite poses are rejected on the host."""
import numpy as np
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(autouse=True)
def _no_leftover_injection():
    yield
    B.debug_fail_allocations(0)


def _raises_enomem(make):
    B.debug_fail_allocations(1)
    with pytest.raises(B.ReloError) as e:
        make()
    assert e.value.status == B.ENOMEM
    return make()          # the injection is used up: the same call succeeds


def test_injected_allocation_failures(room, room_forest):
    _, blocks = room
    assert _raises_enomem(lambda: B.Scene(blocks, 16)).handle
    assert _raises_enomem(lambda: B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes,
                                           max_modes=10)).handle
    assert _raises_enomem(lambda: B.FusionScene(256, synth.VOXEL_SIZE, synth.TRUNCATION, log2_buckets=8)).handle
    assert _raises_enomem(lambda: B.Regressor(seed=1)).handle
    prm = B.ransac_params(n_hyps=16, batch=32)
    srv = _raises_enomem(lambda: B.Server(prm, workspace_bytes=1 << 20, max_batch=2, slots=2))
    srv.close()


def _attempts(room, room_training, scene, forest, n=3, **over):
    world, _ = room
    intr = synth.Intrinsics.for_size(96, 72)
    qs = synth.query_poses(world, [f[1] for f in room_training], n, seed=77)
    items = [dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=P, seed=40 + i, **over)
             for i, P in enumerate(qs)]
    prm = B.ransac_params(n_hyps=32, batch=64, max_tries=2000)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    return B.relocalise_batch(att, prm, ws)


def test_corrupted_hash_chains_report_edevice(room, room_training, room_forest):
    _, blocks = room
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    good = B.Scene(blocks, 16)
    ok = _attempts(room, room_training, good, forest)
    assert all(r["status"] == B.OK for r in ok)
    bad = B.Scene(blocks, 16)
    bad.use_grid(False)                     # raycasts walk the hash
    B.debug_corrupt_scene(bad)
    res = _attempts(room, room_training, bad, forest)
    assert all(r["status"] == B.EDEVICE and r["verified"] == 0 for r in res)
    # the context is still usable: the intact scene gives the same results as before
    again = _attempts(room, room_training, good, forest)
    for a, b in zip(ok, again):
        assert a["hypothesis"] == b["hypothesis"] and np.array_equal(a["pose"], b["pose"])


def test_empty_leaves_find_no_hypothesis(room, room_training, room_forest):
    _, blocks = room
    scene = B.Scene(blocks, 16)
    empty = B.Forest(room_forest.nodes, max_modes=10)      # no modes: every leaf is empty
    res = _attempts(room, room_training, scene, empty)
    assert all(r["status"] == B.ENOTFOUND and r["verified"] == 0 and r["n_valid"] > 0 for r in res)


def test_non_finite_poses_are_rejected_on_the_host(room, room_training, room_forest):
    _, blocks = room
    scene = B.Scene(blocks, 16)
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    intr = synth.Intrinsics.for_size(32, 24)
    P = np.eye(4)
    P[1, 3] = np.nan
    depth = torch.zeros((24, 32), dtype=torch.int16, device=DEV)
    for call in (lambda: B.raycast_view(scene, intr, P, depth),
                 lambda: B.render_global([scene], [np.eye(4)], intr, P, depth),
                 lambda: B.render_global([scene], [P], intr, np.eye(4), depth),
                 lambda: B.FusionScene(64, synth.VOXEL_SIZE, synth.TRUNCATION, log2_buckets=8).fuse(intr, P, depth)):
        with pytest.raises(B.ReloError) as e:
            call()
        assert e.value.status == B.EINVAL
    Q = np.eye(4)
    Q[0, 0] = np.inf
    item = dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=Q)
    prm = B.ransac_params(n_hyps=8, batch=16)
    att = B.make_attempts([item])
    assert B.batch_workspace_size(att, prm) == 0
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.ReloError) as e:
        B.relocalise_batch(att, prm, ws)
    assert e.value.status == B.EINVAL
