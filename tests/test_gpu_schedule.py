"""Launch schedules and the autotuner (relo_batch_set_schedule / relo_batch_autotune): every value
of every schedule field gives the same results, query images and forest leaves bit for bit as the
default schedule, on a batch of forest and learned attempts with ragged image sizes (tiles cut by
the image edge); the autotuner returns a valid schedule, and a graph captured under it replays
the same results; invalid schedules are rejected."""
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
SIZES = [(200, 152), (150, 101), (96, 72), (320, 240)]
VALUES = {"ray_warp_width": [2, 4, 8, 16], "forest_threads": [128, 256], "forest_tiles": [0, 1],
          "search_ctas_per_sm": [0, 1, 2, 3], "refit_per": [0, 1, 4, 16, 32], "persistent": [0, 1],
          "forest_smem_levels": [0, 1, 4, 6, 8, 10]}


@pytest.fixture(scope="module")
def batch(room, room_training, room_forest):
    world, blocks = room
    scene = B.Scene(blocks, 16)
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    reg = B.Regressor(seed=9, origin=(2.0, 2.0, 1.5))
    train = [f[1] for f in room_training]
    qs = synth.query_poses(world, train, len(SIZES) + 2, seed=91)
    items = []
    for i, (W, H) in enumerate(SIZES):
        items.append(dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=synth.Intrinsics.for_size(W, H),
                          pose_b=qs[i], n_hyps=[64, 40, 17, 128][i], seed=500 + i))
    for i in range(2):  # learned attempts with the forest as fallback, one shared size
        items.append(dict(scene_b=scene, forest_a=forest, scene_a=scene, regressor_a=reg,
                          intr=synth.Intrinsics.for_size(160, 120), pose_b=qs[len(SIZES) + i], seed=600 + i))
    prm = B.ransac_params(n_hyps=64, batch=100, max_tries=3000)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    bt = B.Batch(att, prm, ws)
    keep = (scene, forest, reg, ws)
    return bt, items, keep


def _run(bt, items):
    out = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.run(out)
    torch.cuda.synchronize()
    imgs = []
    for k, it in enumerate(items):
        intr = it["intr"]
        d, c, lv = bt.attempt_images(k, intr.width, intr.height, trees=5)
        imgs.append((d.clone(), c.clone(), None if lv is None else lv.clone()))
    return out.cpu(), imgs


def _equal(a, b):
    assert torch.equal(a[0], b[0])
    for (d0, c0, l0), (d1, c1, l1) in zip(a[1], b[1]):
        assert torch.equal(d0, d1) and torch.equal(c0, c1)
        assert (l0 is None) == (l1 is None)
        if l0 is not None:
            assert torch.equal(l0, l1)


def test_every_schedule_value_gives_the_default_results(batch):
    bt, items, _ = batch
    default = bt.schedule()
    assert default == {"ray_warp_width": 8, "forest_threads": 256, "forest_tiles": 0, "search_ctas_per_sm": 0,
                       "refit_per": 0, "persistent": 0, "forest_smem_levels": 0}
    ref = _run(bt, items)
    assert sum(B.result_from_bytes(ref[0][k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES])["status"] == 0
               for k in range(len(items))) >= 3
    for field, values in VALUES.items():
        for v in values:
            bt.set_schedule(**{**default, field: v})
            _equal(_run(bt, items), ref)
    bt.set_schedule(ray_warp_width=16, forest_threads=128, forest_tiles=1, search_ctas_per_sm=1, refit_per=32,
                    persistent=1, forest_smem_levels=7)
    _equal(_run(bt, items), ref)
    bt.set_schedule(**default)


def test_autotuned_schedule_replays_the_same_results(batch):
    bt, items, _ = batch
    ref = _run(bt, items)
    chosen = bt.autotune(repeats=1)
    assert chosen == bt.schedule()
    for field, values in VALUES.items():
        assert chosen[field] in values, field
    _equal(_run(bt, items), ref)
    out = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.capture(out)
    bt.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), ref[0])


def test_invalid_schedules_are_rejected(batch):
    bt, _, _ = batch
    before = bt.schedule()
    for bad in (dict(ray_warp_width=3), dict(ray_warp_width=32), dict(forest_threads=64), dict(forest_tiles=2),
                dict(search_ctas_per_sm=-1), dict(refit_per=33), dict(persistent=2), dict(forest_smem_levels=-1),
                dict(forest_smem_levels=11)):
        with pytest.raises(B.ReloError):
            bt.set_schedule(**bad)
    assert bt.schedule() == before
