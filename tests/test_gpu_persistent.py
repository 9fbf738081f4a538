"""Bounded waits of the persistent RANSAC launch: a batch prepared with one item waiting for a
counter that never reaches its target (relo_debug_persistent_stall) stops within its time limit
instead of hanging; the attempts it did not finish report RELO_ETIMEOUT and are left unverified;
afterwards the context is usable and a batch prepared without the stall gives the per-stage
launches' results bit for bit.  The failure is made on the host (the item table), no GPU fault."""
import time

import numpy as np
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def room_batch_items(room, room_forest, room_training):
    world, blocks = room
    scene = B.Scene(blocks, 16)
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    intr = synth.Intrinsics.for_size(160, 120)
    qs = synth.query_poses(world, [f[1] for f in room_training], 6, seed=31)
    items = [dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=P, n_hyps=64 + 32 * (k % 3),
                  seed=k) for k, P in enumerate(qs)]
    return items, scene, forest


def _run(items, persistent):
    prm = B.ransac_params(n_hyps=64, batch=100, max_tries=2000)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    bt = B.Batch(att, prm, ws)
    bt.set_schedule(persistent=1 if persistent else 0)
    res = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.run(res)
    torch.cuda.synchronize()
    return res.cpu().numpy()


def test_stalled_persistent_launch_reports_timeout(room_batch_items):
    items = room_batch_items[0]
    want = _run(items, persistent=False)
    B.debug_persistent_stall(True, 50)
    try:
        t0 = time.perf_counter()
        got = _run(items, persistent=True)
        elapsed = time.perf_counter() - t0
    finally:
        B.debug_persistent_stall(False, 0)
    assert elapsed < 10.0
    res = [B.result_from_bytes(got[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES]) for k in range(len(items))]
    assert res[0]["status"] == B.ETIMEOUT and res[0]["verified"] == 0
    for r in res:
        assert r["status"] in (B.OK, B.ENOTFOUND, B.ETIMEOUT)
        assert not (r["status"] == B.ETIMEOUT and r["verified"])
    # the context is usable and an unstalled batch gives the per-stage results
    assert np.array_equal(_run(items, persistent=True), want)
