"""The serving runtime (relo_server_*): attempts submitted one at a time from several threads,
batched by the worker, give exactly the results of the same attempts run alone; a full request
pool discards new requests (the pooled queue's discard policy, Appendix B.1); a request whose
workspace exceeds the server's budget completes with RELO_EINVAL; the latency statistics are
consistent."""
import threading

import numpy as np
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def setup(room, room_training, room_forest):
    world, blocks = room
    scene = B.Scene(blocks, 16)
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    intr = synth.Intrinsics.for_size(160, 120)
    qs = synth.query_poses(world, [f[1] for f in room_training], 24, seed=71)
    items = [dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=P, seed=300 + i, n_hyps=64)
             for i, P in enumerate(qs)]
    prm = B.ransac_params(n_hyps=64, batch=100, max_tries=4000)
    return scene, forest, items, prm


def _alone(item, prm):
    att = B.make_attempts([item])
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    return B.relocalise_batch(att, prm, ws)[0]


def _same(a, b):
    for k in ("hypothesis", "status", "omega", "omega_a", "omega_ab", "sum_absdiff_mm", "verified", "tries", "path"):
        assert a[k] == b[k], k
    assert np.array_equal(a["pose"], b["pose"])


def test_threads_submit_and_results_equal_single_runs(setup):
    _, _, items, prm = setup
    att = B.make_attempts(items)
    one = B.batch_workspace_size(B.make_attempts(items[:1]), prm)
    srv = B.Server(prm, workspace_bytes=16 * one + (1 << 20), max_batch=8, max_wait_us=3000, slots=64)
    out = {}

    def agent(ids):
        for k in ids:
            t = srv.submit(att[k])
            out[k] = srv.wait(t)

    threads = [threading.Thread(target=agent, args=(list(range(a, len(items), 4)),)) for a in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    st = srv.stats()
    srv.close()
    assert sorted(out) == list(range(len(items)))
    for k, it in enumerate(items):
        _same(out[k][0], _alone(it, prm))
        assert out[k][1] > 0
    assert st["completed"] == len(items) and st["discarded"] == 0
    assert st["batches"] >= len(items) / 8 and 1 <= st["mean_batch"] <= 8
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_full_pool_discards_new_requests(setup):
    _, _, items, prm = setup
    att = B.make_attempts(items[:4])
    one = B.batch_workspace_size(B.make_attempts(items[:1]), prm)
    # the worker waits up to 0.3 s for a batch of 8, so both slots stay taken while we submit
    srv = B.Server(prm, workspace_bytes=8 * one + (1 << 20), max_batch=8, max_wait_us=300000, slots=2)
    t0, t1 = srv.submit(att[0]), srv.submit(att[1])
    for k in (2, 3):
        with pytest.raises(B.ReloError) as e:
            srv.submit(att[k])
        assert e.value.status == B.EBUSY
    r0, r1 = srv.wait(t0)[0], srv.wait(t1)[0]
    st = srv.stats()
    srv.close()
    _same(r0, _alone(items[0], prm))
    _same(r1, _alone(items[1], prm))
    assert st["discarded"] == 2 and st["completed"] == 2


def test_request_beyond_the_budget_completes_with_einval(setup):
    _, _, items, prm = setup
    att = B.make_attempts(items[:1])
    srv = B.Server(prm, workspace_bytes=4096, max_batch=4, max_wait_us=100, slots=4)
    r, _ = srv.wait(srv.submit(att[0]))
    srv.close()
    assert r["status"] == B.EINVAL
    with pytest.raises(B.ReloError):
        srv2 = B.Server(prm, workspace_bytes=0)
