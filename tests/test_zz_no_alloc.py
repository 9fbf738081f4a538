"""The allocation-free RANSAC entry point (relo_ransac_relocalise_noalloc) against the
workspace one.

Some callers cannot allocate device memory while they relocalise (their memory belongs to
another allocator, or an allocation could stall a latency-bound loop), so the library offers a
variant whose scratch is a fixed array inside the library.  This file is collected last so
that a run stopping at the first failure has already run every other test; it also passes on
its own in a fresh process.  Both entry points run the same kernels on the same inputs, so every
call must give the workspace entry point's result byte for byte.  The calls run in a row with
changing sizes -- a small view, a larger hypothesis count, a 640 x 480 view with 1024 hypotheses
(the largest the header says fits), then the first view again -- which also shows that no call
is disturbed by what the previous one left in the shared array."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(DEV)


def _views(room, oracle_room, room_forest, room_training, sizes):
    world, _ = room
    out = []
    for k, (W, H) in enumerate(sizes):
        intr = synth.Intrinsics.for_size(W, H)
        P = synth.query_poses(world, [f[1] for f in room_training], len(sizes), seed=77)[k]
        d, c = oracle_room.raycast(intr, P)
        out.append((intr, d, oracle.forest_eval(room_forest.nodes, d, c)))
    return out


def test_noalloc_matches_workspace_entry_point(room, oracle_room, room_forest, room_training):
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    small, large = _views(room, oracle_room, room_forest, room_training, [(320, 240), (640, 480)])
    calls = [(small, dict(n_hyps=64, batch=200, seed=5)),
             (small, dict(n_hyps=96, batch=300, seed=6)),
             (large, dict(n_hyps=1024, batch=64, seed=7)),
             (small, dict(n_hyps=64, batch=200, seed=5))]
    for call, ((intr, d, leaves), kw) in enumerate(calls):    # calls in a row on the shared array
        prm = B.ransac_params(**kw)
        dd, ld = _u16(d), _u16(leaves)
        got = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        want = torch.zeros_like(got)
        B.ransac_relocalise_noalloc(forest, dd, ld, intr, prm, got)
        ws = torch.empty(B.ransac_workspace_size(intr.width, intr.height, prm), dtype=torch.uint8, device=DEV)
        B.ransac_relocalise(forest, dd, ld, intr, prm, ws, want)
        torch.cuda.synchronize()
        g, w = B.result_from_bytes(got), B.result_from_bytes(want)
        assert w["status"] == B.OK and w["n_valid"] > 0, call
        assert torch.equal(got, want), (call, g, w)


def test_noalloc_rejects_views_beyond_its_scratch(room_forest):
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    intr = synth.Intrinsics.for_size(2048, 2048)
    prm = B.ransac_params(n_hyps=64, batch=64)
    d = torch.zeros((16, 16), dtype=torch.int16, device=DEV)
    res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.ReloError) as e:
        B.ransac_relocalise_noalloc(forest, d, d, intr, prm, res)
    assert e.value.status == B.EINVAL and "static scratch" in str(e.value)
