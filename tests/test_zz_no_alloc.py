"""The allocation-free RANSAC entry point (relo_ransac_relocalise_noalloc) against the
workspace one.

Some callers cannot allocate device memory while they relocalise (their memory belongs to
another allocator, or an allocation could stall a latency-bound loop), so the library offers a
variant whose scratch is a fixed array inside the library.  This file is collected last so
that a run stopping at the first failure has already run every other test; it also passes on
its own in a fresh process.  Two calls in a row must each match relo_ransac_relocalise on the
same inputs (the library's RANSAC tolerances: poses 1e-4, energies 1e-5 relative; integer
fields exact), which also shows that the second call is not disturbed by what the first left
in the shared array."""
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


def _views(room, oracle_room, room_forest, room_training, n):
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    poses = synth.query_poses(world, [f[1] for f in room_training], n, seed=77)
    out = []
    for P in poses:
        d, c = oracle_room.raycast(intr, P)
        out.append((intr, d, oracle.forest_eval(room_forest.nodes, d, c)))
    return out


def test_noalloc_matches_workspace_entry_point(room, oracle_room, room_forest, room_training):
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    views = _views(room, oracle_room, room_forest, room_training, 2)
    for call, (intr, d, leaves) in enumerate(views):       # two calls in a row
        prm = B.ransac_params(n_hyps=64 + 32 * call, batch=200 + 100 * call, seed=5 + call)
        dd, ld = _u16(d), _u16(leaves)
        got = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        want = torch.zeros_like(got)
        B.ransac_relocalise_noalloc(forest, dd, ld, intr, prm, got)
        ws = torch.empty(B.ransac_workspace_size(intr.width, intr.height, prm), dtype=torch.uint8, device=DEV)
        B.ransac_relocalise(forest, dd, ld, intr, prm, ws, want)
        torch.cuda.synchronize()
        g, w = B.result_from_bytes(got), B.result_from_bytes(want)
        assert g["status"] == w["status"] == B.OK
        for k in ("hypothesis", "n_inliers", "n_valid", "n_rounds", "tries"):
            assert g[k] == w[k], k
        assert np.abs(g["pose"] - w["pose"]).max() <= 1e-4
        assert abs(g["energy"] - w["energy"]) <= 1e-5 * abs(w["energy"])


def test_noalloc_rejects_views_beyond_its_scratch(room_forest):
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    intr = synth.Intrinsics.for_size(2048, 2048)
    prm = B.ransac_params(n_hyps=64, batch=64)
    d = torch.zeros((16, 16), dtype=torch.int16, device=DEV)
    res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.ReloError) as e:
        B.ransac_relocalise_noalloc(forest, d, d, intr, prm, res)
    assert e.value.status == B.EINVAL and "static scratch" in str(e.value)
