"""Edge cases at the limits of the ABI: the largest hypothesis count (4096) gives, for its first
hypotheses, the oracle's hypotheses and try indices bit for bit (each hypothesis draws from its
own Philox stream, so a prefix of a larger K is a smaller K), and a batch of one 4096-hypothesis
attempt equals the single-attempt call; a large view with ragged sides (1283 x 961: tiles, forest
slots and compaction chunks all cut by the edge) matches the oracle's raycast on sampled pixels
and its forest leaves on every pixel, inside a batch."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def u16_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(DEV)


@pytest.fixture(scope="module")
def gpu(room, room_forest):
    _, blocks = room
    return (B.Scene(blocks, 16),
            B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10))


def test_the_largest_hypothesis_count(room, oracle_room, room_forest, room_training, gpu):
    scene, forest = gpu
    world, _ = room
    intr = synth.Intrinsics.for_size(160, 120)
    P = synth.query_poses(world, [f[1] for f in room_training], 1, seed=8)[0]
    d, c = oracle_room.raycast(intr, P)
    leaves = oracle.forest_eval(room_forest.nodes, d, c)
    K, k0 = 4096, 96
    prm = B.ransac_params(n_hyps=K, batch=128, seed=4, max_tries=4000)
    poses = torch.zeros((K, 12), dtype=torch.float64, device=DEV)
    valid = torch.zeros(K, dtype=torch.int32, device=DEV)
    tries = torch.zeros(K, dtype=torch.int32, device=DEV)
    ws = torch.empty(B.ransac_workspace_size(intr.width, intr.height, prm), dtype=torch.uint8, device=DEV)
    B.ransac_hypotheses(forest, u16_dev(d), u16_dev(leaves), intr, prm, ws, poses, valid, tries)
    torch.cuda.synchronize()
    po, ok, tr = oracle.generate_hypotheses(d, intr, leaves, room_forest,
                                            oracle.RansacParams(n_hyps=k0, batch=128, seed=4, max_tries=4000))
    assert np.array_equal(valid.cpu().numpy()[:k0].astype(bool), ok)
    assert np.array_equal(tries.cpu().numpy()[:k0], tr)
    assert np.abs(poses.cpu().numpy().reshape(K, 3, 4)[:k0][ok] - po[ok, :3, :]).max() < 1e-9
    assert valid.cpu().numpy().sum() > K // 8
    # the batch path with the same attempt (its RANSAC seed is the attempt's seed)
    item = dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=P, n_hyps=K, seed=4)
    att = B.make_attempts([item])
    wsb = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    got = B.relocalise_batch(att, prm, wsb)[0]
    res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    depth = torch.zeros((120, 160), dtype=torch.int16, device=DEV)
    rgba = torch.zeros((120, 160, 4), dtype=torch.uint8, device=DEV)
    B.raycast_view(scene, intr, P, depth, rgba)
    lv = torch.zeros((5, 120, 160), dtype=torch.int16, device=DEV)
    B.forest_eval(forest, depth, rgba, lv)
    B.ransac_relocalise(forest, depth, lv, intr, prm, ws, res)
    B.verify(scene, intr, depth, res)
    torch.cuda.synchronize()
    one = B.result_from_bytes(res)
    for k in ("hypothesis", "status", "n_inliers", "n_valid", "n_rounds", "omega_a", "omega_ab", "verified"):
        assert got[k] == one[k], k
    assert got["n_rounds"] == 12 and np.array_equal(got["pose"], one["pose"])


def test_a_large_ragged_view_inside_a_batch(room, oracle_room, room_forest, room_training, gpu):
    scene, forest = gpu
    world, _ = room
    W, H = 1283, 961
    intr = synth.Intrinsics.for_size(W, H)
    P = synth.query_poses(world, [f[1] for f in room_training], 1, seed=12)[0]
    item = dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=P, n_hyps=64, seed=1)
    prm = B.ransac_params(n_hyps=64, batch=256, max_tries=3000)
    att = B.make_attempts([item])
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    bt = B.Batch(att, prm, ws)
    out = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.run(out)
    torch.cuda.synchronize()
    depth, rgba, leaves = bt.attempt_images(0, W, H, trees=5)
    d = depth.cpu().numpy().view(np.uint16)
    c = rgba.cpu().numpy()
    # raycast on sampled pixels, the right and bottom edges included
    rng = np.random.default_rng(5)
    px = np.concatenate([rng.choice(W * H, 4000, replace=False),
                         np.arange(H) * W + (W - 1), (H - 1) * W + np.arange(W)])
    do, co = oracle_room.raycast(intr, P, pixels=px)
    dg = d.reshape(-1)[px]
    both = (dg > 0) & (do > 0)
    assert np.mean((dg > 0) != (do > 0)) <= 1e-3
    assert np.mean(np.abs(dg[both].astype(int) - do[both]) <= 1) >= 0.999
    # forest leaves on the batch's own image, every pixel
    lo = oracle.forest_eval(room_forest.nodes, d, c)
    assert np.array_equal(leaves.cpu().numpy().view(np.uint16), lo)
    r = B.result_from_bytes(out)
    assert r["status"] == B.OK and r["n_valid"] == int((d > 0).sum())
