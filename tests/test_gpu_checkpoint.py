"""Checkpoints (paper_1801_08361_gb300.checkpoint): a saved and reloaded forest gives the same
leaves and modes; a reloaded regressor continues training exactly like the original; a fused
scene saved through its export reloads as a static scene that raycasts like the fused one."""
import numpy as np
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import checkpoint as C
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _view(scene, intr, P):
    d = torch.zeros((intr.height, intr.width), dtype=torch.int16, device=DEV)
    c = torch.zeros((intr.height, intr.width, 4), dtype=torch.uint8, device=DEV)
    B.raycast_view(scene, intr, P, d, c)
    return d, c


def test_forest_round_trip(tmp_path, room, room_forest, room_training):
    world, blocks = room
    scene = B.Scene(blocks, 16)
    f1 = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    C.save_forest(tmp_path / "f.npz", room_forest.nodes, f1)
    nodes, f2 = C.load_forest(tmp_path / "f.npz")
    assert np.array_equal(nodes, room_forest.nodes)
    intr = synth.Intrinsics.for_size(160, 120)
    d, c = _view(scene, intr, room_training[0][1])
    out = []
    for f in (f1, f2):
        lv = torch.zeros((5, 120, 160), dtype=torch.int16, device=DEV)
        B.forest_eval(f, d, c, lv)
        out.append(lv.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    for a, b in zip(f1.get_modes(), f2.get_modes()):
        assert np.array_equal(a, b)


def test_regressor_round_trip_continues_training(tmp_path, room, oracle_room):
    world, _ = room
    intr = synth.Intrinsics.for_size(64, 48)
    poses = synth.training_poses(world, 4, seed=3)[:4]
    imgs = [oracle_room.raycast(intr, P) for P in poses]
    d = torch.from_numpy(np.stack([i[0] for i in imgs]).view(np.int16)).to(DEV)
    c = torch.from_numpy(np.stack([i[1] for i in imgs])).to(DEV)
    ws = torch.empty(B.regressor_workspace_size(4, 64, 48, True), dtype=torch.uint8, device=DEV)
    a = B.Regressor(seed=2, origin=(2.0, 2.0, 1.5))
    for _ in range(3):
        B.regressor_train_step(a, d, c, intr, poses, 1e-3, ws)
    C.save_regressor(tmp_path / "r.npz", a)
    b = C.load_regressor(tmp_path / "r.npz")
    assert b.origin == a.origin
    for reg in (a, b):
        for _ in range(2):
            B.regressor_train_step(reg, d, c, intr, poses, 1e-3, ws)
    torch.cuda.synchronize()
    assert np.array_equal(a.params().view(np.uint32), b.params().view(np.uint32))


def test_fused_scene_round_trip(tmp_path, room, room_training):
    world, blocks = room
    scene = B.Scene(blocks, 16)
    intr = synth.Intrinsics.for_size(160, 120)
    fs = B.FusionScene(1 << 16, synth.VOXEL_SIZE, synth.TRUNCATION, log2_buckets=14)
    for _, P, _, _ in room_training[:5]:
        d, c = _view(scene, intr, P)
        fs.fuse(intr, P, d, c)
    C.save_fused_scene(tmp_path / "s.npz", fs, synth.VOXEL_SIZE, synth.TRUNCATION)
    static = C.load_scene(tmp_path / "s.npz", log2_buckets=16)
    for _, P, _, _ in room_training[:3]:
        d1, c1 = _view(fs, intr, P)
        d2, c2 = _view(static, intr, P)
        a, b = d1.cpu().numpy().view(np.uint16), d2.cpu().numpy().view(np.uint16)
        assert np.mean(a == b) >= 0.999 and np.abs(a.astype(int) - b).max() <= 1
