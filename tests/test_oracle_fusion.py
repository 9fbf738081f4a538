"""Pins of the oracle's TSDF fusion (Sec. 3.3 (a), Appendix B.3): a fronto-parallel plane gives
the closed-form truncated distance min(1, (Z0 - z) / mu) with weight 1 on every updated voxel and
leaves voxels more than mu behind the surface untouched; allocated blocks lie in the band; equal
frames average to themselves; two planes average to the float32 mean; weights stop at the cap; a
uniform colour is kept; a full scene reports it; and renders of the room fused from several poses
raycast back to the depths they came from."""
import numpy as np
import pytest

import oracle
from paper_1801_08361_gb300 import synth

VOX, MU = 0.005, 0.02
BS = 8 * VOX


def plane(intr, mm):
    return np.full((intr.height, intr.width), mm, dtype=np.uint16)


def voxel_z(fb):
    """Camera z (identity pose) of every voxel of the fused blocks, float64 [n, 512]."""
    k = np.arange(512) >> 6
    return (8 * fb.coords[:, 2:3] + k[None, :]).astype(np.float64) * VOX


def test_plane_closed_form():
    # the plane at 1.51 m does not sit on a block boundary, so the allocated blocks hold voxels more
    # than mu in front of it, where the truncated distance is clamped to 1
    Z0 = 1.51
    intr = synth.Intrinsics.for_size(64, 48)
    fs = oracle.FusionScene(4096, VOX, MU)
    assert fs.fuse(intr, np.eye(4), plane(intr, 1510))
    fb = fs.blocks()
    assert len(fb.coords) > 0
    # every allocated block meets the band [Z0 - mu, Z0 + mu] in z
    assert np.all(fb.coords[:, 2] * BS <= Z0 + MU + 1e-6) and np.all((fb.coords[:, 2] + 1) * BS >= Z0 - MU - 1e-6)
    z = voxel_z(fb)
    upd = fb.weight == 1
    assert np.all((fb.weight == 0) | upd)
    want = np.minimum(1.0, (Z0 - z) / MU)
    assert np.abs(fb.tsdf[upd] - want[upd]).max() < 1e-5
    assert np.any(upd & (Z0 - z > MU + 1e-6))              # the clamp is exercised
    # voxels more than mu behind the surface were not updated; those in front of it mostly were
    assert not np.any(upd & (z > Z0 + MU + 1e-6))
    assert np.all(fb.tsdf[~upd] == 1.0)
    assert upd[np.abs(z - Z0) < MU / 2].mean() > 0.5


def test_equal_frames_average_to_themselves_and_weights_stop_at_the_cap():
    intr = synth.Intrinsics.for_size(32, 24)
    one = oracle.FusionScene(4096, VOX, MU, max_weight=3)
    one.fuse(intr, np.eye(4), plane(intr, 1200))
    b1 = one.blocks()
    for _ in range(4):
        one.fuse(intr, np.eye(4), plane(intr, 1200))
    b5 = one.blocks()
    assert np.array_equal(b1.coords, b5.coords)
    assert np.array_equal(b1.tsdf, b5.tsdf)
    assert np.array_equal(b5.weight, np.where(b1.weight > 0, 3, 0))


def test_two_planes_average_in_float32():
    intr = synth.Intrinsics.for_size(32, 24)
    fs = oracle.FusionScene(4096, VOX, MU)
    fs.fuse(intr, np.eye(4), plane(intr, 1500))
    fs.fuse(intr, np.eye(4), plane(intr, 1510))
    fb = fs.blocks()
    z = voxel_z(fb).astype(np.float32)
    both = fb.weight == 2
    assert both.sum() > 100

    def f(mm):
        eta = np.float32(mm) * np.float32(0.001) - z
        return np.minimum(np.float32(1), eta / np.float32(MU))

    w1 = (f(1500) * np.float32(0) + f(1500)) / np.float32(1)
    want = (w1 * np.float32(1) + f(1510)) / np.float32(2)
    assert np.array_equal(fb.tsdf[both], want[both])


def test_uniform_colour_is_kept():
    intr = synth.Intrinsics.for_size(32, 24)
    rgba = np.zeros((24, 32, 4), np.uint8)
    rgba[..., :3] = (200, 17, 99)
    fs = oracle.FusionScene(4096, VOX, MU)
    for _ in range(3):
        fs.fuse(intr, np.eye(4), plane(intr, 1000), rgba)
    fb = fs.blocks()
    upd = fb.weight > 0
    assert np.all(fb.rgba[upd] == np.array([200, 17, 99, 255], np.uint8))
    assert np.all(fb.rgba[~upd] == 0)


def test_colour_average_rounds_half_up():
    """Colours 10 then 11: the running average after the second frame is 10.5, stored as 11."""
    intr = synth.Intrinsics.for_size(32, 24)
    fs = oracle.FusionScene(4096, VOX, MU)
    for c in (10, 11):
        rgba = np.zeros((24, 32, 4), np.uint8)
        rgba[..., :3] = c
        fs.fuse(intr, np.eye(4), plane(intr, 1000), rgba)
    fb = fs.blocks()
    both = fb.weight == 2
    assert both.any()
    assert np.all(fb.rgba[both][:, :3] == 11)


def test_full_scene_reports_it():
    intr = synth.Intrinsics.for_size(64, 48)
    fs = oracle.FusionScene(5, VOX, MU)
    assert not fs.fuse(intr, np.eye(4), plane(intr, 1500))
    assert len(fs.blocks().coords) == 5


@pytest.fixture(scope="module")
def room():
    world = synth.room_world(1)
    return world, oracle.Scene(synth.sample_scene(world))


def test_fused_renders_raycast_back(room):
    world, sc = room
    intr = synth.Intrinsics.for_size(80, 60)
    poses = synth.training_poses(world, 8, seed=21)
    fs = oracle.FusionScene(1 << 17, VOX, MU)
    frames = [sc.raycast(intr, P) for P in poses]
    for P, (d, c) in zip(poses, frames):
        assert fs.fuse(intr, P, d, c)
    fused = oracle.Scene(fs.blocks())
    for P, (d, c) in zip(poses[:3], frames[:3]):
        d2, c2 = fused.raycast(intr, P)
        both = (d > 0) & (d2 > 0)
        assert np.mean((d > 0) == (d2 > 0)) > 0.97
        assert np.mean(np.abs(d2[both].astype(int) - d[both]) <= 3) > 0.95
        assert np.mean(np.abs(c2[both].astype(int) - c[both]).max(-1) <= 24) > 0.9
