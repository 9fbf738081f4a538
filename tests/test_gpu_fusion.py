"""TSDF fusion on the GPU (relo_create_fusion_scene / relo_fuse_frame) against the oracle's fusion
on the same frames: the same blocks, and bit-identical truncated distances, colours and weights
(both sides take every decision and average in float32 in the same order); raycasts of the fused
scene (which walk its hash) match the oracle's raycast of the oracle's fused blocks; a full pool
reports RELO_ENOMEM; weights stop at the cap."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
VOX, MU = synth.VOXEL_SIZE, synth.TRUNCATION


@pytest.fixture(scope="module")
def frames(room, oracle_room):
    world, _ = room
    out = {}
    for W, H, n in ((160, 120, 6), (640, 480, 3)):
        intr = synth.Intrinsics.for_size(W, H)
        poses = synth.training_poses(world, n, seed=31 + W)[:n]
        out[W] = (intr, [(P,) + oracle_room.raycast(intr, P, noise=synth.depth_noise(H, W, 900 + i))
                         for i, P in enumerate(poses)])
    return out


def _fuse_both(intr, fr, capacity=1 << 17, max_weight=100, colour=True):
    g = B.FusionScene(capacity, VOX, MU, log2_buckets=16, max_weight=max_weight)
    o = oracle.FusionScene(capacity, VOX, MU, max_weight=max_weight)
    for P, d, c in fr:
        dd = torch.from_numpy(d.view(np.int16)).to(DEV)
        cc = torch.from_numpy(c).to(DEV) if colour else None
        g.fuse(intr, P, dd, cc)
        o.fuse(intr, P, d, c if colour else None)
    torch.cuda.synchronize()
    return g, o


@pytest.mark.parametrize("W", [160, 640])
def test_fused_blocks_equal_the_oracle(frames, W):
    intr, fr = frames[W]
    g, o = _fuse_both(intr, fr)
    coords, tsdf, rgba, weight = g.export()
    ob = o.blocks()
    assert len(coords) > 1000
    assert np.array_equal(coords, ob.coords)
    assert np.array_equal(weight, ob.weight)
    assert np.array_equal(tsdf.view(np.uint32), ob.tsdf.view(np.uint32))
    assert np.array_equal(rgba, ob.rgba)


def test_fused_scene_raycasts_like_the_oracle(frames):
    intr, fr = frames[160]
    g, o = _fuse_both(intr, fr)
    fused_o = oracle.Scene(o.blocks())
    for P, d_in, _ in fr[:3]:
        depth = torch.zeros((intr.height, intr.width), dtype=torch.int16, device=DEV)
        rgba = torch.zeros((intr.height, intr.width, 4), dtype=torch.uint8, device=DEV)
        B.raycast_view(g, intr, P, depth, rgba)
        torch.cuda.synchronize()
        d = depth.cpu().numpy().view(np.uint16)
        c = rgba.cpu().numpy()
        do, co = fused_o.raycast(intr, P)
        both = (d > 0) & (do > 0)
        assert np.mean((d > 0) != (do > 0)) <= 5e-4
        assert np.mean(np.abs(d[both].astype(int) - do[both]) <= 1) >= 0.999
        assert np.mean(np.abs(c[both].astype(int) - co[both]).max(-1) <= 1) >= 0.995
        # and the fused surface is where the frames put it
        ok = both & (d_in > 0)
        assert np.mean(np.abs(d[ok].astype(int) - d_in[ok]) <= 5) > 0.9


def test_weight_cap_and_depth_only(frames):
    intr, fr = frames[160]
    g, o = _fuse_both(intr, [fr[0]] * 5, max_weight=3, colour=False)
    coords, tsdf, rgba, weight = g.export()
    ob = o.blocks()
    assert weight.max() == 3 and np.array_equal(weight, ob.weight)
    assert np.array_equal(tsdf.view(np.uint32), ob.tsdf.view(np.uint32))
    assert not rgba.any()


def test_full_pool_reports_enomem(frames):
    intr, fr = frames[160]
    g = B.FusionScene(64, VOX, MU, log2_buckets=8)
    P, d, c = fr[0]
    g.fuse(intr, P, torch.from_numpy(d.view(np.int16)).to(DEV), torch.from_numpy(c).to(DEV))
    with pytest.raises(B.ReloError) as e:
        g.block_count()
    assert e.value.status == B.ENOMEM


def test_bad_arguments(frames):
    intr, fr = frames[160]
    with pytest.raises(B.ReloError):
        B.FusionScene(0, VOX, MU)
    with pytest.raises(B.ReloError):
        B.FusionScene(16, VOX, MU, max_weight=0)
    g = B.FusionScene(1024, VOX, MU, log2_buckets=8)
    tiny = torch.empty(64, dtype=torch.uint8, device=DEV)
    P, d, _ = fr[0]
    with pytest.raises(B.ReloError):
        g.fuse(intr, P, torch.from_numpy(d.view(np.int16)).to(DEV), workspace_dev=tiny)


def test_frame_statistics_count_the_blocks(frames):
    intr, fr = frames[160]
    g = B.FusionScene(1 << 16, VOX, MU, log2_buckets=14)
    created = updated = 0
    for P, d, c in fr:
        g.fuse(intr, P, torch.from_numpy(d.view(np.int16)).to(DEV), torch.from_numpy(c).to(DEV))
        vis, new = g.last_frame_stats(intr)
        assert vis >= new >= 0 and vis > 0
        created += new
        updated += vis
    assert created == g.block_count()
    assert updated == g.block_updates()


def test_many_frames_in_one_call_equal_frame_by_frame(frames):
    intr, fr = frames[160]
    g1 = B.FusionScene(1 << 16, VOX, MU, log2_buckets=14)
    g2 = B.FusionScene(1 << 16, VOX, MU, log2_buckets=14)
    d = torch.from_numpy(np.stack([f[1] for f in fr]).view(np.int16)).to(DEV)
    c = torch.from_numpy(np.stack([f[2] for f in fr])).to(DEV)
    for k, (P, _, _) in enumerate(fr):
        g1.fuse(intr, P, d[k], c[k])
    g2.fuse_many(intr, [f[0] for f in fr], d, c)
    torch.cuda.synchronize()
    for a, b in zip(g1.export(), g2.export()):
        assert np.array_equal(a, b)
