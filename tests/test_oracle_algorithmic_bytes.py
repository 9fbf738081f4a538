"""Pins of oracle.raycast_touched, the count of the distinct data one view's raycast reads (the
algorithmic bytes behind the raycast rooflines): an empty scene reads no voxel; on a wall facing
the camera at mid-voxel depth the colour voxels are exactly the distinct trilinear corners of the
analytic hit points; a depth-only render reads no colour and no more than the colour render."""
import numpy as np
import pytest

import oracle
from paper_1801_08361_gb300 import synth
from scenes import blocks_from_sdf, empty_blocks, ray_dirs

S = 0.005
X0 = 1.0025   # the wall x = X0 sits at x / s = 200.5: every hit's x corners are voxels 200 and 201


def _wall_scene():
    blocks = blocks_from_sdf(lambda p: X0 - p[:, 0], lambda p: np.full((len(p), 3), 90, np.uint8),
                             (0.95, -0.7, -0.55), (1.05, 0.7, 0.55))
    return oracle.Scene(blocks)


def _looking_along_x():
    # camera right = world -y, camera down = world -z; the centre is off the voxel grid
    return synth.look_pose(np.array([0.0, 0.01137, -0.00713]), 0.0, 0.0)


def test_an_empty_scene_reads_no_voxel():
    sc = oracle.Scene(empty_blocks())
    intr = synth.Intrinsics.for_size(24, 18, 2.0)
    t = oracle.raycast_touched(sc, intr, _looking_along_x(), with_colour=True)
    assert t["tsdf_voxels"] == 0 and t["colour_voxels"] == 0
    assert t["block_keys"] > 0          # the march still looks its blocks up


@pytest.mark.parametrize("size", [(40, 30), (320, 240)])
def test_colour_voxels_are_the_corners_of_the_hit_points(size):
    """At 40 x 30 each pixel's footprint on the wall (3 cm) exceeds a voxel, so no two pixels share
    a corner; at 320 x 240 (3.8 mm) neighbouring pixels share corners, and each counts once."""
    W, H = size
    sc = _wall_scene()
    intr = synth.Intrinsics.for_size(W, H, 2.0)
    pose = _looking_along_x()
    depth, _ = sc.raycast(intr, pose)
    dirs, C = ray_dirs(intr, pose)
    lam = (X0 - C[0]) / dirs[..., 0]
    assert (depth > 0).all() and np.abs(depth - 1000.0 * lam).max() <= 0.5 + 1e-6
    hit = C + lam[..., None] * dirs
    q = hit[..., 1:] / S
    assert np.abs(q - np.round(q)).min() > 1e-6        # no hit on a voxel plane in y or z
    jk = np.floor(q).reshape(-1, 2).astype(np.int64)
    corners = np.concatenate([np.stack([np.full(len(jk), 200 + a), jk[:, 0] + b, jk[:, 1] + c], 1)
                              for a in (0, 1) for b in (0, 1) for c in (0, 1)])
    corners = np.unique(corners, axis=0)
    t = oracle.raycast_touched(sc, intr, pose, with_colour=True)
    assert t["colour_voxels"] == len(corners)
    if W >= 320:
        assert len(corners) < 2 * W * H             # shared corners counted once
    assert t["tsdf_voxels"] >= t["colour_voxels"]
    assert t["block_keys"] >= len(np.unique(corners // 8, axis=0))
    v = oracle.raycast_touched(sc, intr, pose, with_colour=False)
    assert v["colour_voxels"] == 0
    assert 0 < v["tsdf_voxels"] <= t["tsdf_voxels"] and v["block_keys"] <= t["block_keys"]
