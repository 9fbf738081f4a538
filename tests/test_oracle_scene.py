"""Pins of the oracle's voxel lookup and raycast against definitions outside it:
a Python dict of the block list, analytic ray-plane / ray-sphere / ray-box depths,
constant or linear colour fields that trilinear interpolation reproduces exactly, and the
invariance of a render under a shift of scene and camera by whole blocks (into negative
coordinates)."""
import functools
import math

import numpy as np

import oracle
from paper_1801_08361_gb300 import synth
from scenes import blocks_from_sdf, empty_blocks, ray_box_entry, ray_box_exit, ray_dirs


def test_lookup_matches_dict(room, oracle_room):
    _, blocks = room
    table = {tuple(c): i for i, c in enumerate(blocks.coords.tolist())}
    got = oracle_room.find_blocks(blocks.coords)
    assert np.array_equal(got, np.arange(blocks.n_blocks))
    rng = np.random.default_rng(0)
    keys = rng.integers(-40, 120, (200000, 3)).astype(np.int32)
    want = np.array([table.get(tuple(k), -1) for k in keys.tolist()])
    assert np.array_equal(oracle_room.find_blocks(keys), want)
    assert (want >= 0).any() and (want < 0).any()


def test_empty_scene_is_all_invalid():
    sc = oracle.Scene(empty_blocks())
    intr = synth.Intrinsics.for_size(32, 24)
    d, c = sc.raycast(intr, synth.look_pose(np.array([0.0, 0, 0]), 0.3, 0.1))
    assert (d == 0).all() and (c == 0).all()


def _plane_room():
    world = synth.room_world(3, n_boxes=0)
    return world, synth.sample_scene(world)


def test_plane_depth_exact_to_rounding():
    """A wall is an exactly linear SDF in its truncation band, so trilinear samples and the
    secant root are exact: depth must be the analytic z rounded half up (Sec. 3.3.1 raycast)."""
    _, blocks = _plane_room()
    sc = oracle.Scene(blocks)
    intr = synth.Intrinsics.for_size(160, 120)
    pose = synth.look_pose(np.array([2.0, 2.0, 1.5]), math.radians(7.0), math.radians(-4.0))
    depth, rgba = sc.raycast(intr, pose)
    dirs, C = ray_dirs(intr, pose)
    lam = (4.0 - C[0]) / dirs[..., 0]                     # plane x = 4
    hit = C + lam[..., None] * dirs
    assert (hit[..., 1] > 0.1).all() and (hit[..., 1] < 3.9).all() and (hit[..., 2] > 0.1).all()
    assert (depth > 0).all()
    err = np.abs(depth.astype(np.float64) - 1000.0 * lam)
    assert err.max() <= 0.5 + 1e-6


def test_sphere_depth_within_interpolation_bound():
    """Sphere R = 0.5 m: trilinear interpolation of |p - c| - R errs by O(s^2 / R) (~0.02 mm at
    s = 5 mm), so rounded depths lie within 0.5 mm + 0.1 mm of the analytic hit on rays that meet
    the surface at less than 60 degrees from the normal."""
    c0, R = np.array([0.3, -0.2, 2.0]), 0.5
    blocks = blocks_from_sdf(lambda p: np.linalg.norm(p - c0, axis=1) - R,
                             lambda p: np.full((len(p), 3), 200, np.uint8), c0 - 0.6, c0 + 0.6)
    sc = oracle.Scene(blocks)
    intr = synth.Intrinsics.for_size(96, 72)
    pose = np.eye(4)
    depth, rgba = sc.raycast(intr, pose)
    dirs, C = ray_dirs(intr, pose)
    oc = C - c0
    a = (dirs * dirs).sum(-1)
    b = 2 * (dirs * oc).sum(-1)
    cc = (oc * oc).sum() - R * R
    disc = b * b - 4 * a * cc
    lam = np.where(disc > 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), np.inf)
    hitp = C + np.where(np.isfinite(lam), lam, 0)[..., None] * dirs
    n = (hitp - c0) / R
    cosang = -(n * dirs).sum(-1) / np.sqrt(a)
    good = np.isfinite(lam) & (cosang > 0.5)
    assert good.sum() > 500
    err = np.abs(depth[good].astype(np.float64) - 1000 * lam[good])
    assert (depth[good] > 0).all()
    assert err.max() <= 0.6
    miss = disc < -1e-3
    assert (depth[miss] == 0).all()
    assert (rgba[good][:, :3] == 200).all()


def test_linear_colour_is_reproduced():
    """A colour field linear in x is reproduced by trilinear interpolation up to the rounding of
    the voxel values (<= 1 level); constant channels come back exactly."""
    blocks = blocks_from_sdf(lambda p: 3.0 - p[:, 2],
                             lambda p: np.stack([np.floor(120.0 + 30.0 * p[:, 0] + 0.5),
                                                 np.full(len(p), 17.0), np.full(len(p), 230.0)], 1).astype(np.uint8),
                             np.array([-2.2, -1.7, 2.9]), np.array([2.2, 1.7, 3.1]))
    sc = oracle.Scene(blocks)
    intr = synth.Intrinsics.for_size(40, 30)
    depth, rgba = sc.raycast(intr, np.eye(4))
    ok = depth > 0
    assert ok.all()
    assert (rgba[..., 1] == 17).all() and (rgba[..., 2] == 230).all()
    dirs, C = ray_dirs(intr, np.eye(4))
    xh = 3.0 * dirs[..., 0]
    assert np.abs(rgba[..., 0].astype(np.float64) - (120.0 + 30.0 * xh)).max() <= 1.0
    assert (np.abs(depth.astype(int) - 3000) <= 0).all()


def test_box_world_matches_ray_box_intersections(room, oracle_room):
    """The synthetic room: depth vs exact slab-method intersections of the room shell and its
    boxes; trilinear interpolation is exact away from edges, so nearly every pixel agrees to 1 mm."""
    world, _ = room
    intr = synth.Intrinsics.for_size(80, 60)
    train = synth.training_poses(world, 4, seed=11)
    for pose in train:
        depth, _ = oracle_room.raycast(intr, pose)
        dirs, C = ray_dirs(intr, pose)
        shell = world.comps[0]
        lam = ray_box_exit(C, dirs, shell[1:4], shell[4:7])
        for comp in world.comps[1:]:
            lam = np.minimum(lam, ray_box_entry(C, dirs, comp[1:4], comp[4:7]))
        err = np.abs(depth.astype(np.float64) - 1000 * lam)
        assert (depth > 0).mean() > 0.99
        assert (err <= 1.0).mean() > 0.97
        assert np.median(err) < 0.5


def test_noise_model_adds_quadratic_term():
    """Depth noise (Appendix, axial noise quadratic in depth): z_mm + 1.5 z^2 n, rounded half up."""
    _, blocks = _plane_room()
    sc = oracle.Scene(blocks)
    intr = synth.Intrinsics.for_size(40, 30)
    pose = synth.look_pose(np.array([2.0, 2.0, 1.5]), 0.0, 0.0)
    noise = np.full((30, 40), 2.0, np.float32)
    d0, _ = sc.raycast(intr, pose)
    d1, _ = sc.raycast(intr, pose, noise=noise)
    dirs, C = ray_dirs(intr, pose)
    lam = (4.0 - C[0]) / dirs[..., 0]
    want = np.floor(1000 * lam + 1.5 * lam * lam * 2.0 + 0.5)
    assert np.abs(d1 - want).max() <= 1
    assert (d1.astype(int) - d0.astype(int) >= 11).all()


@functools.lru_cache(maxsize=1)
def _room_blocks():
    return synth.sample_scene(synth.room_world(1))


def test_shift_by_whole_blocks_into_negative_coordinates():
    """Moving the scene and the camera by -120 blocks in x and y (-4.8 m: every voxel of the room
    then has negative x and y) leaves the render unchanged up to last-bit rounding of positions:
    the voxel grid, block lookups and trilinear corners must treat negative coordinates like
    positive ones (floor, not truncation)."""
    blocks = _room_blocks()
    shift = np.array([-120, -120, 0])
    moved = synth.SceneBlocks(np.ascontiguousarray(blocks.coords + shift.astype(np.int32)), blocks.tsdf,
                              blocks.rgba, blocks.voxel_size, blocks.mu, blocks.scene_to_world)
    intr = synth.Intrinsics.for_size(80, 60)
    pose = synth.look_pose(np.array([1.3, 1.1, 1.4]), math.radians(35.0), math.radians(-10.0))
    pose_moved = pose.copy()
    pose_moved[:3, 3] += shift * 8 * blocks.voxel_size
    d0, c0 = oracle.Scene(blocks).raycast(intr, pose)
    d1, c1 = oracle.Scene(moved).raycast(intr, pose_moved)
    assert (d0 > 0).mean() > 0.9 and (moved.coords[:, :2] < 0).all()
    assert np.mean(d0 != d1) <= 1e-3 and np.abs(d0.astype(int) - d1).max() <= 1
    dc = np.abs(c0.astype(int) - c1)
    assert np.mean(dc > 0) <= 1e-3 and dc.max() <= 1
