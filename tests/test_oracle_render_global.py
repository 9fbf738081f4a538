"""Pins of the oracle's global map rendering (Appendix B.2): the per-pixel depth test against a
brute-force loop over hand-made depth images (ties to the lower index, no hit = +inf); one scene
reduces to its own raycast; and a room cut into two overlapping pieces, each sampled in its own
random frame and placed by its true global pose, renders like the whole room."""

import numpy as np
import pytest

import oracle
from paper_1801_08361_gb300 import synth


class FakeScene:
    def __init__(self, depth, rgba):
        self.depth, self.rgba, self.poses = depth, rgba, []

    def raycast(self, intr, pose, pixels=None):
        self.poses.append(np.array(pose))
        return self.depth, self.rgba


def test_depth_test_against_a_brute_force_loop():
    rng = np.random.default_rng(2)
    n, H, W = 4, 7, 9
    depths = rng.integers(0, 6, (n, H, W)).astype(np.uint16)      # many ties and misses
    cols = rng.integers(0, 256, (n, H, W, 4)).astype(np.uint8)
    scenes = [FakeScene(depths[a], cols[a]) for a in range(n)]
    g = [np.eye(4) for _ in range(n)]
    d, c, o, _ = oracle.render_global(scenes, g, synth.Intrinsics.for_size(W, H), np.eye(4))
    for v in range(H):
        for u in range(W):
            best = -1
            for a in range(n):
                if depths[a, v, u] > 0 and (best < 0 or depths[a, v, u] < depths[best, v, u]):
                    best = a
            assert o[v, u] == best
            assert d[v, u] == (depths[best, v, u] if best >= 0 else 0)
            assert np.array_equal(c[v, u], cols[best, v, u] if best >= 0 else np.zeros(4, np.uint8))


def test_local_poses_are_inverse_global_times_camera():
    rng = np.random.default_rng(4)
    gs = [synth.random_rigid(rng) for _ in range(3)]
    Pg = synth.random_rigid(rng)
    scenes = [FakeScene(np.ones((2, 2), np.uint16), np.zeros((2, 2, 4), np.uint8)) for _ in range(3)]
    oracle.render_global(scenes, gs, synth.Intrinsics.for_size(2, 2), Pg)
    for sc, g in zip(scenes, gs):
        # the local pose maps camera coordinates into scene a: gT_a (local) = P_g
        assert np.allclose(g @ sc.poses[0], Pg, atol=1e-12)


@pytest.fixture(scope="module")
def room_pieces():
    world = synth.room_world(1)
    shell = world.comps[0]
    lo, hi = shell[1:4], shell[4:7]
    mid = 0.5 * (lo[0] + hi[0])
    rng = np.random.default_rng(8)
    pieces = []
    for x0, x1 in ((lo[0] - 0.1, mid + 0.3), (mid - 0.3, hi[0] + 0.1)):
        S = synth.random_rigid(rng)
        crop = np.array([x0, lo[1] - 0.1, lo[2] - 0.1, x1, hi[1] + 0.1, hi[2] + 0.1])
        pieces.append((oracle.Scene(synth.sample_scene(world, scene_to_world=S, crop=crop)), S))
    whole = oracle.Scene(synth.sample_scene(world))
    return world, pieces, whole


def test_one_scene_is_its_own_raycast(room_pieces):
    world, pieces, _ = room_pieces
    intr = synth.Intrinsics.for_size(64, 48)
    sc, S = pieces[0]
    Pw = synth.training_poses(world, 1, seed=5)[0]
    d, c, o, _ = oracle.render_global([sc], [S], intr, Pw)
    d1, c1 = sc.raycast(intr, np.linalg.inv(S) @ Pw)
    assert np.array_equal(d, d1) and np.array_equal(c, c1)
    assert np.array_equal(o, np.where(d1 > 0, 0, -1))


def test_two_pieces_render_like_the_whole_room(room_pieces):
    world, pieces, whole = room_pieces
    intr = synth.Intrinsics.for_size(80, 60)
    for Pw in synth.training_poses(world, 3, seed=6):
        d, c, o, _ = oracle.render_global([p[0] for p in pieces], [p[1] for p in pieces], intr, Pw)
        dw, cw = whole.raycast(intr, Pw)
        both = (d > 0) & (dw > 0)
        assert np.mean((d > 0) == (dw > 0)) > 0.995
        assert np.mean(np.abs(d[both].astype(int) - dw[both]) <= 1) > 0.99
        assert set(np.unique(o[d > 0])) <= {0, 1}
