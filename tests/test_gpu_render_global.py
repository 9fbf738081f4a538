"""Global map rendering on the GPU (relo_render_global, Appendix B.2).  The fused kernel (each
scene's march cut past the depth it must beat) equals, bit for bit, the composite of separate
relo_raycast_view renders of every scene; it matches the oracle's global rendering within the
raycast tolerances on a room cut into two pieces in random frames (and at 640 x 480 on sampled
pixels); one scene is its own raycast; ties go to the lower index."""
import numpy as np
import pytest
import torch

import oracle
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def pieces():
    world = synth.room_world(1)
    shell = world.comps[0]
    lo, hi = shell[1:4], shell[4:7]
    mid = 0.5 * (lo[0] + hi[0])
    rng = np.random.default_rng(8)
    out = []
    for x0, x1 in ((lo[0] - 0.1, mid + 0.3), (mid - 0.3, hi[0] + 0.1)):
        S = synth.random_rigid(rng)
        crop = np.array([x0, lo[1] - 0.1, lo[2] - 0.1, x1, hi[1] + 0.1, hi[2] + 0.1])
        blocks = synth.sample_scene(world, scene_to_world=S, crop=crop)
        out.append((B.Scene(blocks, 16), oracle.Scene(blocks), S))
    poses = synth.training_poses(world, 3, seed=6)
    return world, out, poses


def _render(scenes, gposes, intr, Pg):
    H, W = intr.height, intr.width
    d = torch.zeros((H, W), dtype=torch.int16, device=DEV)
    c = torch.zeros((H, W, 4), dtype=torch.uint8, device=DEV)
    o = torch.zeros((H, W), dtype=torch.int8, device=DEV)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    B.render_global(scenes, gposes, intr, Pg, d, c, o, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return d.cpu().numpy().view(np.uint16), c.cpu().numpy(), o.cpu().numpy()


def _separate(scenes, gposes, intr, Pg):
    """Each scene by relo_raycast_view, then the depth test in numpy (no cut)."""
    H, W = intr.height, intr.width
    ds, cs = [], []
    for sc, g in zip(scenes, gposes):
        d = torch.zeros((H, W), dtype=torch.int16, device=DEV)
        c = torch.zeros((H, W, 4), dtype=torch.uint8, device=DEV)
        B.raycast_view(sc, intr, np.linalg.inv(g) @ Pg, d, c)
        ds.append(d.cpu().numpy().view(np.uint16))
        cs.append(c.cpu().numpy())
    torch.cuda.synchronize()
    ds, cs = np.stack(ds), np.stack(cs)
    key = np.where(ds > 0, ds.astype(np.int64), 1 << 40)
    own = np.argmin(key, 0)
    hit = np.take_along_axis(ds, own[None], 0)[0] > 0
    depth = np.where(hit, np.take_along_axis(ds, own[None], 0)[0], 0)
    col = np.where(hit[..., None], np.take_along_axis(cs, own[None, ..., None], 0)[0], 0)
    return depth, col, np.where(hit, own, -1)


def test_fused_kernel_equals_separate_renders(pieces):
    _, ps, poses = pieces
    intr = synth.Intrinsics.for_size(200, 150)
    scenes = [p[0] for p in ps]
    gp = [p[2] for p in ps]
    for Pg in poses:
        for order in ((0, 1), (1, 0)):
            sc = [scenes[k] for k in order]
            g = [gp[k] for k in order]
            got = _render(sc, g, intr, Pg)
            want = _separate(sc, g, intr, Pg)
            for a, b in zip(got, want):
                assert np.array_equal(a, b)


def test_matches_oracle(pieces):
    _, ps, poses = pieces
    intr = synth.Intrinsics.for_size(160, 120)
    for Pg in poses:
        d, c, o = _render([p[0] for p in ps], [p[2] for p in ps], intr, Pg)
        do, co, oo, depths = oracle.render_global([p[1] for p in ps], [p[2] for p in ps], intr, Pg)
        both = (d > 0) & (do > 0)
        assert np.mean((d > 0) != (do > 0)) <= 5e-4
        assert np.mean(np.abs(d[both].astype(int) - do[both]) <= 1) >= 0.999
        # the owner is decided where the oracle's two depths differ by more than 2 mm
        key = np.where(depths > 0, depths.astype(np.int64), 1 << 40)
        clear = both & (np.abs(key[0] - key[1]) > 2)
        assert np.array_equal(o[clear], oo[clear])
        same = both & (o == oo)
        assert np.mean(np.abs(c[same].astype(int) - co[same]).max(-1) <= 1) >= 0.995


def test_full_size_sampled_pixels_match_oracle(pieces):
    _, ps, poses = pieces
    intr = synth.Intrinsics.for_size(640, 480)
    rng = np.random.default_rng(3)
    px = rng.choice(640 * 480, 3000, replace=False)
    d, _, o = _render([p[0] for p in ps], [p[2] for p in ps], intr, poses[0])
    do, _, oo, depths = oracle.render_global([p[1] for p in ps], [p[2] for p in ps], intr, poses[0], pixels=px)
    d, o = d.reshape(-1)[px], o.reshape(-1)[px]
    both = (d > 0) & (do > 0)
    assert np.mean((d > 0) != (do > 0)) <= 1e-3
    assert np.mean(np.abs(d[both].astype(int) - do[both]) <= 1) >= 0.999
    key = np.where(depths > 0, depths.astype(np.int64), 1 << 40)
    clear = both & (np.abs(key[0] - key[1]) > 2)
    assert np.array_equal(o[clear], oo[clear])


def test_one_scene_and_ties(pieces):
    _, ps, poses = pieces
    intr = synth.Intrinsics.for_size(96, 72)
    sc, _, S = ps[0]
    d1, c1, o1 = _render([sc], [S], intr, poses[1])
    dv = torch.zeros((72, 96), dtype=torch.int16, device=DEV)
    cv = torch.zeros((72, 96, 4), dtype=torch.uint8, device=DEV)
    B.raycast_view(sc, intr, np.linalg.inv(S) @ poses[1], dv, cv)
    torch.cuda.synchronize()
    assert np.array_equal(d1, dv.cpu().numpy().view(np.uint16)) and np.array_equal(c1, cv.cpu().numpy())
    assert np.array_equal(o1, np.where(d1 > 0, 0, -1))
    d2, c2, o2 = _render([sc, sc], [S, S], intr, poses[1])     # identical copies: the first wins
    assert np.array_equal(d2, d1) and np.array_equal(c2, c1) and np.array_equal(o2, o1)


def test_bad_arguments(pieces):
    _, ps, poses = pieces
    intr = synth.Intrinsics.for_size(32, 24)
    d = torch.zeros((24, 32), dtype=torch.int16, device=DEV)
    with pytest.raises(B.ReloError):
        B.render_global([], [], intr, poses[0], d)
    tiny = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.ReloError):
        B.render_global([ps[0][0]], [ps[0][2]], intr, poses[0], d, workspace_dev=tiny)
