"""GPU parity: every stage of the relocalisation path through the C ABI against the CPU oracle on
identical seeded inputs (stage-isolated: each GPU stage gets the images the oracle stage got).

Bars: block lookup, forest leaves, verification counts, hypothesis sets, drawn pixels and
reservoirs bit-exact; raycast depth within 1 mm on >= 99.9 % of co-valid pixels (FP32 march
against FP64); energies within 1e-5 relative; poses within 1e-4 m / 1e-4 (rotation entries);
survivor sets exact except at near-ties (oracle cut margin below 1e-5 relative), which the round
test resolves by teacher forcing."""

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


def u16_np(t):
    return t.cpu().numpy().view(np.uint16)


@pytest.fixture(scope="module")
def gpu_room(room):
    return B.Scene(room[1], 16)


@pytest.fixture(scope="module")
def gpu_forest(room_forest):
    return B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)


def gpu_render(scene, intr, pose, noise=None):
    depth = torch.zeros((intr.height, intr.width), dtype=torch.int16, device=DEV)
    rgba = torch.zeros((intr.height, intr.width, 4), dtype=torch.uint8, device=DEV)
    nz = None if noise is None else torch.from_numpy(noise).to(DEV)
    B.raycast_view(scene, intr, pose, depth, rgba, noise_dev=nz)
    torch.cuda.synchronize()
    return u16_np(depth), rgba.cpu().numpy()


# ------------------------------------------------------------------------------------------------
# a0: hash lookup
# ------------------------------------------------------------------------------------------------
def test_lookup_bit_exact(room, oracle_room, gpu_room):
    _, blocks = room
    rng = np.random.default_rng(1)
    keys = np.concatenate([blocks.coords, rng.integers(-60, 140, (300000, 3)).astype(np.int32),
                           np.array([[32767, -32768, 0], [40000, 0, 0], [-40000, 5, 5]], np.int32)])
    kd = torch.from_numpy(keys).to(DEV)
    out = torch.empty(len(keys), dtype=torch.int64, device=DEV)
    B.scene_lookup(gpu_room, kd, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle_room.find_blocks(keys))


# ------------------------------------------------------------------------------------------------
# a1: raycast
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("size", [(320, 240), (100, 75), (17, 9), (1, 1)])
@pytest.mark.parametrize("noisy", [False, True])
@pytest.mark.parametrize("grid", [True, False])
@pytest.mark.parametrize("apron", [True, False])
def test_raycast_parity(room, oracle_room, gpu_room, size, noisy, grid, apron):
    """Both lookup paths of the raycast (dense grid with empty-cell skipping, hash walk), each with
    the tsdf's apron copy and with neighbour lookups for samples on a block's last voxel."""
    world, _ = room
    W, H = size
    intr = synth.Intrinsics.for_size(W, H)
    poses = synth.training_poses(world, 3, seed=21)
    gpu_room.use_grid(grid)
    gpu_room.use_apron(apron)
    try:
        _raycast_parity_poses(oracle_room, gpu_room, intr, poses, noisy)
    finally:
        gpu_room.use_grid(True)
        gpu_room.use_apron(True)


def _raycast_parity_poses(oracle_room, gpu_room, intr, poses, noisy):
    W, H = intr.width, intr.height
    for i, P in enumerate(poses):
        noise = synth.depth_noise(H, W, 50 + i) if noisy else None
        dg, cg = gpu_render(gpu_room, intr, P, noise)
        do, co = oracle_room.raycast(intr, P, noise=noise)
        both = (dg > 0) & (do > 0)
        mismatch = ((dg > 0) != (do > 0)).mean()
        assert mismatch <= max(5e-4, 1.0 / (W * H) if W * H < 100 else 5e-4)
        if both.any():
            diff = np.abs(dg[both].astype(int) - do[both].astype(int))
            assert (diff <= 1).mean() >= 0.999
            close = both & (np.abs(dg.astype(int) - do.astype(int)) <= 1)
            cdiff = np.abs(cg[close][:, :3].astype(int) - co[close][:, :3].astype(int)).max(1)
            assert (cdiff <= 1).mean() >= 0.995
            assert (cg[both][:, 3] == 255).all()
        assert (cg[dg == 0] == 0).all()


def test_raycast_grid_skips_match_the_block_walk(room, gpu_room):
    """Through the grid the march jumps over whole cubes of unallocated blocks; through the hash
    it steps one block at a time.  Both end each free run on the same block face, so both
    evaluate the same samples: the images agree (up to a last-bit difference of an exit
    parameter where a ray crosses a block edge exactly)."""
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    for i, P in enumerate(synth.training_poses(world, 4, seed=23)):
        noise = synth.depth_noise(240, 320, 90 + i)
        dg, cg = gpu_render(gpu_room, intr, P, noise)
        gpu_room.use_grid(False)
        try:
            dh, ch = gpu_render(gpu_room, intr, P, noise)
        finally:
            gpu_room.use_grid(True)
        assert (dg == dh).mean() >= 0.9999
        assert np.abs(dg.astype(int) - dh.astype(int)).max() <= 1
        assert (np.abs(cg.astype(int) - ch.astype(int)).max(-1) <= 1).all()


@pytest.mark.parametrize("grid", [True, False])
def test_raycast_apron_equals_neighbour_lookups(room, gpu_room, grid):
    """The apron copy holds, on each block's last plane, the neighbouring blocks' first voxels (+1
    where unallocated): exactly the values the march otherwise looks up, in the same order, so
    depth and colour images are identical, in both lookup paths."""
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    gpu_room.use_grid(grid)
    try:
        for i, P in enumerate(synth.training_poses(world, 4, seed=29)):
            noise = synth.depth_noise(240, 320, 70 + i)
            da, ca = gpu_render(gpu_room, intr, P, noise)
            gpu_room.use_apron(False)
            try:
                dn, cn = gpu_render(gpu_room, intr, P, noise)
            finally:
                gpu_room.use_apron(True)
            assert (da > 0).mean() > 0.5
            assert np.array_equal(da, dn) and np.array_equal(ca, cn)
    finally:
        gpu_room.use_grid(True)


def test_raycast_views_equals_single_views(room, gpu_room):
    """The batched render is the same raycast per view: identical images."""
    world, _ = room
    intr = synth.Intrinsics.for_size(96, 72)
    poses = synth.training_poses(world, 2, seed=27)[:5]
    n = len(poses)
    noise = torch.from_numpy(np.stack([synth.depth_noise(72, 96, 300 + k) for k in range(n)])).to(DEV)
    depth = torch.zeros((n, 72, 96), dtype=torch.int16, device=DEV)
    rgba = torch.zeros((n, 72, 96, 4), dtype=torch.uint8, device=DEV)
    ws = torch.empty(B.raycast_views_workspace_size(n), dtype=torch.uint8, device=DEV)
    B.raycast_views(gpu_room, intr, poses, depth, rgba, noise_dev=noise, workspace_dev=ws)
    torch.cuda.synchronize()
    for k, P in enumerate(poses):
        d1 = torch.zeros((72, 96), dtype=torch.int16, device=DEV)
        c1 = torch.zeros((72, 96, 4), dtype=torch.uint8, device=DEV)
        B.raycast_view(gpu_room, intr, P, d1, c1, noise_dev=noise[k])
        torch.cuda.synchronize()
        assert torch.equal(d1, depth[k]) and torch.equal(c1, rgba[k])
    with pytest.raises(B.ReloError) as e:
        B.raycast_views(gpu_room, intr, poses, depth, rgba, workspace_dev=ws[:64])
    assert e.value.status == B.EINVAL


def test_raycast_empty_scene():
    from scenes import empty_blocks
    sc = B.Scene(empty_blocks(), 8)
    intr = synth.Intrinsics.for_size(48, 32)
    d, c = gpu_render(sc, intr, synth.look_pose(np.array([0.0, 0, 1]), 0.2, 0.0))
    assert (d == 0).all() and (c == 0).all()


def test_raycast_rejects_bad_arguments(gpu_room):
    intr = synth.Intrinsics.for_size(0, 10)
    depth = torch.zeros((10, 10), dtype=torch.int16, device=DEV)
    with pytest.raises(B.ReloError) as e:
        B.raycast_view(gpu_room, intr, np.eye(4), depth)
    assert e.value.status == B.EINVAL


# ------------------------------------------------------------------------------------------------
# a2: forest
# ------------------------------------------------------------------------------------------------
def test_forest_bit_exact_on_query(room, oracle_room, room_forest, gpu_forest):
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    P = synth.training_poses(world, 2, seed=31)[1]
    d, c = oracle_room.raycast(intr, P)
    leaves = torch.zeros((5, 240, 320), dtype=torch.int16, device=DEV)
    B.forest_eval(gpu_forest, u16_dev(d), torch.from_numpy(c).to(DEV), leaves)
    torch.cuda.synchronize()
    assert np.array_equal(u16_np(leaves), oracle.forest_eval(room_forest.nodes, d, c))


@pytest.mark.parametrize("trees,depth", [(3, 1), (3, 7), (3, 15), (5, 15), (6, 9), (8, 12), (11, 15)])
def test_forest_bit_exact_ragged_random(trees, depth):
    """Every unrolled width of the kernel (4, 5, 6, 8 and 16 tree slots) on ragged random images."""
    rng = np.random.default_rng(depth + 100 * trees)
    H, W = 23, 37
    d = rng.integers(200, 9000, (H, W)).astype(np.uint16)
    d[rng.random((H, W)) < 0.2] = 0
    c = rng.integers(0, 256, (H, W, 4)).astype(np.uint8)
    nodes = synth.random_forest_nodes(trees, depth, seed=depth + 100 * trees)
    f = B.Forest(nodes, max_modes=4)
    leaves = torch.zeros((trees, H, W), dtype=torch.int16, device=DEV)
    B.forest_eval(f, u16_dev(d), torch.from_numpy(c).to(DEV), leaves)
    torch.cuda.synchronize()
    want = oracle.forest_eval(nodes, d, c)
    assert np.array_equal(u16_np(leaves), want)
    assert (want[:, d == 0] == 0xFFFF).all()


# ------------------------------------------------------------------------------------------------
# a3 / a4: RANSAC
# ------------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def room_query(room, oracle_room, room_forest, room_training):
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    P = synth.query_poses(world, [f[1] for f in room_training], 1, seed=3)[0]
    d, c = oracle_room.raycast(intr, P)
    leaves = oracle.forest_eval(room_forest.nodes, d, c)
    return intr, P, d, c, leaves


def _workspace(intr, prm):
    return torch.empty(B.ransac_workspace_size(intr.width, intr.height, prm), dtype=torch.uint8, device=DEV)


def test_hypotheses_bit_exact(room_forest, gpu_forest, room_query):
    intr, P, d, c, leaves = room_query
    K = 64
    prm_o = oracle.RansacParams(n_hyps=K, batch=500, seed=9)
    poses_o, ok_o, tries_o = oracle.generate_hypotheses(d, intr, leaves, room_forest, prm_o)
    prm = B.ransac_params(n_hyps=K, batch=500, seed=9)
    poses = torch.zeros((K, 12), dtype=torch.float64, device=DEV)
    valid = torch.zeros(K, dtype=torch.int32, device=DEV)
    tries = torch.zeros(K, dtype=torch.int32, device=DEV)
    B.ransac_hypotheses(gpu_forest, u16_dev(d), u16_dev(leaves), intr, prm, _workspace(intr, prm), poses, valid, tries)
    torch.cuda.synchronize()
    assert np.array_equal(valid.cpu().numpy().astype(bool), ok_o)
    assert np.array_equal(tries.cpu().numpy(), tries_o)
    pg = poses.cpu().numpy().reshape(K, 3, 4)
    assert np.abs(pg[ok_o] - poses_o[ok_o, :3, :]).max() < 1e-9
    assert ok_o.sum() > K // 4


def _cut_is_near_tie(E, alive, keep):
    srt = sorted(alive.tolist(), key=lambda h: (E[h], h))
    if keep >= len(srt):
        return False
    a, b = E[srt[keep - 1]], E[srt[keep]]
    if not (np.isfinite(a) and np.isfinite(b)):
        return False
    return abs(b - a) <= 1e-5 * max(abs(a), abs(b)) + 1e-6


def test_rounds_teacher_forced(room_forest, gpu_forest, room_query):
    """Each round on the GPU starts from the oracle's state (alive set, poses, energies, earlier
    draws) and must reproduce the oracle's draws, energies, survivors, inlier counts and re-fits."""
    intr, P, d, c, leaves = room_query
    K, Bn = 64, 500
    prm_o = oracle.RansacParams(n_hyps=K, batch=Bn, seed=9)
    res = oracle.preemptive_ransac(d, intr, leaves, room_forest, prm_o, trace=True)
    tr = res["trace"]
    prm = B.ransac_params(n_hyps=K, batch=Bn, seed=9)
    ws = _workspace(intr, prm)
    dd, ld = u16_dev(d), u16_dev(leaves)
    valid = torch.from_numpy(tr.valid0.astype(np.int32)).to(DEV)
    poses_prev = tr.poses0[:, :3, :].copy()
    E_prev = np.where(tr.valid0, 0.0, np.inf)
    drawn_prev = np.zeros(0, np.int64)
    vpix = oracle.valid_pixels(d)          # the GPU draws positions in this raster-order list
    strict_rounds = 0
    for r, rd in enumerate(tr.rounds):
        alive = rd["alive_before"]
        n_alive = len(alive)
        keep = (n_alive + 1) // 2
        poses = torch.from_numpy(poses_prev.reshape(K, 12).copy()).to(DEV)
        energy = torch.from_numpy(E_prev.copy()).to(DEV)
        drawn = torch.zeros((r + 1) * Bn, dtype=torch.int32, device=DEV)
        drawn[: r * Bn] = torch.from_numpy(np.searchsorted(vpix, drawn_prev).astype(np.int32)).to(DEV)
        surv = torch.zeros(keep, dtype=torch.int32, device=DEV)
        inl = torch.zeros(K, dtype=torch.int32, device=DEV)
        if r > 0:
            inl.copy_(torch.from_numpy(tr.rounds[r - 1]["inliers"].astype(np.int32)))
        B.ransac_round(gpu_forest, dd, ld, intr, prm, r, torch.from_numpy(alive.astype(np.int32)).to(DEV), valid,
                       poses, energy, drawn, surv, inl, ws)
        torch.cuda.synchronize()
        # draws are integer-exact
        assert np.array_equal(vpix[drawn.cpu().numpy()[r * Bn:]], rd["pixels"])
        # energies of the alive hypotheses
        Eg, Eo = energy.cpu().numpy(), rd["energy"]
        fin = np.isfinite(Eo[alive])
        assert np.array_equal(np.isfinite(Eg[alive]), fin)
        rel = np.abs(Eg[alive][fin] - Eo[alive][fin]) / np.maximum(np.abs(Eo[alive][fin]), 1.0)
        assert rel.max() <= 1e-5
        # survivors: exact unless the oracle's cut is a near-tie
        sg = surv.cpu().numpy()
        if not _cut_is_near_tie(Eo, alive, keep):
            assert np.array_equal(sg, rd["survivors"])
            strict_rounds += 1
        # re-fits of survivors the two sides share, skipping near-threshold inlier decisions
        all_drawn = np.concatenate([drawn_prev, rd["pixels"]])
        cam = oracle.camera_points(d, intr, all_drawn)
        pg = poses.cpu().numpy().reshape(K, 3, 4)
        ig = inl.cpu().numpy()
        for h in set(sg.tolist()) & set(rd["survivors"].tolist()):
            if not tr.valid0[h]:
                continue
            pose_in = np.eye(4)
            pose_in[:3, :] = poses_prev[h]
            dm, am = oracle.decision_margins(pose_in, cam, all_drawn, leaves, room_forest, prm_o.inlier_dist)
            if dm.min() < 1e-4 or am.min() < 1e-3:
                continue
            assert ig[h] == rd["inliers"][h]
            assert np.abs(pg[h] - rd["poses"][h][:3, :]).max() < 1e-4
        # teacher forcing: continue from the oracle's state
        poses_prev = rd["poses"][:, :3, :].copy()
        E_prev = rd["energy"].copy()
        drawn_prev = all_drawn
    assert strict_rounds >= len(tr.rounds) - 1


def test_relocalise_matches_oracle(room, oracle_room, room_forest, gpu_forest, gpu_room, room_training):
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    queries = synth.query_poses(world, [f[1] for f in room_training], 3, seed=3)
    same = 0
    for i, P in enumerate(queries):
        d, c = oracle_room.raycast(intr, P)
        leaves = oracle.forest_eval(room_forest.nodes, d, c)
        ro = oracle.preemptive_ransac(d, intr, leaves, room_forest, oracle.RansacParams(n_hyps=64, batch=500, seed=i),
                                      trace=True)
        tied = any(_cut_is_near_tie(rd["energy"], rd["alive_before"], (len(rd["alive_before"]) + 1) // 2)
                   for rd in ro["trace"].rounds)
        prm = B.ransac_params(n_hyps=64, batch=500, seed=i)
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        dd = u16_dev(d)
        B.ransac_relocalise(gpu_forest, dd, u16_dev(leaves), intr, prm, _workspace(intr, prm), res)
        depth_a = torch.zeros_like(dd)
        B.verify(gpu_room, intr, dd, res, depth_a)
        torch.cuda.synchronize()
        r = B.result_from_bytes(res)
        assert r["status"] == 0 and r["n_valid"] == int((d > 0).sum())
        if not tied:
            assert r["hypothesis"] == ro["index"], i
        if r["hypothesis"] == ro["index"]:
            same += 1
            assert np.abs(r["pose"][:3] - ro["pose"][:3]).max() < 1e-4
            assert abs(r["energy"] - ro["energy"]) <= 1e-5 * abs(ro["energy"])
        dt, dr = oracle.pose_error(r["pose"], P)
        assert dt <= 0.05 and dr <= 5.0
        # verification counts are integer-exact given the GPU's own render of scene a
        da = u16_np(depth_a)
        counts = oracle.verify_counts(da, d)
        assert [r["omega"], r["omega_a"], r["omega_b"], r["omega_ab"], r["sum_absdiff_mm"]] == counts.tolist()
        assert bool(r["verified"]) == oracle.verify_accept(counts)
        assert r["verified"] == 1
    assert same >= 2


def test_ransac_degenerate_cases(room_forest, gpu_forest, gpu_room):
    intr = synth.Intrinsics.for_size(64, 48)
    d = np.zeros((48, 64), np.uint16)
    leaves = np.full((5, 48, 64), 0xFFFF, np.uint16)
    for K in (1, 7):
        prm = B.ransac_params(n_hyps=K, batch=16, seed=1, max_tries=100)
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        B.ransac_relocalise(gpu_forest, u16_dev(d), u16_dev(leaves), intr, prm, _workspace(intr, prm), res)
        B.verify(gpu_room, intr, u16_dev(d), res)
        torch.cuda.synchronize()
        r = B.result_from_bytes(res)
        assert r["status"] == B.ENOTFOUND and r["hypothesis"] == 0 and r["n_valid"] == 0
        assert r["verified"] == 0 and r["omega"] == 64 * 48 and r["omega_a"] == 0
    with pytest.raises(B.ReloError):
        prm = B.ransac_params(n_hyps=8, batch=16)
        tiny = torch.empty(16, dtype=torch.uint8, device=DEV)
        B.ransac_relocalise(gpu_forest, u16_dev(d), u16_dev(leaves), intr, prm, tiny,
                            torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV))


# ------------------------------------------------------------------------------------------------
# Batches: the batched launch equals the single-attempt calls
# ------------------------------------------------------------------------------------------------
def test_batch_equals_single_calls(room, gpu_room, gpu_forest, room_training):
    world, _ = room
    train = [f[1] for f in room_training]
    sizes = [(320, 240), (160, 120), (96, 72)]
    Ks = [64, 33, 16]
    qs = synth.query_poses(world, train, 3, seed=44)
    items = []
    for i, ((W, H), K, P) in enumerate(zip(sizes, Ks, qs)):
        intr = synth.Intrinsics.for_size(W, H)
        items.append(dict(scene_b=gpu_room, forest_a=gpu_forest, scene_a=gpu_room, intr=intr, pose_b=P,
                          noise=torch.from_numpy(synth.depth_noise(H, W, 70 + i)).to(DEV), n_hyps=K, seed=100 + i))
    prm = B.ransac_params(n_hyps=64, batch=200, seed=0)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    got = B.relocalise_batch(att, prm, ws)
    for it, g in zip(items, got):
        intr = it["intr"]
        depth = torch.zeros((intr.height, intr.width), dtype=torch.int16, device=DEV)
        rgba = torch.zeros((intr.height, intr.width, 4), dtype=torch.uint8, device=DEV)
        B.raycast_view(gpu_room, intr, it["pose_b"], depth, rgba, noise_dev=it["noise"])
        leaves = torch.zeros((5, intr.height, intr.width), dtype=torch.int16, device=DEV)
        B.forest_eval(gpu_forest, depth, rgba, leaves)
        p1 = B.ransac_params(n_hyps=it["n_hyps"], batch=200, seed=it["seed"])
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        B.ransac_relocalise(gpu_forest, depth, leaves, intr, p1, _workspace(intr, p1), res)
        B.verify(gpu_room, intr, depth, res)
        torch.cuda.synchronize()
        s = B.result_from_bytes(res)
        for k in ("hypothesis", "status", "n_inliers", "n_valid", "omega", "omega_a", "omega_b", "omega_ab",
                  "sum_absdiff_mm", "verified", "energy"):
            assert g[k] == s[k], k
        assert np.array_equal(g["pose"], s["pose"])
        rel = g["pose"] @ np.linalg.inv(it["pose_b"])
        assert np.abs(g["rel_a_b"] - rel).max() < 1e-9


def test_batch_prepared_replay_is_deterministic(room, gpu_room, gpu_forest, room_training):
    world, _ = room
    qs = synth.query_poses(world, [f[1] for f in room_training], 4, seed=45)
    intr = synth.Intrinsics.for_size(160, 120)
    items = [dict(scene_b=gpu_room, forest_a=gpu_forest, scene_a=gpu_room, intr=intr, pose_b=P, seed=i)
             for i, P in enumerate(qs)]
    prm = B.ransac_params(n_hyps=32, batch=100)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    bt = B.Batch(att, prm, ws)
    out1 = torch.zeros(4 * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    out2 = torch.zeros_like(out1)
    bt.run(out1)
    bt.run(out2)
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)
    # result init + query raycast, merge; forest pass: forest, compaction (2), search + fit, 5 rounds
    # of draw / energy / select / refine / refit, finalise, verification raycast + decision
    assert bt.launch_count == 2 + 1 + 1 + 2 + 2 + 5 * 5 + 1 + 2


# ------------------------------------------------------------------------------------------------
# Relocaliser training: reservoirs bit-exact, modes to FP32 tolerance
# ------------------------------------------------------------------------------------------------
def test_training_matches_oracle(room, oracle_room):
    world, _ = room
    intr = synth.Intrinsics.for_size(160, 120)
    train = synth.training_poses(world, 4, seed=12)
    nodes = synth.random_forest_nodes(3, 8, seed=6, depth_tau=100, colour_tau=32)
    lp = oracle.LeafParams(capacity=32, max_modes=8, seed=13, stride=2)
    r = oracle.Reservoirs(nodes, lp)
    f = B.Forest(nodes, max_modes=8)
    B.forest_train_begin(f, B.train_params(capacity=32, stride=2, seed=13))
    for i, P in enumerate(train):
        d, c = oracle_room.raycast(intr, P, noise=synth.depth_noise(120, 160, i))
        r.add_frame(intr, P, d, c)
        B.forest_train_frame(f, intr, P, u16_dev(d), torch.from_numpy(c).to(DEV))
    so, co = r.contents()
    sg, cg = B.forest_train_reservoirs(f, 32)
    assert np.array_equal(cg, co)
    assert np.array_equal(sg, so)
    B.forest_train_finish(f)
    mg, ng = f.get_modes()
    fo = r.modes()
    same = ng == fo.n_modes
    assert same.mean() >= 0.99
    k = np.arange(8)[None, None, :] < ng[..., None]
    sel = same[..., None] & k
    assert np.abs(mg[sel][:, :3] - fo.modes[sel][:, :3]).max() < 1e-4
    assert np.abs(mg[sel][:, 10] - fo.modes[sel][:, 10]).max() < 1e-6
