"""GPU parity at the benchmark's configuration: a 640 x 480 noisy query of the 10 x 8 x 3 m house,
a forest of 5 trees of depth 15 (reservoirs of 1024, <= 10 modes), preemptive RANSAC with 1024
hypotheses and 64 pixels per round (10 rounds).

The forest's leaves are filled by the oracle from renders of the house at every training pose
(the benchmark's trajectory and noise seeds; every 8th pixel of every 8th row, which keeps the
oracle's mean shift to tens of seconds) and handed to the library, so both sides search the same
modes.  Bars: leaves and the hypothesis set bit-exact, hypothesis poses 1e-9, every round's draws
exact, energies 1e-5 relative, survivors exact outside near-ties, re-fits 1e-4 (teacher-forced:
each GPU round starts from the oracle's state), and the untouched end-to-end RANSAC equal to the
oracle's when no round had a near-tie."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth
from paper_1801_08361_gb300.presets import HOUSE

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
W, H = HOUSE.sizes[0]
K, BPIX = HOUSE.hypotheses[0], HOUSE.batch_pixels
ORACLE_STRIDE = 8


def _u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(DEV)


@pytest.fixture(scope="module")
def house():
    world = synth.house_world(2)
    blocks = synth.sample_scene(world)
    sc = oracle.Scene(blocks)
    intr = synth.Intrinsics.for_size(W, H, 12.0)
    train = synth.training_poses(world, HOUSE.train_per_room, seed=11)
    nodes = synth.random_forest_nodes(HOUSE.trees, HOUSE.depth, seed=5, depth_tau=100, colour_tau=32)
    threads = max(1, min(16, os.cpu_count() or 1))

    def render(i):     # the oracle's C raycast releases the GIL
        return sc.raycast(intr, train[i], noise=synth.depth_noise(H, W, 100 + i))

    with ThreadPoolExecutor(threads) as ex:
        imgs = list(ex.map(render, range(len(train))))
    frames = [(intr, P, d, c) for P, (d, c) in zip(train, imgs)]
    forest = oracle.train_forest(nodes, frames, oracle.LeafParams(capacity=HOUSE.reservoir, max_modes=HOUSE.max_modes,
                                                                  seed=7, stride=ORACLE_STRIDE), threads=threads)
    P = synth.query_poses(world, train, 1, seed=2024)[0]
    d, c = sc.raycast(intr, P, noise=synth.depth_noise(H, W, 31))
    leaves = oracle.forest_eval(nodes, d, c)
    gforest = B.Forest(nodes, forest.modes, forest.n_modes, max_modes=HOUSE.max_modes)
    prm_o = oracle.RansacParams(n_hyps=K, batch=BPIX, seed=9)
    res = oracle.preemptive_ransac(d, intr, leaves, forest, prm_o, trace=True)
    return dict(intr=intr, P=P, d=d, c=c, nodes=nodes, forest=forest, gforest=gforest, leaves=leaves, res=res,
                prm_o=prm_o)


def _workspace(intr, prm):
    return torch.empty(B.ransac_workspace_size(intr.width, intr.height, prm), dtype=torch.uint8, device=DEV)


def _near_tie(E, alive, keep):
    srt = sorted(alive.tolist(), key=lambda h: (E[h], h))
    if keep >= len(srt):
        return False
    a, b = E[srt[keep - 1]], E[srt[keep]]
    if not (np.isfinite(a) and np.isfinite(b)):
        return False
    return abs(b - a) <= 1e-5 * max(abs(a), abs(b)) + 1e-6


def test_house_leaves_and_hypotheses_bit_exact(house):
    intr, d, c = house["intr"], house["d"], house["c"]
    dd = _u16(d)
    rgba = torch.from_numpy(np.ascontiguousarray(c)).to(DEV)
    leaves = torch.zeros((HOUSE.trees, H, W), dtype=torch.int16, device=DEV)
    B.forest_eval(house["gforest"], dd, rgba, leaves)
    prm = B.ransac_params(n_hyps=K, batch=BPIX, seed=9)
    poses = torch.zeros((K, 12), dtype=torch.float64, device=DEV)
    valid = torch.zeros(K, dtype=torch.int32, device=DEV)
    tries = torch.zeros(K, dtype=torch.int32, device=DEV)
    B.ransac_hypotheses(house["gforest"], dd, leaves, intr, prm, _workspace(intr, prm), poses, valid, tries)
    torch.cuda.synchronize()
    assert np.array_equal(leaves.cpu().numpy().view(np.uint16), house["leaves"])
    tr = house["res"]["trace"]
    ok = valid.cpu().numpy().astype(bool)
    assert np.array_equal(ok, tr.valid0)
    assert tr.valid0.sum() >= K // 8
    pg = poses.cpu().numpy().reshape(K, 3, 4)
    assert np.abs(pg[ok] - tr.poses0[ok, :3, :]).max() < 1e-9


def _refit_is_ill_posed(pose_in, cam, drawn, leaves, forest, inlier_dist):
    """True when the oracle's own re-fit moves by more than 1e-5 if its camera points are rounded
    to FP32 (the precision the library holds them in): then the re-fit is not determined at the
    pose tolerance.  This happens for inlier sets of rank one -- pixels are drawn with
    replacement, so "three inliers" can be two distinct points, whose rotation about their line is
    arbitrary."""
    _, mu, found, x = oracle.pixel_energies(pose_in, cam, drawn, leaves, forest)
    dist = np.where(found, np.linalg.norm(x - mu, axis=1), np.inf)
    m = dist < inlier_dist
    if m.sum() < 3:
        return False
    R0, t0 = oracle.kabsch(cam[m], mu[m])
    R1, t1 = oracle.kabsch(cam[m].astype(np.float32).astype(np.float64), mu[m])
    return max(np.abs(R1 - R0).max(), np.abs(t1 - t0).max()) > 1e-5


def test_house_rounds_teacher_forced(house):
    """Each of the 10 rounds on the GPU starts from the oracle's state (alive set, poses, energies,
    earlier draws) and must reproduce the oracle's draws, energies, survivors, inlier counts and
    re-fits (re-fits that FP32 rounding of the oracle's own inputs moves beyond the tolerance are
    not compared)."""
    intr, d, leaves_o, forest = house["intr"], house["d"], house["leaves"], house["forest"]
    tr = house["res"]["trace"]
    prm = B.ransac_params(n_hyps=K, batch=BPIX, seed=9)
    ws = _workspace(intr, prm)
    dd, ld = _u16(d), _u16(leaves_o)
    valid = torch.from_numpy(tr.valid0.astype(np.int32)).to(DEV)
    poses_prev = tr.poses0[:, :3, :].copy()
    E_prev = np.where(tr.valid0, 0.0, np.inf)
    drawn_prev = np.zeros(0, np.int64)
    vpix = oracle.valid_pixels(d)
    strict_rounds = refits = ill_posed = 0
    assert len(tr.rounds) == 10
    for r, rd in enumerate(tr.rounds):
        alive = rd["alive_before"]
        keep = (len(alive) + 1) // 2
        poses = torch.from_numpy(poses_prev.reshape(K, 12).copy()).to(DEV)
        energy = torch.from_numpy(E_prev.copy()).to(DEV)
        drawn = torch.zeros((r + 1) * BPIX, dtype=torch.int32, device=DEV)
        drawn[: r * BPIX] = torch.from_numpy(np.searchsorted(vpix, drawn_prev).astype(np.int32)).to(DEV)
        surv = torch.zeros(keep, dtype=torch.int32, device=DEV)
        inl = torch.zeros(K, dtype=torch.int32, device=DEV)
        if r > 0:
            inl.copy_(torch.from_numpy(tr.rounds[r - 1]["inliers"].astype(np.int32)))
        B.ransac_round(house["gforest"], dd, ld, intr, prm, r, torch.from_numpy(alive.astype(np.int32)).to(DEV), valid,
                       poses, energy, drawn, surv, inl, ws)
        torch.cuda.synchronize()
        assert np.array_equal(vpix[drawn.cpu().numpy()[r * BPIX:]], rd["pixels"])
        Eg, Eo = energy.cpu().numpy(), rd["energy"]
        fin = np.isfinite(Eo[alive])
        assert np.array_equal(np.isfinite(Eg[alive]), fin)
        rel = np.abs(Eg[alive][fin] - Eo[alive][fin]) / np.maximum(np.abs(Eo[alive][fin]), 1.0)
        assert rel.max() <= 1e-5, (r, rel.max())
        sg = surv.cpu().numpy()
        if not _near_tie(Eo, alive, keep):
            assert np.array_equal(sg, rd["survivors"]), r
            strict_rounds += 1
        all_drawn = np.concatenate([drawn_prev, rd["pixels"]])
        cam = oracle.camera_points(d, intr, all_drawn)
        pg = poses.cpu().numpy().reshape(K, 3, 4)
        ig = inl.cpu().numpy()
        for h in set(sg.tolist()) & set(rd["survivors"].tolist()):
            if not tr.valid0[h]:
                continue
            pose_in = np.eye(4)
            pose_in[:3, :] = poses_prev[h]
            dm, am = oracle.decision_margins(pose_in, cam, all_drawn, leaves_o, forest, house["prm_o"].inlier_dist)
            if dm.min() < 1e-4 or am.min() < 1e-3:
                continue
            assert ig[h] == rd["inliers"][h], (r, h)
            if _refit_is_ill_posed(pose_in, cam, all_drawn, leaves_o, forest, house["prm_o"].inlier_dist):
                ill_posed += 1
                continue
            assert np.abs(pg[h] - rd["poses"][h][:3, :]).max() < 1e-4, (r, h)
            refits += 1
        poses_prev = rd["poses"][:, :3, :].copy()
        E_prev = rd["energy"].copy()
        drawn_prev = all_drawn
    assert strict_rounds >= len(tr.rounds) - 1
    assert refits >= 100 and ill_posed <= refits // 20, (refits, ill_posed)


def test_house_relocalise_matches_oracle_end_to_end(house):
    """relo_ransac_relocalise on the same inputs, no teacher forcing: when no round of the
    oracle's run had a near-tie, the same final hypothesis, its pose within 1e-4 and its energy
    within 1e-5 relative; either way the oracle's pose relocalises the query."""
    intr, d, P = house["intr"], house["d"], house["P"]
    ro = house["res"]
    prm = B.ransac_params(n_hyps=K, batch=BPIX, seed=9)
    res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    B.ransac_relocalise(house["gforest"], _u16(d), _u16(house["leaves"]), intr, prm, _workspace(intr, prm), res)
    torch.cuda.synchronize()
    r = B.result_from_bytes(res)
    assert r["status"] == 0 and ro["valid"]
    assert r["n_valid"] == int((d > 0).sum())
    dt, dr = oracle.pose_error(ro["pose"], P)
    assert dt <= 0.05 and dr <= 5.0
    tr = ro["trace"]
    ties = any(_near_tie(rd["energy"], rd["alive_before"], (len(rd["alive_before"]) + 1) // 2) for rd in tr.rounds)
    if not ties:
        assert r["hypothesis"] == ro["index"]
        assert np.abs(r["pose"][:3] - ro["pose"][:3]).max() < 1e-4
        assert abs(r["energy"] - ro["energy"]) <= 1e-5 * abs(ro["energy"])
