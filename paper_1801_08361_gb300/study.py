"""The collaborative pipeline on synthetic house fragments, measured the way the tables of
Sec. 4.2.3 (depth-difference verification) and Sec. 4.2.4 (relative transform clustering)
measure the paper's: for pairs of overlapping sub-scenes {a, b}, frames of each agent's
trajectory are relocalised against the other agent's scene (one batched launch), each proposed
relative transform is classified verified / rejected (Sec. 3.3.1) and correct / incorrect
(within 5 degrees and 5 cm of the known transform), the verified samples are clustered
(Sec. 3.3.2), and the largest cluster is compared with the largest cluster whose blend is not
within 20 degrees and 10 cm of it (the safety margin).  Then the pose graph is optimised and
its global poses compared with the fragments' true frames, the global map (Appendix B.2)
rendered with the optimised poses is compared with the render under the true poses, and the
agents' frames are fused into a single global model with the optimised poses (Appendix B.3).

Every GPU step runs in the library's kernels; this module only arranges inputs and counts.
Usage: python -m paper_1801_08361_gb300.study [--frames 64] [--fragments 8] [--json out.json]
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

W, H = 640, 480
TREES, DEPTH = 5, 15
CORRECT_DEG, CORRECT_M = 5.0, 0.05        # Sec. 4.2.3: "correct" within 5 degrees and 5 cm
CLUSTER_DEG, CLUSTER_M = 20.0, 0.10       # Sec. 4.2.4


def rel_error(T, T_true):
    """(rotation error in degrees, translation error in metres) of T against T_true."""
    c = (np.trace(T[:3, :3] @ T_true[:3, :3].T) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c)))), float(np.linalg.norm(T[:3, 3] - T_true[:3, 3]))


def within(T, T_ref, deg, metres):
    r, t = rel_error(T, T_ref)
    return r <= deg and t <= metres


def build_fragments(n_fragments, seed=3, train_per_room=12, capacity=1024, dev=None):
    """Fragments of the 10 x 8 x 3 m house, each sampled in its own frame, with a forest trained
    on the GPU from noisy renders of its own trajectory."""
    import torch
    from . import binding as B
    from . import synth
    world = synth.house_world(2)
    frags = synth.house_fragments(world, n_fragments, seed=seed)
    intr = synth.Intrinsics.for_size(W, H, 12.0)
    depth = torch.zeros((H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((H, W, 4), dtype=torch.uint8, device=dev)

    def sample(f):
        return synth.sample_scene(world, scene_to_world=f["scene_to_world"], crop=f["crop"])

    with ThreadPoolExecutor(4) as ex:           # the sampler is C code run without the GIL
        for k, blocks in enumerate(ex.map(sample, frags)):
            f = frags[k]
            f["scene"] = B.Scene(blocks, 19)
            del blocks
            f["train_w"] = synth.training_poses(world, train_per_room, seed=40 + k, rooms=f["rooms"])
            nodes = synth.random_forest_nodes(TREES, DEPTH, seed=60 + k, depth_tau=100, colour_tau=32)
            f["forest"] = B.Forest(nodes, max_modes=10)
            B.forest_train_begin(f["forest"], B.train_params(capacity=capacity, stride=2, seed=k))
            for i, Pw in enumerate(f["train_w"]):
                P = synth.world_to_scene_pose(Pw, f["scene_to_world"])
                nz = torch.from_numpy(synth.depth_noise(H, W, 7000 + 100 * k + i)).to(dev)
                B.raycast_view(f["scene"], intr, P, depth, rgba, noise_dev=nz)
                B.forest_train_frame(f["forest"], intr, P, depth, rgba)
            B.forest_train_finish(f["forest"])
    return world, frags, intr


def overlapping_pairs(frags, limit=8):
    """Unordered pairs of fragments that share a room (the paper's pairs overlap too)."""
    pairs = [(a, b) for a, b in itertools.combinations(range(len(frags)), 2)
             if set(frags[a]["rooms"]) & set(frags[b]["rooms"])]
    return pairs[:limit]


def true_rel(frags, a, b):
    """aT_b: scene b -> scene a."""
    return np.linalg.inv(frags[a]["scene_to_world"]) @ frags[b]["scene_to_world"]


def run(n_fragments=8, frames=64, n_pairs=8, seed=3, n_views=4, dev=None, log=print):
    import torch
    from . import binding as B
    from . import synth
    t0 = time.time()
    world, frags, intr = build_fragments(n_fragments, seed=seed, dev=dev)
    log(f"fragments built in {time.time() - t0:.0f} s")
    pairs = overlapping_pairs(frags, n_pairs)
    rng = np.random.default_rng(seed + 100)
    # every frame of b's trajectory (a perturbed copy of it) against a, and the other way round
    items, meta = [], []
    for a0, b0 in pairs:
        for a, b in ((a0, b0), (b0, a0)):
            for Pw in synth.query_poses(world, frags[b]["train_w"], frames, seed=int(rng.integers(1 << 30))):
                items.append(dict(scene_b=frags[b]["scene"], forest_a=frags[a]["forest"], scene_a=frags[a]["scene"],
                                  intr=intr, pose_b=synth.world_to_scene_pose(Pw, frags[b]["scene_to_world"]),
                                  seed=int(rng.integers(1 << 40))))
                meta.append((a, b))
    prm = B.ransac_params(n_hyps=1024, batch=64, max_tries=10000)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
    bt = B.Batch(att, prm, ws)
    out = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bt.run(out)
    e1.record()
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1)
    raw = out.cpu()
    results = [B.result_from_bytes(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES]) for k in range(len(items))]

    # verification table (Sec. 4.2.3) and clustering (Sec. 3.3.2) per unordered pair
    graph = B.PoseGraph(n_fragments)
    verifier, clustering = [], []
    per_pair = {p: dict(total=0, reloc=0, tp=0, fp=0, tn=0, fn=0) for p in pairs}
    order = sorted(range(len(items)), key=lambda k: (k % frames, k))   # interleave the pairs' streams
    for k in order:
        a, b = meta[k]
        key = (min(a, b), max(a, b))
        r, c = results[k], per_pair[key]
        c["total"] += 1
        if r["status"] != 0:
            continue
        c["reloc"] += 1
        correct = within(r["rel_a_b"], true_rel(frags, a, b), CORRECT_DEG, CORRECT_M)
        ver = bool(r["verified"])
        c["tp" if ver and correct else "fp" if ver else "fn" if correct else "tn"] += 1
        if ver:
            graph.add_sample(a, b, r["rel_a_b"])
    for (a, b), c in per_pair.items():
        prec = c["tp"] / max(1, c["tp"] + c["fp"])
        rec = c["tp"] / max(1, c["tp"] + c["fn"])
        spec = c["tn"] / max(1, c["tn"] + c["fp"])
        verifier.append(dict(pair=f"{a}-{b}", total=c["total"], relocalised=c["reloc"], tp=c["tp"], fp=c["fp"],
                             tn=c["tn"], fn=c["fn"], precision=prec, recall=rec, specificity=spec))
        sizes = graph.cluster_sizes(a, b)
        added = sum(sizes)
        if not sizes:
            clustering.append(dict(pair=f"{a}-{b}", samples=0, correct=0, incorrect=0, margin=0, largest_ok=None))
            continue
        big = int(np.argmax(sizes))
        ref = graph.cluster_blend(a, b, big)
        wrong = [s for c2, s in enumerate(sizes)
                 if c2 != big and not within(graph.cluster_blend(a, b, c2), ref, CLUSTER_DEG, CLUSTER_M)]
        inc = max(wrong, default=0)
        clustering.append(dict(pair=f"{a}-{b}", samples=added, correct=sizes[big], incorrect=inc,
                               margin=sizes[big] - inc,
                               largest_ok=within(ref, true_rel(frags, a, b), CORRECT_DEG, CORRECT_M)))

    # pose graph (Sec. 3.3.2) against the true frames, with fragment 0 as the gauge
    poses, in_graph, eps = graph.optimise()
    S0_inv = np.linalg.inv(frags[0]["scene_to_world"])
    pg = []
    for s in range(n_fragments):
        if in_graph[s]:
            r_deg, t_m = rel_error(poses[s], S0_inv @ frags[s]["scene_to_world"])
            pg.append(dict(scene=s, rot_deg=r_deg, trans_m=t_m))

    # global map (Appendix B.2) with the optimised poses vs the true poses, over the graph's scenes
    render = None
    members = [s for s in range(n_fragments) if in_graph[s]]
    if len(members) >= 2:
        views = synth.query_poses(world, sum((frags[s]["train_w"] for s in members), []), n_views, seed=seed + 7)
        sc = [frags[s]["scene"] for s in members]
        diffs, valid_opt, valid_true, render_ms = [], 0, 0, []
        rgba = torch.zeros((H, W, 4), dtype=torch.uint8, device=dev)
        wsr = torch.empty(B.render_global_workspace_size(len(sc)), dtype=torch.uint8, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for Pw in views:
            Pg = S0_inv @ Pw                       # the camera in fragment 0's frame (the global frame)
            outs = []
            for g in ([poses[s] for s in members], [S0_inv @ frags[s]["scene_to_world"] for s in members]):
                d = torch.zeros((H, W), dtype=torch.int16, device=dev)
                o = torch.zeros((H, W), dtype=torch.int8, device=dev)
                e0.record()
                B.render_global(sc, g, intr, Pg, d, rgba, o, workspace_dev=wsr)
                e1.record()
                torch.cuda.synchronize()
                render_ms.append(e0.elapsed_time(e1))
                outs.append((d.cpu().numpy().view(np.uint16), o.cpu().numpy()))
            (d_opt, _), (d_true, _) = outs
            both = (d_opt > 0) & (d_true > 0)
            valid_opt += int((d_opt > 0).sum())
            valid_true += int((d_true > 0).sum())
            diffs.append(np.abs(d_opt[both].astype(np.int64) - d_true[both]))
        diffs = np.concatenate(diffs) if diffs else np.zeros(0, np.int64)
        n = max(1, diffs.size)
        render = dict(views=n_views, scenes=members, pixels=int(diffs.size), ms_per_view=float(np.median(render_ms)),
                      median_abs_diff_mm=float(np.median(diffs)) if diffs.size else None,
                      depth_within_1cm=float((diffs <= 10).sum() / n), depth_within_5cm=float((diffs <= 50).sum() / n),
                      valid_ratio=valid_opt / max(1, valid_true))

    # the single global model (Appendix B.3): every graph member's trajectory frames, re-rendered
    # from its own scene, fused into one scene with their poses moved by the member's global pose;
    # compared with the global map of the true poses from the same views
    fused = None
    if len(members) >= 2:
        fs = B.FusionScene(1 << 21, synth.VOXEL_SIZE, synth.TRUNCATION, log2_buckets=21)
        seq = [(s_, synth.world_to_scene_pose(Pw, frags[s_]["scene_to_world"]))
               for s_ in members for Pw in frags[s_]["train_w"][::2]]
        n_frames = len(seq)
        depth = torch.zeros((n_frames, H, W), dtype=torch.int16, device=dev)
        rgba = torch.zeros((n_frames, H, W, 4), dtype=torch.uint8, device=dev)
        for k, (s_, P) in enumerate(seq):       # the agents' saved sequences, re-rendered
            B.raycast_view(frags[s_]["scene"], intr, P, depth[k], rgba[k])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fs.fuse_many(intr, [poses[s_] @ P for s_, P in seq], depth, rgba)
        e1.record()
        torch.cuda.synchronize()
        fuse_ms = e0.elapsed_time(e1)
        diffs = []
        for Pw in views:
            Pg = S0_inv @ Pw
            d_f = torch.zeros((H, W), dtype=torch.int16, device=dev)
            B.raycast_view(fs, intr, Pg, d_f)
            d_t = torch.zeros((H, W), dtype=torch.int16, device=dev)
            B.render_global(sc, [S0_inv @ frags[s]["scene_to_world"] for s in members], intr, Pg, d_t)
            torch.cuda.synchronize()
            a, b = d_f.cpu().numpy().view(np.uint16), d_t.cpu().numpy().view(np.uint16)
            both = (a > 0) & (b > 0)
            diffs.append(np.abs(a[both].astype(np.int64) - b[both]))
        diffs = np.concatenate(diffs) if diffs else np.zeros(0, np.int64)
        k = max(1, diffs.size)
        fused = dict(frames=n_frames, blocks=fs.block_count(), fuse_ms_per_frame=fuse_ms / max(1, n_frames),
                     median_abs_diff_mm=float(np.median(diffs)) if diffs.size else None,
                     depth_within_1cm=float((diffs <= 10).sum() / k), depth_within_5cm=float((diffs <= 50).sum() / k))
    return dict(attempts=len(items), batch_ms=batch_ms, pairs=[f"{a}-{b}" for a, b in pairs],
                verifier=verifier, clustering=clustering, pose_graph=dict(epsilon=eps, scenes=pg), render=render,
                fused=fused)


def markdown(rep) -> str:
    lines = ["| pair | frames | relocalised | TP | FP | TN | FN | precision | recall | specificity |",
             "|---|---|---|---|---|---|---|---|---|---|"]
    for r in rep["verifier"]:
        lines.append(f"| {r['pair']} | {r['total']} | {r['relocalised']} | {r['tp']} | {r['fp']} | {r['tn']} | "
                     f"{r['fn']} | {100 * r['precision']:.1f} % | {100 * r['recall']:.1f} % | "
                     f"{100 * r['specificity']:.1f} % |")
    lines += ["", "| pair | samples added | largest cluster | largest incorrect | safety margin | largest within 5 cm / 5 deg |",
              "|---|---|---|---|---|---|"]
    for r in rep["clustering"]:
        lines.append(f"| {r['pair']} | {r['samples']} | {r['correct']} | {r['incorrect']} | {r['margin']} | "
                     f"{r['largest_ok']} |")
    lines += ["", "| scene | rotation error (deg) | translation error (m) |", "|---|---|---|"]
    for r in rep["pose_graph"]["scenes"]:
        lines.append(f"| {r['scene']} | {r['rot_deg']:.3f} | {r['trans_m']:.4f} |")
    if rep["render"]:
        r = rep["render"]
        lines.append(f"\nGlobal map of scenes {r['scenes']} ({r['ms_per_view']:.3f} ms per {W}x{H} view, colour "
                     f"and owner included), optimised vs true poses over {r['views']} views: median "
                     f"|depth difference| {r['median_abs_diff_mm']} mm; within 1 cm on {100 * r['depth_within_1cm']:.1f} %, "
                     f"within 5 cm on {100 * r['depth_within_5cm']:.1f} % of the pixels both renders hit.")
    if rep.get("fused"):
        f = rep["fused"]
        lines.append(f"\nSingle global model (Appendix B.3): {f['frames']} frames fused with the optimised global poses "
                     f"into {f['blocks']} blocks ({f['fuse_ms_per_frame']:.3f} ms per frame); against the global map of "
                     f"the true poses: median |depth difference| {f['median_abs_diff_mm']} mm, within 1 cm on "
                     f"{100 * f['depth_within_1cm']:.1f} %, within 5 cm on {100 * f['depth_within_5cm']:.1f} %.")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--fragments", type=int, default=8)
    ap.add_argument("--frames", type=int, default=64, help="frames per agent and direction")
    ap.add_argument("--pairs", type=int, default=8)
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    rep = run(args.fragments, args.frames, args.pairs, dev=torch.device("cuda:0"),
              log=lambda m: print(m, file=sys.stderr, flush=True))
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rep, f, indent=1)
    print(markdown(rep))
    return 0


if __name__ == "__main__":
    sys.exit(main())
