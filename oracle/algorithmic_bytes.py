"""Algorithmic bytes of the raycast stages on the paper-sized house workload (oracle count).

Prints, per query pixel, the distinct bytes the method must read or write once: for the query
render, the tsdf (4 B) and colour (4 B) voxels its samples touch, one 16-byte hash entry per
distinct block looked up, the noise value read (4 B) and the depth (2 B) + colour (4 B)
written; for the verification render (depth only, from the query pose), tsdf voxels, hash
entries and the reference depth read (2 B).  Averaged over 8 query views of the workload.
With ``fragments``: the same counts summed over the 56 attempts of the batched workload (8 house
fragments, every ordered pair, mixed sizes; the verification render from the query's pose in
a's frame), with each attempt's 16 B per pixel of the forest stage (depth and colour read, 5
leaf ids written) beside them.
Calls only the oracle and the seeded input generators.
Run: python -m oracle.algorithmic_bytes [n_views] | python -m oracle.algorithmic_bytes fragments
"""
import sys

import numpy as np


def main(n_views: int = 8):
    import oracle
    from paper_1801_08361_gb300 import synth
    world = synth.house_world(2)
    blocks = synth.sample_scene(world)
    sc = oracle.Scene(blocks)
    intr = synth.Intrinsics.for_size(640, 480, 12.0)
    train = synth.training_poses(world, 16, seed=11)
    qs = synth.query_poses(world, train, n_views, seed=1000)
    n_pix = intr.width * intr.height
    q_bytes, v_bytes = [], []
    for P in qs:
        t = oracle.raycast_touched(sc, intr, P, with_colour=True)
        q_bytes.append((4 * t["tsdf_voxels"] + 4 * t["colour_voxels"] + 16 * t["block_keys"]) / n_pix + 4 + 6)
        t = oracle.raycast_touched(sc, intr, P, with_colour=False)
        v_bytes.append((4 * t["tsdf_voxels"] + 16 * t["block_keys"]) / n_pix + 2)
        print(f"view: query {q_bytes[-1]:.2f} B/px, verification {v_bytes[-1]:.2f} B/px", flush=True)
    print(f"query_raycast {np.mean(q_bytes):.2f} B/px  verify_raycast {np.mean(v_bytes):.2f} B/px")


def fragments(seed: int = 17):
    import oracle
    from paper_1801_08361_gb300 import synth
    sizes = [(320, 240), (480, 360), (640, 480)]
    world = synth.house_world(2)
    frags = synth.house_fragments(world, 8, seed=3)
    synth.fragment_trajectories(world, frags, 12)
    pairs = synth.fragment_pairs(world, frags, sizes, seed=seed)
    scenes = [oracle.Scene(synth.sample_scene(world, scene_to_world=f["scene_to_world"], crop=f["crop"]))
              for f in frags]
    q = v = px = 0
    for p in pairs:
        intr = synth.Intrinsics.for_size(p["width"], p["height"], 12.0)
        n = p["width"] * p["height"]
        t = oracle.raycast_touched(scenes[p["b"]], intr, p["pose_b"], with_colour=True)
        q += 4 * t["tsdf_voxels"] + 4 * t["colour_voxels"] + 16 * t["block_keys"] + 10 * n
        t = oracle.raycast_touched(scenes[p["a"]], intr, p["pose_a"], with_colour=False)
        v += 4 * t["tsdf_voxels"] + 16 * t["block_keys"] + 2 * n
        px += n
        print(f"pair {p['a']}-{p['b']} {p['width']}x{p['height']}: query {q / px:.2f} B/px, verification "
              f"{v / px:.2f} B/px so far", flush=True)
    print(f"batch of {len(pairs)}: pixels {px}, query_raycast {q} B, forest_eval {16 * px} B, verify_raycast {v} B")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "fragments":
        fragments()
    else:
        main(int(sys.argv[1]) if len(sys.argv) > 1 else 8)
