"""Algorithmic bytes of the raycast stages on the paper-sized house workload (oracle count).

Prints, per query pixel, the distinct bytes the method must read or write once: for the query
render, the tsdf (4 B) and colour (4 B) voxels its samples touch, one 16-byte hash entry per
distinct block looked up, the noise value read (4 B) and the depth (2 B) + colour (4 B)
written; for the verification render (depth only, from the query pose), tsdf voxels, hash
entries and the reference depth read (2 B).  Averaged over 8 query views of the workload.
Calls only the oracle and the seeded input generators.  Run: python -m oracle.algorithmic_bytes
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


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 8)
