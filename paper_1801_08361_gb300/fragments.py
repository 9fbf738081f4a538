"""The batched workload: 8 sub-scenes cut from the 10 x 8 x 3 m house (1 to 3 rooms each, 13-40 m^2
of floor, each in its own random rigid frame, so that every relative transform aT_b is known),
each with a forest (5 trees of depth 13, reservoirs of 512, <= 10 modes) trained on the GPU from
noisy renders of its own trajectory, and all 56 ordered pairs (a, b) as one batch of attempts:
query sizes drawn from 320 x 240, 480 x 360 and 640 x 480, hypothesis counts from 256-1024.

Every GPU step runs in the library's kernels; this module only arranges seeded inputs (the same
for the tests and the benchmark).
"""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np

SIZES = [(320, 240), (480, 360), (640, 480)]
N_FRAG = 8
TREES, DEPTH, RESERVOIR, MAX_MODES = 5, 13, 512, 10
TRAIN_PER_ROOM = 12
LOG2_BUCKETS = 19
BATCH_PIXELS, MAX_TRIES = 64, 10000


def build(dev, keep_blocks=()):
    """(world, frags, scenes, forests, blocks): the fragments sampled in their own frames, their
    device scenes and GPU-trained forests; blocks[k] holds fragment k's host blocks for k in
    keep_blocks (None otherwise).  Each training frame is rendered at all three query sizes: a
    feature's pixel offsets are divided by depth but not scaled by the focal length, so a forest
    trained at one image size sees other responses at another."""
    import torch

    from . import binding as B
    from . import synth
    world = synth.house_world(2)
    frags = synth.house_fragments(world, N_FRAG, seed=3)
    synth.fragment_trajectories(world, frags, TRAIN_PER_ROOM)

    def sample(f):
        return synth.sample_scene(world, scene_to_world=f["scene_to_world"], crop=f["crop"])

    scenes, forests, kept = [], [], [None] * N_FRAG
    views = []
    for W, H in SIZES:
        views.append((synth.Intrinsics.for_size(W, H, 12.0), torch.zeros((H, W), dtype=torch.int16, device=dev),
                      torch.zeros((H, W, 4), dtype=torch.uint8, device=dev)))
    with ThreadPoolExecutor(4) as ex:           # the sampler is C code called without the GIL
        for k, blocks in enumerate(ex.map(sample, frags)):
            sc = B.Scene(blocks, LOG2_BUCKETS)
            if k in keep_blocks:
                kept[k] = blocks
            del blocks
            f = frags[k]
            S = f["scene_to_world"]
            f["nodes"] = synth.random_forest_nodes(TREES, DEPTH, seed=60 + k, depth_tau=100, colour_tau=32)
            fo = B.Forest(f["nodes"], max_modes=MAX_MODES)
            B.forest_train_begin(fo, B.train_params(capacity=RESERVOIR, stride=2, seed=k))
            for i, Pw in enumerate(f["train_w"]):
                P = synth.world_to_scene_pose(Pw, S)
                for j, (intr, depth, rgba) in enumerate(views):
                    nz = torch.from_numpy(synth.depth_noise(intr.height, intr.width, 7000 + 100 * k + 3 * i + j)).to(dev)
                    B.raycast_view(sc, intr, P, depth, rgba, noise_dev=nz)
                    B.forest_train_frame(fo, intr, P, depth, rgba)
            B.forest_train_finish(fo)
            scenes.append(sc)
            forests.append(fo)
    return world, frags, scenes, forests, kept


def pairs(world, frags, scenes, forests, dev, seed=17):
    """The 56 ordered pairs: the query of (a, b) is a perturbed view of b's trajectory with depth
    noise, relocalised with a's forest and verified against a.  Returns (items for
    binding.make_attempts, meta: a, b, the query's pose in a's frame, whether its room lies in a)."""
    import torch

    from . import synth
    items, meta = [], []
    for p in synth.fragment_pairs(world, frags, SIZES, seed=seed):
        a, b, W, H = p["a"], p["b"], p["width"], p["height"]
        noise = torch.from_numpy(synth.depth_noise(H, W, p["noise_seed"])).to(dev)
        items.append(dict(scene_b=scenes[b], forest_a=forests[a], scene_a=scenes[a],
                          intr=synth.Intrinsics.for_size(W, H, 12.0), pose_b=p["pose_b"], noise=noise,
                          n_hyps=p["n_hyps"], seed=p["seed"]))
        meta.append(dict(a=a, b=b, pose_a=p["pose_a"], covered=p["covered"]))
    return items, meta
