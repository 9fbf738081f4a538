"""End-to-end oracle attempt on the tiny room (Sec. 3.3.1, Fig. 3): a view of the room rendered
near the training trajectory relocalises to within 5 cm / 5 degrees (the paper's success
criterion, Sec. 4.2.2) and passes depth-difference verification; a wrong pose is rejected."""
import math

import numpy as np
import pytest

import oracle
from paper_1801_08361_gb300 import synth


@pytest.fixture(scope="module")
def tiny_forest(room_training, room_forest):
    return room_forest, [f[1] for f in room_training]


def test_tiny_room_attempts_succeed_and_verify(room, oracle_room, tiny_forest):
    world, _ = room
    forest, train = tiny_forest
    intr = synth.Intrinsics.for_size(320, 240)
    q = synth.query_poses(world, train, 3, seed=3)
    for i, P in enumerate(q):
        res = oracle.relocalise(oracle_room, P, forest, oracle_room, intr,
                                oracle.RansacParams(n_hyps=64, batch=500, seed=i))
        dt, dr = oracle.pose_error(res["pose"], P)
        assert dt <= 0.05 and dr <= 5.0
        assert res["verified"]
        rel = res["rel_a_b"]                  # a = b here: the sample is close to identity
        assert np.abs(rel - np.eye(4)).max() < 0.1


def test_wrong_pose_is_rejected(room, oracle_room):
    world, _ = room
    intr = synth.Intrinsics.for_size(160, 120)
    P = synth.look_pose(np.array([2.0, 2.0, 1.5]), 0.4, 0.0)
    Q = synth.look_pose(np.array([2.0, 2.0, 1.5]), 0.4 + math.radians(40), 0.0)
    db, _ = oracle_room.raycast(intr, P)
    da, _ = oracle_room.raycast(intr, Q)
    assert not oracle.verify_accept(oracle.verify_counts(da, db))
    assert oracle.verify_accept(oracle.verify_counts(db, db))
