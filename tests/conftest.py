"""Shared fixtures.  Tests marked ``gpu`` need a GB300 and the built CUDA library."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built relocalisation library")


def pytest_runtest_setup(item):
    if item.get_closest_marker("gpu") is not None:
        import torch
        if not torch.cuda.is_available():
            pytest.skip("no CUDA device")


@pytest.fixture(scope="session")
def room():
    """Tiny workload: 4 x 4 x 3 m room with 20 boxes, 5 mm voxels (seed 1)."""
    from paper_1801_08361_gb300 import synth
    world = synth.room_world(1)
    return world, synth.sample_scene(world)


@pytest.fixture(scope="session")
def oracle_room(room):
    import oracle
    return oracle.Scene(room[1])


@pytest.fixture(scope="session")
def room_training(room, oracle_room):
    """Ten noisy 320 x 240 training renders of the tiny room and their poses (oracle renders)."""
    from paper_1801_08361_gb300 import synth
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    train = synth.training_poses(world, 10, seed=11)
    frames = []
    for i, P in enumerate(train):
        d, c = oracle_room.raycast(intr, P, noise=synth.depth_noise(240, 320, 100 + i))
        frames.append((intr, P, d, c))
    return frames


@pytest.fixture(scope="session")
def room_forest(room_training):
    """Tiny-workload forest (5 trees, depth 10, reservoirs of 64, <= 10 modes) filled by the oracle."""
    import oracle
    from paper_1801_08361_gb300 import synth
    nodes = synth.random_forest_nodes(5, 10, seed=5, depth_tau=100, colour_tau=32)
    return oracle.train_forest(nodes, room_training, oracle.LeafParams(capacity=64, max_modes=10, seed=7))


def pytest_sessionfinish(session, exitstatus):
    """With RELO_CHECK_REPORT set (runs against the bounds-checked build), write the number of
    failed index checks the library counted during the session to that file."""
    path = os.environ.get("RELO_CHECK_REPORT")
    if path:
        from paper_1801_08361_gb300 import binding as B
        with open(path, "w") as f:
            f.write(str(int(B.lib().relo_debug_check_failures())))
