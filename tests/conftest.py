"""Shared fixtures.  Tests marked ``gpu`` need a GB300 and the built CUDA library."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built relocalisation library")


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
