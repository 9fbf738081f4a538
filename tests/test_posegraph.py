"""The library's pose graph (relo_pose_graph_*, host code) against the oracle on the same seeded
sample streams: cluster sizes after every sample (exact), the scenes in the pose graph (exact),
the optimised global poses and epsilon (1e-6: the two minimise the same function with different
Levenberg-Marquardt implementations from the same start), and Phi of random candidates (exact).
Runs on the CPU; no GPU call is made."""
import math

import numpy as np
import pytest

from oracle import posegraph as PG
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def rot(axis, deg):
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    th = math.radians(deg)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def rigid(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def sample_stream(n, n_samples, seed, outlier_rate=0.2, rot_noise_deg=4.0, t_noise_m=0.03):
    """Relative transform samples as inter-agent relocalisation yields them: a random pair, its
    true aT_b perturbed by small noise, or (at outlier_rate) a random wrong transform."""
    rng = np.random.default_rng(seed)
    gt = [np.eye(4)] + [rigid(rot(rng.normal(size=3), rng.uniform(-170, 170)), rng.uniform(-3, 3, 3))
                        for _ in range(n - 1)]
    out = []
    for _ in range(n_samples):
        a, b = rng.choice(n, 2, replace=False)
        if rng.random() < outlier_rate:
            T = rigid(rot(rng.normal(size=3), rng.uniform(-180, 180)), rng.uniform(-3, 3, 3))
        else:
            T = np.linalg.inv(gt[a]) @ gt[b] @ rigid(rot(rng.normal(size=3), rng.uniform(0, rot_noise_deg)),
                                                    rng.normal(scale=t_noise_m, size=3))
        out.append((int(a), int(b), T))
    return gt, out


def _compare(n, stream, seed):
    lib, ora = B.PoseGraph(n), PG.PoseGraph(n)
    for a, b, T in stream:
        assert lib.add_sample(a, b, T) == ora.add_sample(a, b, T)
    for a in range(n):
        for b in range(a + 1, n):
            assert lib.cluster_sizes(a, b) == [len(c) for c in ora.clusters.get((a, b), [])]
            assert lib.cluster_sizes(b, a) == lib.cluster_sizes(a, b)
            for c, samples in enumerate(ora.clusters.get((a, b), [])):
                blend = PG.dq_blend(samples)
                assert np.abs(lib.cluster_blend(a, b, c) - blend).max() < 1e-12
                assert np.abs(lib.cluster_blend(b, a, c) - np.linalg.inv(blend)).max() < 1e-12
    pl, fl, el = lib.optimise()
    po, fo, eo = ora.optimise()
    assert list(fl) == list(fo)
    assert np.abs(pl - po).max() < 1e-6
    assert abs(el - eo) <= 1e-6 * max(1.0, eo)
    rng = np.random.default_rng(seed)
    poses = [rigid(rot(rng.normal(size=3), rng.uniform(-180, 180)), rng.uniform(-2, 2, 3)) for _ in range(12)]
    for k in range(40):
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        P = poses[k % len(poses)]
        if k % 3 == 0:
            P = P @ rigid(rot(rng.normal(size=3), rng.uniform(0, 8)), rng.normal(scale=0.04, size=3))
        assert lib.score(a, b, P) == ora.score(a, b, P)
        if k % 2 == 0:
            lib.mark_tried(a, b, P)
            ora.mark_tried(a, b, P)
    lib.close()
    return fl, el


@pytest.mark.parametrize("n,n_samples,seed", [(2, 6, 1), (4, 40, 2), (6, 120, 3), (8, 300, 4)])
def test_library_matches_oracle_on_sample_streams(n, n_samples, seed):
    _, stream = sample_stream(n, n_samples, seed)
    flags, eps = _compare(n, stream, seed)
    if n_samples >= 40:
        assert flags.sum() >= 2


def test_exact_samples_recover_the_true_poses():
    gt, stream = sample_stream(5, 60, 7, outlier_rate=0.0, rot_noise_deg=0.0, t_noise_m=0.0)
    g = B.PoseGraph(5)
    for a, b, T in stream:
        g.add_sample(a, b, T)
    poses, flags, eps = g.optimise()
    assert flags.all() and eps < 1e-9
    assert np.abs(poses - np.stack(gt)).max() < 1e-9


def test_empty_graph_and_single_scene():
    g = B.PoseGraph(1)
    poses, flags, eps = g.optimise()
    assert flags.tolist() == [True] and np.allclose(poses[0], np.eye(4)) and eps == 0.0
    g3 = B.PoseGraph(3)
    poses, flags, eps = g3.optimise()
    assert flags.tolist() == [True, False, False] and eps == 0.0
    assert g3.cluster_sizes(1, 2) == []


def test_bad_arguments_are_rejected():
    with pytest.raises(B.ReloError):
        B.PoseGraph(0)
    g = B.PoseGraph(3)
    for a, b in ((0, 0), (-1, 1), (0, 3)):
        with pytest.raises(B.ReloError):
            g.add_sample(a, b, np.eye(4))
        with pytest.raises(B.ReloError):
            g.score(a, b, np.eye(4))
        with pytest.raises(B.ReloError):
            g.cluster_sizes(a, b)
