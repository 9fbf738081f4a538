"""Pins of the oracle's relocaliser training: Algorithm R reservoirs and mean-shift modes."""
import math

import numpy as np

import oracle
from paper_1801_08361_gb300 import synth


def test_mean_shift_recovers_blob_centres_and_weights():
    rng = np.random.default_rng(0)
    centres = np.array([[0.0, 0.0, 1.0], [0.5, 0.0, 1.0], [0.0, 0.6, 1.2]])
    sizes = [30, 20, 10]
    pts = np.concatenate([c + rng.normal(0, 0.01, (n, 3)) for c, n in zip(centres, sizes)]).astype(np.float32)
    perm = rng.permutation(len(pts))
    p = oracle.LeafParams()
    modes = oracle.mean_shift_leaf(pts[perm], p)
    assert len(modes) == 3
    for k in range(3):                                   # ranked by support
        assert np.linalg.norm(modes[k, :3] - centres[k]) < 0.01
        assert modes[k, 10] == np.float32(sizes[k] / 60)
        # inverse covariance ~ 1 / (0.01^2 + 1e-4) on the diagonal
        assert 1 / (3e-4) < modes[k, 3] < 1 / (1e-4 + 0.4e-4)
        sub = pts[perm][np.linalg.norm(pts[perm] - centres[k], axis=1) < 0.1].astype(np.float64)
        cov = np.cov(sub.T, bias=True) + 1e-4 * np.eye(3)
        want_ln = math.log(sizes[k] / 60) - 0.5 * math.log(np.linalg.det(2 * math.pi * cov))
        assert abs(modes[k, 9] - want_ln) < 1e-4
    p2 = oracle.LeafParams(max_modes=2)
    m2 = oracle.mean_shift_leaf(pts[perm], p2)
    assert len(m2) == 2 and np.allclose(m2, modes[:2])


def test_mean_shift_bandwidth_decides_when_two_clusters_merge():
    """A Gaussian kernel of width h over two equal point masses a distance d apart gives a density
    with one maximum when d <= 2 h and two when d > 2 h (h = 5 cm): at 8.5 cm one mode at the
    midpoint holds all samples, at 13 cm each cluster is a mode of half the weight."""
    p = oracle.LeafParams()
    assert p.bandwidth == 0.05
    for d, n_modes in ((0.085, 1), (0.13, 2)):
        pts = np.array([[0.0, 0.0, 1.0]] * 25 + [[d, 0.0, 1.0]] * 25, np.float32)
        m = oracle.mean_shift_leaf(pts, p)
        assert len(m) == n_modes, d
        assert np.allclose(m[:, 10], 1.0 / n_modes)
        if n_modes == 1:
            assert np.allclose(m[0, :3], [d / 2, 0.0, 1.0], atol=1e-6)


def test_mean_shift_single_point_and_empty():
    p = oracle.LeafParams()
    m = oracle.mean_shift_leaf(np.array([[1.0, 2.0, 3.0]], np.float32), p)
    assert len(m) == 1 and np.allclose(m[0, :3], [1, 2, 3]) and m[0, 10] == 1.0
    assert np.allclose(m[0, 3:9], [1e4, 0, 0, 1e4, 0, 1e4], rtol=1e-6)
    assert len(oracle.mean_shift_leaf(np.zeros((0, 3), np.float32), p)) == 0


def _one_leaf_nodes():
    nodes = np.zeros((1, 1), dtype=synth.NODE_DTYPE)
    nodes["tau"] = 2 ** 30        # everything goes left: leaf 0
    return nodes


def _frame(n_valid, seed):
    rng = np.random.default_rng(seed)
    W, H = 40, 25
    d = np.zeros(W * H, np.uint16)
    d[:n_valid] = rng.integers(500, 3000, n_valid)
    return synth.Intrinsics.for_size(W, H), d.reshape(H, W), np.zeros((H, W, 4), np.uint8)


def test_reservoir_keeps_everything_below_capacity_in_arrival_order():
    intr, d, rgb = _frame(30, 1)
    pose = np.eye(4)
    pose[:3, 3] = [1, 2, 3]
    r = oracle.Reservoirs(_one_leaf_nodes(), oracle.LeafParams(capacity=64))
    r.add_frame(intr, pose, d, rgb)
    samples, count = r.contents()
    assert count[0, 0] == 30 and count[0, 1] == 0
    pix = np.arange(30)
    want = oracle.camera_points(d, intr, pix) + [1, 2, 3]
    assert np.array_equal(samples[0, 0, :30], want.astype(np.float32))


def test_reservoir_inclusion_is_uniform():
    """Algorithm R keeps each of n offered samples with probability capacity / n."""
    intr, d, rgb = _frame(1000, 2)
    cap, trials = 32, 300
    hits = np.zeros(1000)
    cam = oracle.camera_points(d, intr, np.arange(1000)).astype(np.float32)
    keys = {tuple(x) for x in cam.tolist()}
    assert len(keys) == 1000
    index = {tuple(x): i for i, x in enumerate(cam.tolist())}
    for s in range(trials):
        r = oracle.Reservoirs(_one_leaf_nodes(), oracle.LeafParams(capacity=cap, seed=s))
        r.add_frame(intr, np.eye(4), d, rgb)
        samples, count = r.contents()
        assert count[0, 0] == cap
        for x in samples[0, 0].tolist():
            hits[index[tuple(x)]] += 1
    p = cap / 1000
    # bins of 100 samples: expected trials * 100 * p each
    b = hits.reshape(10, 100).sum(1)
    e = trials * 100 * p
    chi2 = ((b - e) ** 2 / e).sum()
    assert chi2 < 30.0                                   # 9 dof
    assert abs(hits.sum() - trials * cap) == 0


def test_reservoir_of_one_keeps_the_second_of_two_samples_half_the_time():
    """Algorithm R with capacity 1: the second sample replaces the first with probability 1/2
    (a draw over [0, n) instead of [0, n] would always replace it)."""
    intr, d, rgb = _frame(2, 4)
    second = oracle.camera_points(d, intr, np.array([1])).astype(np.float32)[0]
    trials = 400
    kept = 0
    for s in range(trials):
        r = oracle.Reservoirs(_one_leaf_nodes(), oracle.LeafParams(capacity=1, seed=s))
        r.add_frame(intr, np.eye(4), d, rgb)
        samples, count = r.contents()
        assert count[0, 0] == 1
        kept += int(np.array_equal(samples[0, 0, 0], second))
    assert abs(kept - trials / 2) < 4 * np.sqrt(trials / 4)        # binomial, 4 standard deviations


def test_stride_and_invalid_pixels_are_skipped():
    intr, d, rgb = _frame(1000, 3)
    d = d.copy()
    d[0, :] = 0
    r = oracle.Reservoirs(_one_leaf_nodes(), oracle.LeafParams(capacity=4096, stride=2))
    r.add_frame(intr, np.eye(4), d, rgb)
    _, count = r.contents()
    v, u = np.mgrid[0:25, 0:40]
    assert count[0, 0] == int(((d > 0) & (u % 2 == 0) & (v % 2 == 0)).sum())


def test_threaded_mode_fill_equals_one_thread(room, oracle_room):
    """Filling the leaves' modes from several threads (disjoint leaf ranges) gives the modes of the
    one-thread fill bit for bit."""
    world, _ = room
    intr = synth.Intrinsics.for_size(160, 120)
    frames = [(intr, P) + oracle_room.raycast(intr, P) for P in synth.training_poses(world, 3, seed=12)]
    nodes = synth.random_forest_nodes(2, 6, seed=3, depth_tau=100, colour_tau=32)
    p = oracle.LeafParams(capacity=32, max_modes=4, seed=1)
    one = oracle.train_forest(nodes, frames, p)
    many = oracle.train_forest(nodes, frames, p, threads=4)
    assert one.n_modes.sum() > 20
    assert np.array_equal(one.n_modes, many.n_modes)
    assert np.array_equal(one.modes.view(np.uint32), many.modes.view(np.uint32))
