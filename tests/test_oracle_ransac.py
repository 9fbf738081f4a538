"""Pins of the oracle's Kabsch step, pixel energy and preemptive RANSAC against definitions
outside it: known rigid transforms, Horn's closed-form quaternion method, scipy's Gaussian
density, and exact recovery from noise-free correspondences."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import multivariate_normal

import oracle
from paper_1801_08361_gb300 import synth


def _random_pose(rng):
    T = np.eye(4)
    T[:3, :3] = Rotation.random(random_state=rng.integers(1 << 31)).as_matrix()
    T[:3, 3] = rng.uniform(-3, 3, 3)
    return T


def horn(c, w):
    """Horn (1987) closed form: the optimal rotation is the unit quaternion of the largest
    eigenvalue of the 4x4 matrix built from the cross-covariance."""
    cb, wb = c.mean(0), w.mean(0)
    S = (c - cb).T @ (w - wb)
    Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz = S.reshape(-1)
    N = np.array([[Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
                  [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
                  [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
                  [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    vals, vecs = np.linalg.eigh(N)
    q0, qx, qy, qz = vecs[:, -1]
    R = Rotation.from_quat([qx, qy, qz, q0]).as_matrix()
    return R, wb - R @ cb


def test_kabsch_recovers_known_transform():
    rng = np.random.default_rng(1)
    for n in (3, 4, 50):
        T = _random_pose(rng)
        c = rng.uniform(-2, 2, (n, 3))
        w = c @ T[:3, :3].T + T[:3, 3]
        R, t = oracle.kabsch(c, w)
        assert np.abs(R - T[:3, :3]).max() < 1e-12
        assert np.abs(t - T[:3, 3]).max() < 1e-12


def test_kabsch_agrees_with_horn_on_noisy_points():
    rng = np.random.default_rng(2)
    for _ in range(20):
        T = _random_pose(rng)
        c = rng.uniform(-2, 2, (30, 3))
        w = c @ T[:3, :3].T + T[:3, 3] + rng.normal(0, 0.05, (30, 3))
        R1, t1 = oracle.kabsch(c, w)
        R2, t2 = horn(c, w)
        assert np.abs(R1 - R2).max() < 1e-10 and np.abs(t1 - t2).max() < 1e-10


def test_kabsch_returns_proper_rotation_for_mirrored_points():
    rng = np.random.default_rng(3)
    c = rng.uniform(-1, 1, (10, 3))
    w = c * np.array([1.0, 1.0, -1.0])            # a reflection: best proper rotation has det +1
    R, _ = oracle.kabsch(c, w)
    assert abs(np.linalg.det(R) - 1.0) < 1e-12
    R2, _ = horn(c, w)
    assert np.abs(R - R2).max() < 1e-9


def _single_leaf_forest(modes_list):
    """One tree of depth 1; leaf 0 holds the given (mean, cov, weight) modes, leaf 1 is empty."""
    M = max(1, len(modes_list))
    modes = np.zeros((1, 2, M, 12), np.float32)
    for k, (mu, cov, w) in enumerate(modes_list):
        inv = np.linalg.inv(cov)
        modes[0, 0, k, :3] = mu
        modes[0, 0, k, 3:9] = [inv[0, 0], inv[0, 1], inv[0, 2], inv[1, 1], inv[1, 2], inv[2, 2]]
        modes[0, 0, k, 9] = math.log(w) - 0.5 * math.log(np.linalg.det(2 * math.pi * cov))
        modes[0, 0, k, 10] = w
    nm = np.array([[len(modes_list), 0]], np.uint8)
    nodes = np.zeros((1, 1), dtype=synth.NODE_DTYPE)
    return oracle.Forest(nodes, modes, nm)


def test_pixel_energy_matches_gaussian_density():
    """e = -log(max(1e-30, max_m w_m N(x; mu_m, Sigma_m))) against scipy's density."""
    rng = np.random.default_rng(4)
    modes = []
    for _ in range(3):
        A = rng.normal(0, 0.03, (3, 3))
        modes.append((rng.uniform(-1, 1, 3), A @ A.T + 1e-4 * np.eye(3), rng.uniform(0.1, 0.6)))
    forest = _single_leaf_forest(modes)
    # stored fields are float32: rebuild the density from what is stored
    st = forest.modes[0, 0].astype(np.float64)
    n = 40
    # scene points within a few standard deviations of the modes (far points would all sit at the
    # density floor and leave the Gaussian untested); camera points through a random pose
    pose = _random_pose(rng)
    near = np.array([modes[k % 3][0] for k in range(n)]) + rng.normal(0, 0.04, (n, 3))
    cam = (near - pose[:3, 3]) @ pose[:3, :3]
    leaves = np.zeros((1, 1, n), np.uint16)
    e, mu, found, x = oracle.pixel_energies(pose, cam, np.arange(n), leaves, forest)
    assert (e < oracle.LOG_EPS - 5.0).all()
    for i in range(n):
        dens = []
        for k in range(3):
            inv = np.array([[st[k, 3], st[k, 4], st[k, 5]], [st[k, 4], st[k, 6], st[k, 7]],
                            [st[k, 5], st[k, 7], st[k, 8]]])
            cov = np.linalg.inv(inv)
            w = math.exp(st[k, 9] + 0.5 * math.log(np.linalg.det(2 * math.pi * cov)))
            dens.append(w * multivariate_normal(st[k, :3], cov).pdf(x[i]))
        want = -math.log(max(1e-30, max(dens)))
        assert abs(e[i] - want) <= 1e-9 * max(1.0, abs(want))


def test_pixel_energy_single_isotropic_gaussian_closed_form():
    sigma, w = 0.02, 0.4
    forest = _single_leaf_forest([(np.zeros(3), sigma ** 2 * np.eye(3), w)])
    r = np.array([0.0, 0.01, 0.05, 0.2, 5.0])
    cam = np.stack([r, np.zeros_like(r), np.zeros_like(r)], 1)
    e, _, _, _ = oracle.pixel_energies(np.eye(4), cam, np.arange(5), np.zeros((1, 1, 5), np.uint16), forest)
    want = -math.log(w) + 1.5 * math.log(2 * math.pi * sigma ** 2) + r ** 2 / (2 * sigma ** 2)
    want = np.minimum(want, -math.log(1e-30))
    assert np.allclose(e, want, rtol=1e-6, atol=1e-6)      # float32-stored inverse covariance
    assert e[-1] == pytest.approx(-math.log(1e-30))
    # an empty leaf gives the floor energy
    e2, _, found, _ = oracle.pixel_energies(np.eye(4), cam, np.arange(5), np.ones((1, 1, 5), np.uint16), forest)
    assert (e2 == -math.log(1e-30)).all() and not found.any()


def _exact_setup(outlier_frac, seed):
    """A 64 x 48 view of a bumpy surface; every pixel gets its own leaf holding its exact scene
    coordinate (or, for outliers, a random point)."""
    rng = np.random.default_rng(seed)
    intr = synth.Intrinsics.for_size(64, 48)
    v, u = np.mgrid[0:48, 0:64]
    depth = (2000 + 300 * np.sin(u / 9.0) + 200 * np.cos(v / 7.0)).astype(np.uint16)
    P = _random_pose(rng)
    pix = np.arange(64 * 48)
    cam = oracle.camera_points(depth, intr, pix)
    wld = cam @ P[:3, :3].T + P[:3, 3]
    out = rng.random(len(pix)) < outlier_frac
    wld[out] = rng.uniform(-5, 5, (out.sum(), 3))
    D = 12
    modes = np.zeros((1, 1 << D, 1, 12), np.float32)
    modes[0, :len(pix), 0, :3] = wld
    sig2 = 1e-4
    modes[0, :len(pix), 0, 3:9] = [1 / sig2, 0, 0, 1 / sig2, 0, 1 / sig2]
    modes[0, :len(pix), 0, 9] = -0.5 * math.log((2 * math.pi * sig2) ** 3)
    modes[0, :len(pix), 0, 10] = 1.0
    nm = np.zeros((1, 1 << D), np.uint8)
    nm[0, :len(pix)] = 1
    forest = oracle.Forest(np.zeros((1, (1 << D) - 1), dtype=synth.NODE_DTYPE), modes, nm)
    leaves = pix.reshape(1, 48, 64).astype(np.uint16)
    return intr, depth, leaves, forest, P


@pytest.mark.parametrize("outliers", [0.0, 0.5])
def test_ransac_recovers_exact_pose(outliers):
    intr, depth, leaves, forest, P = _exact_setup(outliers, seed=7)
    prm = oracle.RansacParams(n_hyps=32, batch=100, seed=3, max_tries=20000)
    res = oracle.preemptive_ransac(depth, intr, leaves, forest, prm)
    assert res["valid"]
    # modes are float32 copies of the exact coordinates: pose exact to float32 rounding
    assert np.abs(res["pose"] - P).max() < 2e-5
    dt, dr = oracle.pose_error(res["pose"], P)
    assert dt < 1e-5 and dr < 1e-3


def test_round_energies_and_halving_match_brute_force():
    intr, depth, leaves, forest, P = _exact_setup(0.7, seed=8)
    prm = oracle.RansacParams(n_hyps=16, batch=50, seed=5, max_tries=20000)
    res = oracle.preemptive_ransac(depth, intr, leaves, forest, prm, trace=True)
    tr = res["trace"]
    r0 = tr.rounds[0]
    cam = oracle.camera_points(depth, intr, r0["pixels"])
    st = forest.modes[0].astype(np.float64)
    for h in range(16):
        if not tr.valid0[h]:
            assert r0["energy"][h] == np.inf
            continue
        R, t = tr.poses0[h][:3, :3], tr.poses0[h][:3, 3]
        tot = 0.0
        for i, p in enumerate(r0["pixels"]):
            x = R @ cam[i] + t
            lf = leaves[0].reshape(-1)[p]
            s2 = 1.0 / st[lf, 0, 3]
            dens = multivariate_normal(st[lf, 0, :3], s2 * np.eye(3)).pdf(x)
            tot += -math.log(max(1e-30, dens))
        assert abs(r0["energy"][h] - tot) <= 1e-7 * abs(tot)
    order = sorted(range(16), key=lambda h: (r0["energy"][h], h))
    assert r0["survivors"].tolist() == order[:8]
    sizes = [len(r["survivors"]) for r in tr.rounds]
    assert sizes == [8, 4, 2, 1]


def test_hypotheses_use_first_passing_try():
    """Every hypothesis is the Kabsch pose of its first passing try: re-drawing that try by hand
    from the published Philox blocks reproduces the hypothesis."""
    intr, depth, leaves, forest, P = _exact_setup(0.5, seed=9)
    prm = oracle.RansacParams(n_hyps=8, batch=10, seed=11, max_tries=20000)
    poses, ok, tries = oracle.generate_hypotheses(depth, intr, leaves, forest, prm)
    valid = oracle.valid_pixels(depth)
    for h in range(8):
        assert ok[h]
        x = oracle.philox(np.array([1, h, tries[h], 0], np.uint32), oracle.seed_key(11))[0]
        pix = [valid[(int(x[k]) * len(valid)) >> 32] for k in range(3)]
        cam = oracle.camera_points(depth, intr, np.array(pix))
        wld = forest.modes[0, np.array(pix), 0, :3].astype(np.float64)
        R, t = oracle.kabsch(cam, wld)
        assert np.abs(poses[h][:3, :3] - R).max() < 1e-12


def test_first_passing_try_is_the_first_triple_of_distinct_inliers():
    """Built so the answer is almost always known: inliers carry their exact scene coordinates and
    outliers are uniform in a 10 m cube, so a try passes the rigidity test when its three pixels are
    distinct inliers and, but for rare coincidences (an outlier within 5 cm of the right distance
    to both inliers of its triple), fails otherwise.  The kept try of a hypothesis is then the first
    all-inlier triple of its Philox stream for all but a few hypotheses."""
    intr, depth, leaves, forest, P = _exact_setup(0.5, seed=9)
    K = 32
    prm = oracle.RansacParams(n_hyps=K, batch=10, seed=11, max_tries=20000)
    _, ok, tries = oracle.generate_hypotheses(depth, intr, leaves, forest, prm)
    valid = oracle.valid_pixels(depth)
    exact = oracle.camera_points(depth, intr, valid) @ P[:3, :3].T + P[:3, 3]
    inlier = np.abs(forest.modes[0, valid, 0, :3] - exact).max(1) < 1e-3
    assert 0.4 < inlier.mean() < 0.6
    key = oracle.seed_key(11)
    same = 0
    for h in range(K):
        j = 0
        while True:
            x = oracle.philox(np.array([1, h, j, 0], np.uint32), key)[0]
            idx = [(int(x[k]) * len(valid)) >> 32 for k in range(3)]
            if len(set(idx)) == 3 and inlier[idx].all():
                break
            j += 1
        assert ok[h]
        same += int(tries[h] == j)
    assert same >= K - 2


def test_camera_points_project_back_to_their_pixels():
    """The pinhole projection u = fx x / z + cx, v = fy y / z + cy of each back-projected point
    returns its pixel, with z the depth in metres (unequal focal lengths and an off-centre
    principal point, so swapped axes show)."""
    intr = synth.Intrinsics(37, 23, 41.5, 57.25, 15.2, 13.7)
    rng = np.random.default_rng(12)
    depth = rng.integers(1, 9000, (23, 37)).astype(np.uint16)
    pix = np.arange(37 * 23)
    X = oracle.camera_points(depth, intr, pix)
    u, v = pix % 37, pix // 37
    assert np.allclose(X[:, 2], depth.reshape(-1) / 1000.0, rtol=0, atol=1e-15)
    assert np.allclose(intr.fx * X[:, 0] / X[:, 2] + intr.cx, u, rtol=0, atol=1e-9)
    assert np.allclose(intr.fy * X[:, 1] / X[:, 2] + intr.cy, v, rtol=0, atol=1e-9)


def test_halving_keeps_the_ceiling_of_half():
    """Preemptive halving keeps ceil(K_r / 2) hypotheses per round: 12 -> 6 -> 3 -> 2 -> 1."""
    intr, depth, leaves, forest, P = _exact_setup(0.3, seed=10)
    prm = oracle.RansacParams(n_hyps=12, batch=20, seed=6, max_tries=20000)
    res = oracle.preemptive_ransac(depth, intr, leaves, forest, prm, trace=True)
    assert [len(r["survivors"]) for r in res["trace"].rounds] == [6, 3, 2, 1]
