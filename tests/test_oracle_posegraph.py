"""Pins of the pose-graph oracle (Sec. 3.3.1-3.3.2) against closed forms and invariants:
dual-quaternion blends whose result is known exactly, the clustering thresholds of Sec. 4.2.4,
exact recovery of global poses from consistent relative transforms, first-order optimality of
the least-squares solution on inconsistent ones, the component of scene 0, and Phi's terms."""
import math

import numpy as np
import pytest

from oracle import posegraph as PG


def rot(axis, deg):
    """Rodrigues' formula, written out for the tests."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    th = math.radians(deg)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def rigid(R=None, t=(0, 0, 0)):
    T = np.eye(4)
    if R is not None:
        T[:3, :3] = R
    T[:3, 3] = t
    return T


def random_rigid(rng, t_scale=2.0):
    axis = rng.normal(size=3)
    return rigid(rot(axis, rng.uniform(-170, 170)), rng.uniform(-t_scale, t_scale, 3))


def inv(T):
    return np.linalg.inv(T)


# -- rotation helpers ------------------------------------------------------------------------

@pytest.mark.parametrize("deg", [0.0, 1.0, 19.9, 90.0, 179.0])
def test_rotation_angle_closed_form(deg):
    R = rot([0.3, -1.0, 0.5], deg)
    assert abs(PG.rot_angle(R, np.eye(3)) - math.radians(deg)) < 1e-7
    S = rot([1, 2, 3], 40)
    assert abs(PG.rot_angle(R @ S, S) - math.radians(deg)) < 1e-7


@pytest.mark.parametrize("deg", [10.0, 170.0, 190.0, 350.0])
def test_vee_takes_the_quaternion_with_nonnegative_w(deg):
    v = PG.vee(rigid(rot([0, 0, 1], deg), (1, 2, 3)))
    # rotation by deg about z: q = (cos(deg/2), 0, 0, sin(deg/2)), flipped when cos < 0
    sgn = 1.0 if math.cos(math.radians(deg / 2)) >= 0 else -1.0
    assert np.allclose(v, [0, 0, sgn * math.sin(math.radians(deg / 2)), 1, 2, 3], atol=1e-12)


# -- dual quaternion blending ------------------------------------------------------------------

def test_blend_of_one_sample_is_the_sample():
    rng = np.random.default_rng(0)
    for _ in range(10):
        T = random_rigid(rng)
        assert np.allclose(PG.dq_blend([T]), T, atol=1e-12)
        assert np.allclose(PG.dq_blend([T, T, T]), T, atol=1e-12)


def test_blend_of_pure_translations_is_their_mean():
    ts = [(0.1, 0.2, 0.3), (-0.4, 0.0, 1.0), (0.9, -0.2, 0.5)]
    B = PG.dq_blend([rigid(t=t) for t in ts])
    assert np.allclose(B, rigid(t=np.mean(ts, axis=0)), atol=1e-12)


def test_blend_of_equal_rotations_averages_translations():
    R = rot([1, 1, 0], 33)
    B = PG.dq_blend([rigid(R, (1, 0, 0)), rigid(R, (0, 1, 2))])
    assert np.allclose(B, rigid(R, (0.5, 0.5, 1.0)), atol=1e-12)


def test_blend_of_coaxial_rotations_is_the_mean_angle():
    # sum of the quaternions of angles a, b about one axis points at angle (a + b) / 2
    B = PG.dq_blend([rigid(rot([0, 1, 0], 10)), rigid(rot([0, 1, 0], 30)), rigid(rot([0, 1, 0], 20))])
    assert np.allclose(B, rigid(rot([0, 1, 0], 20)), atol=1e-12)


def test_blend_of_opposite_rotations_about_an_offset_axis_is_the_identity():
    # rotations by +-theta about the z axis through p = (2, 0, 0): T = (R, p - R p).  The blend is
    # exactly the identity; averaging translations would leave p (1 - cos theta) behind.
    p = np.array([2.0, 0.0, 0.0])
    Ts = [rigid(rot([0, 0, 1], s * 40), p - rot([0, 0, 1], s * 40) @ p) for s in (1, -1)]
    assert np.allclose(PG.dq_blend(Ts), np.eye(4), atol=1e-12)
    assert np.linalg.norm(np.mean([T[:3, 3] for T in Ts], axis=0)) > 0.4


def test_blend_aligns_quaternion_signs():
    # rotations by 179 and -179 degrees (181) about x are 2 degrees apart; their quaternions with
    # w >= 0 have opposite signs, so an unaligned sum would nearly cancel
    B = PG.dq_blend([rigid(rot([1, 0, 0], 179)), rigid(rot([1, 0, 0], 181))])
    assert np.allclose(B, rigid(rot([1, 0, 0], 180)), atol=1e-12)


# -- clustering -----------------------------------------------------------------------------

def test_clustering_thresholds_and_chains():
    g = PG.PoseGraph(3)
    A = rigid(rot([0, 0, 1], 0), (0, 0, 0))
    assert g.add_sample(0, 1, A) == 1
    assert g.add_sample(0, 1, rigid(rot([0, 0, 1], 19.0))) == 2               # within 20 degrees
    assert g.add_sample(0, 1, rigid(t=(0.099, 0, 0))) == 3                   # within 10 cm
    assert g.add_sample(0, 1, rigid(rot([0, 0, 1], 38.0))) == 4               # 19 deg from a member
    assert g.add_sample(0, 1, rigid(rot([1, 0, 0], 25.0))) == 1               # 25 deg from all
    assert g.add_sample(0, 1, rigid(t=(0.0, 0.25, 0))) == 1                  # 25 cm from all
    assert g.add_sample(0, 1, rigid(t=(0.0, -0.15, 0))) == 1                 # 15 cm from the nearest
    assert [len(c) for c in g.clusters[(0, 1)]] == [4, 1, 1, 1]


def test_reversed_samples_are_inverted_into_the_pair():
    rng = np.random.default_rng(3)
    T = random_rigid(rng)
    g = PG.PoseGraph(3)
    assert g.add_sample(2, 0, T) == 1
    assert g.add_sample(0, 2, inv(T) @ rigid(rot([0, 1, 0], 3), (0.01, 0, 0))) == 2
    assert list(g.clusters) == [(0, 2)]
    assert np.allclose(g.clusters[(0, 2)][0][0], inv(T), atol=1e-12)


# -- optimisation -----------------------------------------------------------------------------

def _consistent_graph(n, edges, seed):
    rng = np.random.default_rng(seed)
    gt = [np.eye(4)] + [random_rigid(rng) for _ in range(n - 1)]
    g = PG.PoseGraph(n)
    for a, b in edges:
        aTb = inv(gt[a]) @ gt[b]                  # the pose graph's fixed point: gT_a^-1 gT_b = aT_b
        g.add_sample(a, b, aTb)
        g.add_sample(b, a, inv(aTb))
    return g, gt


def test_consistent_relative_transforms_give_the_true_poses():
    g, gt = _consistent_graph(5, [(0, 1), (1, 2), (2, 3), (3, 0), (1, 3), (4, 2)], seed=5)
    poses, flags, eps = g.optimise()
    assert all(flags) and eps < 1e-9
    for s in range(5):
        assert np.allclose(poses[s], gt[s], atol=1e-9)


def test_scene_zero_is_the_gauge_and_other_components_stay_out():
    g, gt = _consistent_graph(6, [(0, 2), (2, 5), (1, 3)], seed=9)
    g.add_sample(0, 4, rigid(t=(1, 0, 0)))        # a single sample: not confident
    poses, flags, eps = g.optimise()
    assert list(flags) == [True, False, True, False, False, True]
    assert np.allclose(poses[0], np.eye(4)) and np.allclose(poses[1], np.eye(4))
    assert np.allclose(poses[5], gt[5], atol=1e-9) and eps < 1e-9


def test_largest_cluster_is_the_edge():
    g = PG.PoseGraph(2)
    good, bad = rigid(rot([0, 0, 1], 30), (1, 0, 0)), rigid(rot([0, 0, 1], -60), (0, 2, 0))
    for T in (bad, good, bad, good, good):
        g.add_sample(0, 1, T)
    poses, flags, eps = g.optimise()
    assert np.allclose(poses[1], good, atol=1e-9)


def test_inconsistent_loop_reaches_a_stationary_point():
    rng = np.random.default_rng(11)
    n = 4
    gt = [np.eye(4)] + [random_rigid(rng) for _ in range(n - 1)]
    g = PG.PoseGraph(n)
    for a, b in [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]:
        for _ in range(2):
            noise = rigid(rot(rng.normal(size=3), rng.uniform(0, 3)), rng.normal(scale=0.02, size=3))
            g.add_sample(a, b, inv(gt[a]) @ gt[b] @ noise)
    poses, flags, eps = g.optimise()
    edges = g.confident_edges()

    def cost(P):
        return sum(float(np.sum(PG.vee(inv(P[b]) @ P[a] @ T) ** 2)) for a, b, T in edges)

    c0 = cost(poses)
    assert eps > 0
    # no small left-multiplied perturbation of a free node lowers the sum of squares
    h = 1e-4
    for s in range(1, n):
        for k in range(6):
            for sg in (1, -1):
                P = poses.copy()
                if k < 3:
                    P[s] = rigid(rot(np.eye(3)[k], sg * math.degrees(h))) @ P[s]
                else:
                    P[s][k - 3, 3] += sg * h
                assert cost(P) >= c0 - 1e-12
    # and it is far better than leaving every global pose at the identity
    assert c0 < 0.5 * sum(float(np.sum(PG.vee(T) ** 2)) for _, _, T in edges)


# -- candidate score Phi ------------------------------------------------------------------------

def test_phi_terms():
    g = PG.PoseGraph(4)
    P = rigid(rot([0, 1, 0], 12), (1, 2, 0.5))
    assert g.score(0, 1, P) == 0.0
    for _ in range(4):
        g.add_sample(0, 1, rigid(t=(0.3, 0, 0)))
    g.optimise()                                  # scenes 0 and 1 have optimised global poses
    assert g.score(0, 1, P) == -2.0               # phi_conf = 4 - N
    assert g.score(1, 0, P) == -2.0               # clusters are per unordered pair
    assert g.score(2, 0, P) == 1.0                # phi_new: only scene 0 is optimised
    assert g.score(2, 3, P) == 0.0
    g.mark_tried(2, 0, P)
    near = rigid(rot([0, 1, 0], 12 + 4.9), (1.04, 2, 0.5))
    far = rigid(rot([0, 1, 0], 12 + 5.1), (1, 2, 0.5))
    assert g.score(2, 0, near) == 1.0 - 5.0
    assert g.score(2, 0, far) == 1.0
    assert g.score(0, 2, near) == 1.0             # tried against scene 2, not scene 0
