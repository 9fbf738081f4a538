"""Pins of the oracle's forest descent and depth-difference verification on hand-computed cases."""
import numpy as np

import oracle
from paper_1801_08361_gb300.synth import NODE_DTYPE


def _node(kind, dx1, dy1, dx2, dy2, tau, c1=0, c2=0):
    n = np.zeros((), dtype=NODE_DTYPE)
    n["kind"], n["dx1"], n["dy1"], n["dx2"], n["dy2"], n["tau"], n["c1"], n["c2"] = kind, dx1, dy1, dx2, dy2, tau, c1, c2
    return n


def test_depth_split_by_hand():
    # 4 x 3 image, depth 1000 mm except (u=2, v=1) = 2000 and (u=0, v=2) = 0 (invalid)
    d = np.full((3, 4), 1000, np.uint16)
    d[1, 2] = 2000
    d[2, 0] = 0
    rgb = np.zeros((3, 4, 4), np.uint8)
    # probe 1 at +1 pixel-metre in x, probe 2 at the pixel itself; left iff D(q1) - D(q2) < 1.
    # Offsets: trunc(1000 / 1000) = 1 px, trunc(1000 / 2000) = 0 px; probes clamp to the image.
    nodes = np.array([[_node(0, 1, 0, 0, 0, 1)]])
    leaves = oracle.forest_eval(nodes, d, rgb)[0]
    want = [[0, 0, 0, 0],        # equal neighbours; u=3 clamps onto itself
            [0, 1, 0, 0],        # (1,1): 2000 - 1000 >= 1 -> right; (2,1): offset 0 -> f = 0 -> left
            [0xFFFF, 0, 0, 0]]   # (0,2) has no depth
    assert leaves.tolist() == want


def test_offset_truncates_toward_zero_and_invalid_probe_reads_zero():
    d = np.zeros((1, 8), np.uint16)
    d[0, 5] = 2000
    d[0, 4] = 0       # probe target, invalid -> reads 0
    d[0, 3] = 700
    rgb = np.zeros((1, 8, 4), np.uint8)
    # at u=5, d=2000: dx1 = -3 -> -3000/2000 = -1.5 -> trunc -1 -> probe u=4 (reads 0)
    # f = 0 - D(5) = -2000 < -1999 ? no (equal bound check): tau = -1999 -> -2000 < -1999 -> left
    nodes = np.array([[_node(0, -3, 0, 0, 0, -1999)]])
    assert oracle.forest_eval(nodes, d, rgb)[0, 0, 5] == 0
    nodes = np.array([[_node(0, -3, 0, 0, 0, -2000)]])
    assert oracle.forest_eval(nodes, d, rgb)[0, 0, 5] == 1   # -2000 < -2000 false -> right
    # floor division would have probed u=3 (700): f = 700 - 2000 = -1300, not < -1999 -> right
    nodes = np.array([[_node(0, -3, 0, 0, 0, -1500)]])
    assert oracle.forest_eval(nodes, d, rgb)[0, 0, 5] == 0   # with trunc: -2000 < -1500 -> left


def test_colour_split_and_two_levels_by_hand():
    # 2 x 2 image, all depths 1000; colours chosen per pixel
    d = np.full((2, 2), 1000, np.uint16)
    rgb = np.zeros((2, 2, 4), np.uint8)
    rgb[0, 0, :3] = (10, 20, 30)
    rgb[0, 1, :3] = (200, 0, 5)
    rgb[1, 0, :3] = (0, 90, 40)
    rgb[1, 1, :3] = (60, 60, 60)
    # root: R of pixel minus B of pixel < 0 -> left (node 1) else right (node 2)
    # node 1: G(pixel) - G(pixel at +1 px x) < 0 -> leaf 0 else leaf 1
    # node 2: depth(pixel) - depth(pixel) < 1 -> leaf 2 (always)
    nodes = np.array([[_node(1, 0, 0, 0, 0, 0, c1=0, c2=2), _node(1, 0, 0, 1, 0, 0, c1=1, c2=1),
                       _node(0, 0, 0, 0, 0, 1)]])
    leaves = oracle.forest_eval(nodes, d, rgb)[0]
    # (0,0): 10-30<0 -> node1: G 20 - G(1,0 neighbour u=1 -> 0) = 20 not <0 -> leaf 1
    # (u=1,v=0): 200-5 >= 0 -> node2 -> leaf 2
    # (u=0,v=1): 0-40 < 0 -> node1: 90 - 60 >= 0 -> leaf 1
    # (u=1,v=1): 60-60 = 0 not < 0 -> node2 -> leaf 2
    assert leaves.tolist() == [[1, 2], [1, 2]]


def test_extreme_thresholds_reach_first_and_last_leaf():
    rng = np.random.default_rng(0)
    d = rng.integers(500, 4000, (20, 30)).astype(np.uint16)
    rgb = rng.integers(0, 256, (20, 30, 4)).astype(np.uint8)
    D = 4
    nodes = np.zeros((2, 2 ** D - 1), dtype=NODE_DTYPE)
    nodes["dx1"] = rng.integers(-100, 100, nodes.shape)
    nodes["dy2"] = rng.integers(-100, 100, nodes.shape)
    nodes["tau"][0] = 2 ** 30          # always left -> leaf 0
    nodes["tau"][1] = -(2 ** 30)       # always right -> leaf 2^D - 1
    leaves = oracle.forest_eval(nodes, d, rgb)
    assert (leaves[0] == 0).all() and (leaves[1] == 2 ** D - 1).all()


def test_verification_counts_by_hand():
    da = np.array([0, 1000, 1200, 0, 3000, 500], np.uint16)
    db = np.array([0, 1010, 0, 900, 2900, 560], np.uint16)
    c = oracle.verify_counts(da, db)
    # Omega = 6, Omega_a = {1,2,4,5}, Omega_b = {1,3,4,5}, Omega_ab = {1,4,5}, sum = 10 + 100 + 60
    assert c.tolist() == [6, 4, 4, 3, 170]
    assert oracle.verify_accept(c) is False         # 4/6 > 0.5 but mean 170/3 = 56.7 mm >= 50 mm


def test_verification_decision_rules():
    n = 100
    same = np.full(n, 1500, np.uint16)
    assert oracle.verify_accept(oracle.verify_counts(same, same))                     # mu = 0
    half = same.copy()
    half[:50] = 0
    assert not oracle.verify_accept(oracle.verify_counts(half, same))                # |Omega_a| / |Omega| = 0.5
    half[49] = 1500
    assert oracle.verify_accept(oracle.verify_counts(half, same))                    # 51 / 100 > 0.5
    assert not oracle.verify_accept(oracle.verify_counts(same, np.zeros(n, np.uint16)))  # empty Omega_ab
    off = same + 49
    assert oracle.verify_accept(oracle.verify_counts(off, same))                     # mean 49 mm < 50
    off = same + 50
    assert not oracle.verify_accept(oracle.verify_counts(off, same))                 # mean 50 mm, not < 50
