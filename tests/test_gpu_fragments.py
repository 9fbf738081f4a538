"""Batched attempts between house fragments: 8 sub-scenes cut from the 10 x 8 x 3 m house (1 to 3
rooms each, 13-40 m^2 of floor, every one in its own random rigid frame) and all 56 ordered pairs
(a, b) in one batch, with view sizes mixed over 320x240, 480x360 and 640x480 and hypothesis
counts drawn from 256-1024.  Checks: the batch equals the same attempts run one by one; the
captured CUDA graph equals the eager launches; at full size, in the batch's own launches, the
query depth and colour on sampled pixels match the oracle's raycast and the forest leaves of the
whole query image match the oracle's forest bit for bit; verified poses agree with the known
relative transforms of the fragments (Sec. 3.3.1: aT_b)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import fragments as F

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
T = F.TREES
ORACLE_FRAG = 7          # the fragment whose host blocks are kept for the oracle checks


@pytest.fixture(scope="module")
def fragments():
    world, frags, scenes, forests, kept = F.build(DEV, keep_blocks=(ORACLE_FRAG,))
    return world, frags, scenes, forests, kept[ORACLE_FRAG]


@pytest.fixture(scope="module")
def pairs(fragments):
    """The 56 ordered pairs: query of b (a perturbed view of b's trajectory), relocalised with a's
    forest and verified against a."""
    world, frags, scenes, forests, _ = fragments
    return F.pairs(world, frags, scenes, forests, DEV)


PRM = dict(batch=F.BATCH_PIXELS, max_tries=F.MAX_TRIES)


def _batch(items):
    prm = B.ransac_params(n_hyps=1024, **PRM)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    return B.Batch(att, prm, ws), att


@pytest.fixture(scope="module")
def batch_run(pairs):
    items, _ = pairs
    bt, att = _batch(items)
    res = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.run(res)
    torch.cuda.synchronize()
    return bt, att, res.cpu().numpy()


def test_mixed_batch_equals_single_attempts(pairs, batch_run):
    items, _ = pairs
    _, _, want = batch_run
    for k, it in enumerate(items):
        bt, _ = _batch([it])
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        bt.run(res)
        torch.cuda.synchronize()
        assert np.array_equal(res.cpu().numpy(), want[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES]), k


def test_graph_replay_equals_eager_run(pairs, batch_run):
    items, _ = pairs
    bt, _, want = batch_run
    res = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.capture(res)
    for _ in range(2):
        res.zero_()
        bt.replay()
        torch.cuda.synchronize()
        assert np.array_equal(res.cpu().numpy(), want)


def test_replay_needs_a_capture(pairs):
    bt, _ = _batch(pairs[0][:1])
    with pytest.raises(B.ReloError) as e:
        bt.replay()
    assert e.value.status == B.EINVAL


def test_full_size_query_images_match_oracle(fragments, pairs, batch_run):
    """The query raycast on every 7th pixel and the forest on every pixel, as the batch computed
    them (the last run), for the attempts whose query comes from the oracle's fragment."""
    _, frags, _, _, blocks = fragments
    items, meta = pairs
    bt, _, _ = batch_run
    bt.run(None)
    torch.cuda.synchronize()
    sc = oracle.Scene(blocks)
    ks = [k for k, m in enumerate(meta) if m["b"] == ORACLE_FRAG]
    assert {items[k]["intr"].width for k in ks} >= {640}
    for k in ks:
        it, m = items[k], meta[k]
        intr = it["intr"]
        W, H = intr.width, intr.height
        d, c, lv = bt.attempt_images(k, W, H, T)
        d = d.cpu().numpy().view(np.uint16)
        c = c.cpu().numpy()
        sub = np.arange(0, W * H, 7)
        do, co = sc.raycast(intr, it["pose_b"], noise=it["noise"].cpu().numpy(), pixels=sub)
        dg, cg = d.reshape(-1)[sub], c.reshape(-1, 4)[sub]
        assert ((dg > 0) != (do > 0)).mean() <= 5e-4
        both = (dg > 0) & (do > 0)
        assert (np.abs(dg[both].astype(int) - do[both].astype(int)) <= 1).mean() >= 0.999
        close = both & (np.abs(dg.astype(int) - do.astype(int)) <= 1)
        assert (np.abs(cg[close][:, :3].astype(int) - co[close][:, :3].astype(int)).max(1) <= 1).mean() >= 0.995
        leaves = oracle.forest_eval(frags[m["a"]]["nodes"], d, c)
        assert np.array_equal(lv.cpu().numpy().view(np.uint16), leaves)


def _pose_error(P, Q):
    dt = float(np.linalg.norm(P[:3, 3] - Q[:3, 3]))
    ca = (np.trace(P[:3, :3] @ Q[:3, :3].T) - 1) / 2
    return dt, math.degrees(math.acos(max(-1.0, min(1.0, ca))))


def test_verified_poses_match_the_fragment_transforms(pairs, batch_run):
    """Relocalising b's query with a's relocaliser estimates the query's pose in a's frame, i.e.
    aT_b applied to its pose in b's frame; half the pairs whose query room lies in fragment a
    succeed.  The depth test of Sec. 3.3.1 accepts any pose whose render of a agrees with the
    query's depth, so a query filled by a flat wall also verifies at a wrong pose facing a wall
    at the same distance (seen here: every pixel valid in both, mean difference about 4 cm, the
    pose metres off); the paper removes such samples later by clustering the relative transforms
    (Sec. 3.3.2), so the bar is that they stay a minority of the verified results."""
    items, meta = pairs
    _, _, raw = batch_run
    covered = ok_cov = verified = wrong_verified = 0
    by_size = {}
    for k, m in enumerate(meta):
        r = B.result_from_bytes(torch.from_numpy(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES]))
        dt, dr = _pose_error(r["pose"], m["pose_a"])
        good = r["status"] == 0 and dt <= 0.05 and dr <= 5.0
        covered += m["covered"]
        ok_cov += m["covered"] and good
        if m["covered"]:
            c = by_size.setdefault(items[k]["intr"].width, [0, 0])
            c[0] += 1
            c[1] += good
        verified += r["verified"]
        if r["verified"] and not (dt <= 0.2 and dr <= 10.0):
            wrong_verified += 1
            print(f"wrong verification: a {m['a']} b {m['b']} covered {m['covered']} width {items[k]['intr'].width} "
                  f"error {dt:.3f} m {dr:.1f} deg, omega_a {r['omega_a']} / {r['omega']}, omega_ab {r['omega_ab']}, "
                  f"mean |D_a - D_b| {r['sum_absdiff_mm'] / max(1, r['omega_ab']):.1f} mm")
        # the relative transform formed from the result: aT_b = P_a P_b^-1 (Sec. 3.3.1)
        if good:
            rel = r["pose"] @ np.linalg.inv(items[k]["pose_b"])
            assert np.allclose(rel[:3, 3], r["rel_a_b"][:3, 3], atol=1e-9)
    print(f"covered {covered}: success {ok_cov} (by width: {by_size}); verified {verified}, "
          f"of which wrong {wrong_verified}")
    assert covered >= 10
    assert ok_cov >= 0.5 * covered
    assert wrong_verified <= max(1, verified // 4)


def test_persistent_schedule_equals_stage_launches(pairs, batch_run):
    """The RANSAC of the 56 attempts in one persistent launch (schedule persistent = 1: the CTAs take
    every attempt's search, fits, rounds and finalisation from a dependency-ordered list, waiting on
    per-attempt counters) gives the per-stage launches' results bit for bit, eagerly and from a
    captured graph, with fewer launches."""
    items, _ = pairs
    staged, _, want = batch_run
    bt, _ = _batch(items)
    bt.set_schedule(persistent=1)
    assert bt.launch_count < staged.launch_count
    res = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    bt.run(res)
    torch.cuda.synchronize()
    assert np.array_equal(res.cpu().numpy(), want)
    res.zero_()
    bt.capture(res)
    bt.replay()
    torch.cuda.synchronize()
    assert np.array_equal(res.cpu().numpy(), want)
