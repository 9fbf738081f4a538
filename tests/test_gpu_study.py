"""The collaborative pipeline study (paper_1801_08361_gb300.study) on three house fragments: the
verifier's confusion counts add up per pair, every verified sample lands in the pair's clusters,
the safety margin is the largest cluster minus the largest incorrect one, scene 0 is the gauge,
and where every confident pair's largest cluster is correct the optimised global poses render
the global map like the true poses, and so does the single model fused with them."""
import pytest
import torch

from paper_1801_08361_gb300 import study

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def report():
    return study.run(n_fragments=3, frames=12, n_pairs=3, seed=5, n_views=2, dev=torch.device("cuda:0"),
                     log=lambda m: None)


def test_counts_add_up(report):
    assert report["attempts"] == 2 * 12 * len(report["pairs"])
    for v, c in zip(report["verifier"], report["clustering"]):
        assert v["pair"] == c["pair"]
        assert v["total"] == 24
        assert v["tp"] + v["fp"] + v["tn"] + v["fn"] == v["relocalised"] <= v["total"]
        assert c["samples"] == v["tp"] + v["fp"]          # every verified sample is clustered
        assert c["correct"] >= c["incorrect"] >= 0
        assert c["margin"] == c["correct"] - c["incorrect"]


def test_pose_graph_and_global_map(report):
    pg = report["pose_graph"]["scenes"]
    assert pg and pg[0]["scene"] == 0 and pg[0]["rot_deg"] < 1e-6 and pg[0]["trans_m"] < 1e-9
    confident = [c for c in report["clustering"] if c["correct"] >= 2]
    if confident and all(c["largest_ok"] for c in confident) and report["render"]:
        for s in pg:
            assert s["rot_deg"] < 5.0 and s["trans_m"] < 0.10
        assert report["render"]["median_abs_diff_mm"] <= 50
        f = report["fused"]
        assert f["frames"] > 0 and f["blocks"] > 0 and f["median_abs_diff_mm"] <= 50
