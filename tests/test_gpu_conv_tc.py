"""The tcgen05 convolutions of the regressor (the forward of every layer but the head, the
backward-data pass of the stride-1 layers; TMA tile loads, MMAs into tensor memory) against the
mma.sync kernel on the same operands, and their bounded waits:
a launch whose loads are withheld gives up within its time limit, reports RELO_ETIMEOUT through
the learned path's result, frees what it holds and leaves the context usable.

Both kernels multiply the same BF16 operands and accumulate them in FP32 in the same order (taps in
turn, 16 channels per instruction), and the two instruction forms round alike: the network outputs
and gradients come out bit for bit equal (the 2000-step online training follows the same
trajectory with either).  Parity with the FP64 oracle is checked in test_gpu_regressor.py with the
tcgen05 path on."""
import numpy as np
import pytest
import torch

from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ORIGIN = (2.0, 2.0, 1.5)


def _u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(DEV)


def _forward(reg, dd, cc, tcgen05):
    n, H, W = dd.shape
    B.debug_conv_path(tcgen05)
    try:
        out = torch.zeros((n, H // 8, W // 8, 4), dtype=torch.float32, device=DEV)
        ws = torch.empty(B.regressor_workspace_size(n, W, H, False), dtype=torch.uint8, device=DEV)
        B.regressor_forward(reg, dd, cc, out, ws)
        torch.cuda.synchronize()
    finally:
        B.debug_conv_path(True)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("size", [(640, 480), (168, 136), (8, 8)])
def test_tcgen05_forward_matches_mma_sync(room, oracle_room, size):
    """Full tiles (640 x 480: output widths 160, 80 fill 64- and 16-pixel tile rows) and ragged
    ones (168 x 136: widths 42 and 21 leave partial tiles; 8 x 8: one pixel)."""
    world, _ = room
    W, H = size
    intr = synth.Intrinsics.for_size(W, H)
    poses = synth.training_poses(world, 2, seed=97)[:3]
    ds, cs = zip(*[oracle_room.raycast(intr, P) for P in poses])
    dd, cc = _u16(np.stack(ds)), torch.from_numpy(np.stack(cs)).to(DEV)
    reg = B.Regressor(seed=12, origin=ORIGIN)
    a = _forward(reg, dd, cc, True)
    b = _forward(reg, dd, cc, False)
    assert np.isfinite(a).all() and np.abs(a).max() > 0
    assert np.array_equal(a, b), np.abs(a - b).max()


def test_tcgen05_bounded_wait_reports_timeout(room, oracle_room):
    """Withhold the loads of the first output tile: the launch's wait for them runs out after
    50 ms, the learned relocalisation reports RELO_ETIMEOUT, and the next launches (no stall)
    give the results of a run before the stall, bit for bit."""
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    P = synth.training_poses(world, 2, seed=98)[0]
    d, c = oracle_room.raycast(intr, P)
    dd, cc = _u16(d), torch.from_numpy(c).to(DEV)
    reg = B.Regressor(seed=13, origin=ORIGIN)
    prm = B.ransac_params(n_hyps=32, batch=64, seed=1, max_tries=500)
    ws = torch.empty(B.regressor_relocalise_workspace_size(320, 240, prm), dtype=torch.uint8, device=DEV)

    def run():
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        B.regressor_relocalise(reg, dd, cc, intr, prm, ws, res)
        torch.cuda.synchronize()
        return res.cpu().numpy()

    before = run()
    assert B.result_from_bytes(torch.from_numpy(before))["status"] != B.ETIMEOUT
    B.debug_conv_stall(0, 50)
    try:
        stalled = run()
    finally:
        B.debug_conv_stall(-1, 0)
    assert B.result_from_bytes(torch.from_numpy(stalled))["status"] == B.ETIMEOUT
    after = run()
    assert np.array_equal(after, before)


def test_tcgen05_gradients_match_mma_sync(room, oracle_room):
    """Training's gradients with the tcgen05 kernels (the forward of every layer but the head, the
    backward-data pass of the stride-1 layers, masked by the ReLU) against the mma.sync kernels on
    the same operands: the loss and every gradient bit for bit."""
    world, _ = room
    intr = synth.Intrinsics.for_size(160, 120)
    poses = synth.training_poses(world, 2, seed=96)[:3]
    ds, cs = zip(*[oracle_room.raycast(intr, P) for P in poses])
    dd, cc = _u16(np.stack(ds)), torch.from_numpy(np.stack(cs)).to(DEV)
    n = len(poses)

    def grads(tcgen05):
        B.debug_conv_path(tcgen05)
        try:
            reg = B.Regressor(seed=14, origin=ORIGIN)
            ws = torch.empty(B.regressor_workspace_size(n, 160, 120, True), dtype=torch.uint8, device=DEV)
            loss = torch.zeros(1, dtype=torch.float32, device=DEV)
            B.regressor_gradients(reg, dd, cc, intr, poses, ws, loss)
            torch.cuda.synchronize()
            return float(loss.item()), reg.grads().astype(np.float64)
        finally:
            B.debug_conv_path(True)

    la, ga = grads(True)
    lb, gb = grads(False)
    assert la == lb and np.abs(gb).max() > 0
    assert np.array_equal(ga, gb), np.abs(ga - gb).max()
