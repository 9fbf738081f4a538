"""GPU parity of the learned regressor (BF16 tensor-core convolutions, FP32 accumulation)
against the FP64 oracle: forward output, loss and per-layer gradients on the same operands
(relative L2 <= 1e-2 forward, gradient cosine >= 0.999 per layer), a short training run, and the
learned RANSAC against the oracle's RANSAC on the same (constructed) cells, a fit of fixed views to
centimetres, and what online training gains on the tiny room."""

import numpy as np
import pytest
import torch

import oracle
from oracle import regressor as R
from paper_1801_08361_gb300 import binding as B
from paper_1801_08361_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ORIGIN = (2.0, 2.0, 1.5)


def _u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(DEV)


def _bf16(a):
    """Round to the nearest bfloat16 (ties to even): the value the tensor cores multiply."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _operands(params: R.Params, x):
    """The oracle's inputs for a like-for-like comparison: the kernels multiply BF16 copies of
    the FP32 master weights and of the input (biases stay FP32), so the FP64 oracle is given
    exactly those values; rounding the weights alone moves layer-1 gradients by ~1 % on a
    64 x 48 view, far above the parity bar."""
    pq = _unflat(_flat(params), params)
    return R.Params([_bf16(w) for w in pq.w], list(pq.b)), _bf16(x)


def _flat(params: R.Params):
    return np.concatenate([p.reshape(-1) for p in params.flat()]).astype(np.float32)


def _unflat(flat, like: R.Params):
    out, off = [], 0
    for p in like.flat():
        out.append(flat[off:off + p.size].reshape(p.shape).astype(np.float64))
        off += p.size
    return R.Params(out[0::2], out[1::2])


@pytest.fixture(scope="module")
def views(room, oracle_room):
    world, _ = room
    intr = synth.Intrinsics.for_size(64, 48)
    poses = synth.training_poses(world, 2, seed=91)
    ds, cs = zip(*[oracle_room.raycast(intr, P) for P in poses])
    return intr, poses, np.stack(ds), np.stack(cs)


@pytest.fixture(scope="module")
def params():
    p = R.init_params(5)
    rng = np.random.default_rng(6)
    for b in p.b:
        b += rng.normal(0, 0.05, b.shape)
    return p


def test_forward_matches_oracle(views, params):
    intr, poses, d, c = views
    reg = B.Regressor(_flat(params), origin=ORIGIN)
    n = d.shape[0]
    out = torch.zeros((n, 6, 8, 4), dtype=torch.float32, device=DEV)
    ws = torch.empty(B.regressor_workspace_size(n, 64, 48, False), dtype=torch.uint8, device=DEV)
    B.regressor_forward(reg, _u16(d), torch.from_numpy(c).to(DEV), out, ws)
    torch.cuda.synchronize()
    pq, x = _operands(params, np.stack([R.network_input(d[i], c[i]) for i in range(n)]))
    want, _ = R.forward(pq, x)
    got = out.cpu().numpy()
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= 1e-2, rel


def _forward_bf16_storage(params: R.Params, x):
    """The oracle's layers composed the way the kernels store activations: each layer computed in
    FP64 from its (BF16) input, its ReLU output rounded to BF16 before the next layer reads it."""
    acts, h = [x], x
    for l in range(len(params.w)):
        z = R.conv3x3(h, params.w[l], params.b[l], R.STRIDES[l])
        h = _bf16(np.maximum(z, 0.0)) if l < len(params.w) - 1 else z
        acts.append(h)
    return h, acts


def _gpu_gradients(views, params):
    intr, poses, d, c = views
    reg = B.Regressor(_flat(params), origin=ORIGIN)
    n = d.shape[0]
    ws = torch.empty(B.regressor_workspace_size(n, 64, 48, True), dtype=torch.uint8, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    B.regressor_gradients(reg, _u16(d), torch.from_numpy(c).to(DEV), intr, poses, ws, loss)
    torch.cuda.synchronize()
    return float(loss.item()), _unflat(reg.grads(), params)


def _oracle_gradients(views, params, bf16_storage):
    intr, poses, d, c = views
    n = d.shape[0]
    pq, x = _operands(params, np.stack([R.network_input(d[i], c[i]) for i in range(n)]))
    out, acts = _forward_bf16_storage(pq, x) if bf16_storage else R.forward(pq, x)
    tg = [R.cell_targets(d[i], intr, poses[i], ORIGIN) for i in range(n)]
    lo, g = R.loss_and_grad_output(out, np.stack([t[0] for t in tg]), np.stack([t[1] for t in tg]))
    return lo, R.backward(pq, acts, g)


def _cosines(got, want):
    out = []
    for gw, ww, gb, wb in zip(got.w, want.w, got.b, want.b):
        a, b = np.concatenate([gw.ravel(), gb.ravel()]), np.concatenate([ww.ravel(), wb.ravel()])
        out.append(float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b))))
    return out


def test_gradients_match_oracle_stage_isolated(views, params):
    """Each layer's gradients against the FP64 oracle evaluated on the same operands the kernels
    use: BF16 weights, input and stored activations (cosine >= 0.999 per layer)."""
    lg, got = _gpu_gradients(views, params)
    lo, want = _oracle_gradients(views, params, bf16_storage=True)
    assert abs(lg - lo) <= 1e-3 * abs(lo)
    cos = _cosines(got, want)
    assert min(cos) >= 0.999, cos


def test_gradients_against_the_fp64_network(views, params):
    """End to end against the FP64 network with BF16 weights and input: storing activations in
    BF16 costs up to ~1 % (cosine ~0.994) in the first layers' gradients on a 64 x 48 view, as the
    same storage rounding applied inside the oracle reproduces; the bar is cosine >= 0.99."""
    lg, got = _gpu_gradients(views, params)
    lo, want = _oracle_gradients(views, params, bf16_storage=False)
    assert abs(lg - lo) <= 1e-2 * abs(lo)
    cos = _cosines(got, want)
    assert min(cos) >= 0.99, cos


def test_training_reduces_loss(views):
    intr, poses, d, c = views
    reg = B.Regressor(seed=3, origin=ORIGIN)
    n = d.shape[0]
    ws = torch.empty(B.regressor_workspace_size(n, 64, 48, True), dtype=torch.uint8, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    dd, cc = _u16(d), torch.from_numpy(c).to(DEV)
    first = None
    for step in range(60):
        B.regressor_train_step(reg, dd, cc, intr, poses, 1e-3, ws, loss)
        torch.cuda.synchronize()
        if first is None:
            first = float(loss.item())
    assert float(loss.item()) < 0.9 * first


def test_training_resumes_from_a_checkpoint(views):
    """Checkpoint (parameters, Adam moments, step) after 4 steps, restore it into a regressor
    created from another seed, train 4 more steps on both: the parameters agree bit for bit."""
    intr, poses, d, c = views
    n = d.shape[0]
    ws = torch.empty(B.regressor_workspace_size(n, 64, 48, True), dtype=torch.uint8, device=DEV)
    dd, cc = _u16(d), torch.from_numpy(c).to(DEV)
    a = B.Regressor(seed=5, origin=ORIGIN)
    for _ in range(4):
        B.regressor_train_step(a, dd, cc, intr, poses, 1e-3, ws)
    state = B.regressor_state(a)
    assert state["step"] == 4 and np.any(state["m"] != 0) and np.any(state["v"] != 0)
    b = B.Regressor(seed=6, origin=ORIGIN)
    B.regressor_set_state(b, state)
    for reg in (a, b):
        for _ in range(4):
            B.regressor_train_step(reg, dd, cc, intr, poses, 1e-3, ws)
    torch.cuda.synchronize()
    sa, sb = B.regressor_state(a), B.regressor_state(b)
    assert sa["step"] == sb["step"] == 8
    for k in ("params", "m", "v"):
        assert np.array_equal(sa[k].view(np.uint32), sb[k].view(np.uint32)), k
    with pytest.raises(B.ReloError):
        B.regressor_set_state(b, dict(state, step=-1))


def _near_tie_in_trace(tr):
    """True when some round's cut between kept and dropped hypotheses is within the energy
    tolerance (FP32 may then keep either side)."""
    for rd in tr.rounds:
        E, alive = rd["energy"], rd["alive_before"]
        srt = sorted(alive.tolist(), key=lambda h: (E[h], h))
        keep = (len(srt) + 1) // 2
        if keep < len(srt):
            a, b = E[srt[keep - 1]], E[srt[keep]]
            if np.isfinite(a) and np.isfinite(b) and abs(b - a) <= 1e-5 * max(abs(a), abs(b)) + 1e-6:
                return True
    return False


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_learned_ransac_matches_oracle_on_constructed_cells(room, oracle_room, seed):
    """The cell-grid RANSAC of the learned path (relo_regressor_relocalise_cells: cell forest,
    coarse view, preemptive RANSAC) against the oracle's RANSAC on the cell forest of the same
    cells.  The cells are built so that hypotheses exist: each cell's value is the true scene
    coordinate of its centre pixel plus 1 cm Gaussian noise, with 15 % of the cells replaced by
    coordinates up to 2 m away (outliers), and log-variances around log(0.03^2)."""
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    P = synth.training_poses(world, 3, seed=93 + seed)[seed]
    d, _ = oracle_room.raycast(intr, P)
    y, m = R.cell_targets(d, intr, P, ORIGIN)
    rng = np.random.default_rng(100 + seed)
    cells = np.zeros(y.shape[:2] + (4,), np.float64)
    cells[..., :3] = y + 0.01 * rng.standard_normal(y.shape)
    out = rng.random(y.shape[:2]) < 0.15
    cells[out, :3] += rng.uniform(-2.0, 2.0, (int(out.sum()), 3))
    cells[..., 3] = np.log(0.03 ** 2) + 0.3 * rng.standard_normal(y.shape[:2])
    cells = cells.astype(np.float32)
    prm = B.ransac_params(n_hyps=64, batch=64, seed=seed, max_tries=2000)
    ws = torch.empty(B.regressor_relocalise_workspace_size(320, 240, prm), dtype=torch.uint8, device=DEV)
    res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
    B.regressor_relocalise_cells(torch.from_numpy(cells).to(DEV), ORIGIN, _u16(d), intr, prm, ws, res)
    torch.cuda.synchronize()
    r = B.result_from_bytes(res)
    dl, ci = R.cell_view(d, intr)
    forest, leaves = R.cell_forest(cells.astype(np.float64), ORIGIN, dl > 0)
    ro = oracle.preemptive_ransac(dl, ci, leaves, forest, oracle.RansacParams(n_hyps=64, batch=64, seed=seed,
                                                                              max_tries=2000), trace=True)
    assert ro["valid"] and r["status"] == 0
    assert r["n_valid"] == int((dl > 0).sum())
    dt, dr = oracle.pose_error(ro["pose"], P)
    assert dt <= 0.05 and dr <= 5.0
    if not _near_tie_in_trace(ro["trace"]):
        assert r["hypothesis"] == ro["index"]
        assert np.abs(r["pose"][:3] - ro["pose"][:3]).max() < 1e-4
        assert abs(r["energy"] - ro["energy"]) <= 1e-5 * abs(ro["energy"])


def test_training_fits_fixed_views(room, oracle_room):
    """Trained on four fixed views (6000 steps of the configured schedule), the regressor brings
    their cells from metres to centimetres (measured: median 2.0 m -> 10 cm, a tenth under 3.4 cm;
    bars 15 cm and 5 cm) and its
    RANSAC relocalises some of them: the optimiser, the loss and the data path work, so the
    network's failure to generalise over the house within the configured budget is a matter of
    data and capacity (with BF16 activations it plateaus at a few centimetres even here), not of a
    broken training loop."""
    from paper_1801_08361_gb300.presets import learning_rate
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    poses = synth.training_poses(world, 2, seed=95)[:4]
    ds, cs = zip(*[oracle_room.raycast(intr, P) for P in poses])
    d, c = np.stack(ds), np.stack(cs)
    reg = B.Regressor(seed=8, origin=ORIGIN)
    n = len(poses)
    ws = torch.empty(B.regressor_workspace_size(n, 320, 240, True), dtype=torch.uint8, device=DEV)
    dd, cc = _u16(d), torch.from_numpy(c).to(DEV)
    out = torch.zeros((n, 30, 40, 4), dtype=torch.float32, device=DEV)
    wsf = torch.empty(B.regressor_workspace_size(n, 320, 240, False), dtype=torch.uint8, device=DEV)

    def cell_errors():
        B.regressor_forward(reg, dd, cc, out, wsf)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        errs = []
        for k, P in enumerate(poses):
            y, m = R.cell_targets(d[k], intr, P, ORIGIN)
            errs.append(np.linalg.norm(o[k, ..., :3] - y, axis=-1)[m])
        return np.concatenate(errs)

    before = np.median(cell_errors())
    steps = 6000
    for k in range(steps):
        B.regressor_train_step(reg, dd, cc, intr, poses, learning_rate(k, steps, 1e-3, 0.05), ws)
    err = cell_errors()
    print(f"fixed views: median cell error {before:.3f} m -> {np.median(err):.3f} m, "
          f"10th percentile {np.percentile(err, 10):.3f} m")
    assert before > 0.5
    assert np.median(err) < 0.15 and np.percentile(err, 10) < 0.05
    prm = B.ransac_params(n_hyps=256, batch=64, seed=1, max_tries=2000)
    wsr = torch.empty(B.regressor_relocalise_workspace_size(320, 240, prm), dtype=torch.uint8, device=DEV)
    ok = 0
    for k, P in enumerate(poses):
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        B.regressor_relocalise(reg, dd[k], cc[k], intr, prm, wsr, res)
        torch.cuda.synchronize()
        r = B.result_from_bytes(res)
        dt, dr = oracle.pose_error(r["pose"], P)
        ok += int(r["status"] == 0 and dt <= 0.05 and dr <= 5.0)
    assert ok >= 1, ok


@pytest.fixture(scope="module")
def gpu_room_scene(room):
    return B.Scene(room[1], 16)


def _learned_items(room, room_training, scene, reg, forest, n, seed):
    world, _ = room
    intr = synth.Intrinsics.for_size(160, 120)
    qs = synth.query_poses(world, [f[1] for f in room_training], n, seed=seed)
    return [dict(scene_b=scene, scene_a=scene, regressor_a=reg, forest_a=forest, intr=intr, pose_b=P, seed=10 + i)
            for i, P in enumerate(qs)]


def test_learned_batch_equals_single_calls(room, room_training, gpu_room_scene):
    """Learned attempts in a batch give exactly the results of relo_regressor_relocalise +
    relo_verify on the same query (same kernels, same inputs)."""
    reg = B.Regressor(seed=7, origin=ORIGIN)
    items = _learned_items(room, room_training, gpu_room_scene, reg, None, 3, seed=61)
    prm = B.ransac_params(n_hyps=32, batch=64, max_tries=2000)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
    got = B.relocalise_batch(att, prm, ws)
    for it, g in zip(items, got):
        intr = it["intr"]
        depth = torch.zeros((intr.height, intr.width), dtype=torch.int16, device=DEV)
        rgba = torch.zeros((intr.height, intr.width, 4), dtype=torch.uint8, device=DEV)
        B.raycast_view(gpu_room_scene, intr, it["pose_b"], depth, rgba)
        p1 = B.ransac_params(n_hyps=32, batch=64, max_tries=2000, seed=it["seed"])
        wsr = torch.empty(B.regressor_relocalise_workspace_size(intr.width, intr.height, p1), dtype=torch.uint8,
                          device=DEV)
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        B.regressor_relocalise(reg, depth, rgba, intr, p1, wsr, res)
        B.verify(gpu_room_scene, intr, depth, res)
        torch.cuda.synchronize()
        s = B.result_from_bytes(res)
        assert g["path"] == B.PATH_LEARNED
        for k in ("hypothesis", "status", "n_valid", "omega", "omega_a", "omega_ab", "sum_absdiff_mm", "verified"):
            assert g[k] == s[k], k
        assert np.array_equal(g["pose"], s["pose"])


def test_fallback_reports_the_forest_result(room, room_training, gpu_room_scene, room_forest):
    """An untrained regressor fails verification; the forest fallback then runs on the device and
    its result equals the forest-only batch's."""
    reg = B.Regressor(seed=8, origin=ORIGIN)
    forest = B.Forest(room_forest.nodes, room_forest.modes, room_forest.n_modes, max_modes=10)
    learned = _learned_items(room, room_training, gpu_room_scene, reg, forest, 4, seed=62)
    plain = [dict(it, regressor_a=None) for it in learned]
    prm = B.ransac_params(n_hyps=32, batch=64, max_tries=2000)
    out = []
    for items in (learned, plain):
        att = B.make_attempts(items)
        ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=DEV)
        out.append(B.relocalise_batch(att, prm, ws))
    for l, f in zip(*out):
        assert f["path"] == B.PATH_FOREST
        if l["path"] == B.PATH_FALLBACK:
            for k in ("hypothesis", "status", "omega_a", "omega_ab", "sum_absdiff_mm", "verified", "energy"):
                assert l[k] == f[k], k
            assert np.array_equal(l["pose"], f["pose"])
        else:
            assert l["path"] == B.PATH_LEARNED and l["verified"] == 1
    assert any(l["path"] == B.PATH_FALLBACK for l in out[0])


def test_full_size_forward_matches_oracle_on_sampled_cells(params):
    """A 640 x 480 forward pass (the bench's view size) on sampled interior cells.  Output cell c
    depends only on input pixels 8c - 47 .. 8c + 47 per axis (five 3x3 layers at 1/8 resolution
    and three stride-2 layers), so the oracle's forward pass on a 128 x 128 crop whose corner is a
    multiple of 8 gives exactly the full image's cells 6 .. 10 of that crop (same tolerance as the
    small-view test: the oracle is given the BF16 weights and input the kernels multiply)."""
    rng = np.random.default_rng(12)
    n, H, W = 2, 480, 640
    d = rng.integers(400, 9000, (n, H, W)).astype(np.uint16)
    d[rng.random((n, H, W)) < 0.05] = 0
    c = rng.integers(0, 256, (n, H, W, 4)).astype(np.uint8)
    reg = B.Regressor(_flat(params), origin=ORIGIN)
    out = torch.zeros((n, H // 8, W // 8, 4), dtype=torch.float32, device=DEV)
    ws = torch.empty(B.regressor_workspace_size(n, W, H, False), dtype=torch.uint8, device=DEV)
    B.regressor_forward(reg, _u16(d), torch.from_numpy(c).to(DEV), out, ws)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    pq = _operands(params, np.zeros((1, 8, 8, 4)))[0]
    crops = [(0, 64, 96), (0, 256, 400), (1, 128, 480), (1, 320, 16)]   # (image, y0, x0)
    g_all, w_all = [], []
    for i, y0, x0 in crops:
        x = _bf16(R.network_input(d[i, y0:y0 + 128, x0:x0 + 128], c[i, y0:y0 + 128, x0:x0 + 128]))[None]
        want, _ = R.forward(pq, x)
        cy, cx = y0 // 8, x0 // 8
        w_all.append(want[0, 6:11, 6:11])
        g_all.append(got[i, cy + 6:cy + 11, cx + 6:cx + 11])
    g_all, w_all = np.stack(g_all), np.stack(w_all)
    rel = np.linalg.norm(g_all - w_all) / np.linalg.norm(w_all)
    assert rel <= 1e-2, rel


def _learned_success(reg, scene, intr, queries, noise_seed):
    """Successes (<= 5 cm, <= 5 deg) of learned-only relocalisation (regressor RANSAC + verification)."""
    prm = B.ransac_params(n_hyps=256, batch=64, max_tries=10000)
    ws = torch.empty(B.regressor_relocalise_workspace_size(intr.width, intr.height, prm), dtype=torch.uint8,
                     device=DEV)
    d = torch.zeros((intr.height, intr.width), dtype=torch.int16, device=DEV)
    c = torch.zeros((intr.height, intr.width, 4), dtype=torch.uint8, device=DEV)
    ok = 0
    for k, P in enumerate(queries):
        nz = torch.from_numpy(synth.depth_noise(intr.height, intr.width, noise_seed + k)).to(DEV)
        B.raycast_view(scene, intr, P, d, c, noise_dev=nz)
        res = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=DEV)
        B.regressor_relocalise(reg, d, c, intr, B.ransac_params(n_hyps=256, batch=64, max_tries=10000, seed=k), ws,
                               res)
        B.verify(scene, intr, d, res)
        torch.cuda.synchronize()
        r = B.result_from_bytes(res)
        dt, dr = oracle.pose_error(r["pose"], P)
        ok += int(r["status"] == 0 and r["verified"] == 1 and dt <= 0.05 and dr <= 5.0)
    return ok


def test_online_training_gains_relocalisations(room, room_training, gpu_room_scene):
    """What the trained network gains: on the tiny room, 2000 online steps of 16 noisy 320 x 240
    renders along the trajectory (the configured schedule) against the same network untrained,
    both relocalising 64 perturbed query views on their own (no forest), verified and within
    5 cm / 5 degrees of the truth."""
    from paper_1801_08361_gb300.presets import LEARNED, learning_rate
    world, _ = room
    intr = synth.Intrinsics.for_size(320, 240)
    train = [f[1] for f in room_training]
    queries = synth.query_poses(world, train, 64, seed=501)
    untrained = B.Regressor(seed=21, origin=ORIGIN)
    reg = B.Regressor(seed=21, origin=ORIGIN)
    nb, steps = 16, 2000
    pool = synth.query_poses(world, train, steps * nb, seed=502)
    d = torch.zeros((nb, 240, 320), dtype=torch.int16, device=DEV)
    c = torch.zeros((nb, 240, 320, 4), dtype=torch.uint8, device=DEV)
    noise = torch.from_numpy(np.stack([synth.depth_noise(240, 320, 600 + k) for k in range(nb)])).to(DEV)
    ws = torch.empty(B.regressor_workspace_size(nb, 320, 240, True), dtype=torch.uint8, device=DEV)
    wsv = torch.empty(B.raycast_views_workspace_size(nb), dtype=torch.uint8, device=DEV)
    for s in range(steps):
        P = pool[s * nb:(s + 1) * nb]
        B.raycast_views(gpu_room_scene, intr, P, d, c, noise_dev=noise, workspace_dev=wsv)
        B.regressor_train_step(reg, d, c, intr, P, learning_rate(s, steps, LEARNED.extra["lr"],
                                                                  LEARNED.extra["warmup"]), ws)
    torch.cuda.synchronize()
    gained = _learned_success(reg, gpu_room_scene, intr, queries, 700)
    base = _learned_success(untrained, gpu_room_scene, intr, queries, 700)
    print(f"learned-only relocalisations of 64 room queries: trained {gained}, untrained {base}")
    assert base == 0
    assert gained >= 2, gained
