"""Relocalisation attempts per second on the paper-sized workload (one JSON line on rank 0).

Workload (synthetic, seeded): a 10 x 8 x 3 m house of 2 x 3 rooms (0.1 m interior walls with
1 x 2 m doorways, 200 furniture boxes) sampled into a 5 mm voxel-hash TSDF (2^20 buckets); a
regression forest of 5 trees of depth 15 with random pixel-pair splits, its leaves filled on the
GPU from noisy 640 x 480 training renders along a trajectory (reservoirs of 1024, <= 10
mean-shift modes); queries are 640 x 480 views near that trajectory with depth noise
sigma = 1.5 mm z^2.  One attempt (Sec. 3.3.1, Fig. 3) = raycast the query RGB-D view of scene b,
evaluate it through a's forest, preemptive RANSAC (1024 hypotheses, 64 pixels per round, 10
halvings), depth raycast of scene a at the proposed pose and the Omega / mu verification.
Scene a and b are the same house here (an agent relocalising against its own map).

A step = one batch of ``--batch`` attempts: one replay of the CUDA graph relo_batch_capture
recorded from relo_batch_run (inputs resident in HBM; the L2 is flushed between steps; each step
timed with CUDA events on the launching stream).
``e2e`` = the same metric through relo_relocalise_batch with the query noise images copied from
pinned host memory and the results copied back inside the timed region, one step after another.
``--impl reference`` times the CPU oracle (the deliberately slow FP64 reference) instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

# the CPU baselines state the cores they use: one BLAS / OpenMP thread per process (set before
# numpy loads its BLAS)
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "reloc attempts/s at 640x480 (forest vs learned, same success); % HBM roofline"
UNIT = "attempts/s"
WORKLOAD = "house 10x8x3 m, 5 mm voxels, 2^20 buckets; 640x480 queries, depth noise 1.5 mm z^2; forest T=5 D=15, " \
           "reservoir 1024, <=10 modes; preemptive RANSAC K=1024, B=64"
from paper_1801_08361_gb300.presets import HOUSE, LEARNED, SERVING, learning_rate  # noqa: E402

W, H = HOUSE.sizes[0]
T_TREES, DEPTH, MAX_MODES, CAPACITY = HOUSE.trees, HOUSE.depth, HOUSE.max_modes, HOUSE.reservoir
K_HYPS, B_PIX = HOUSE.hypotheses[0], HOUSE.batch_pixels
TRAIN_PER_ROOM = HOUSE.train_per_room
L2_FLUSH_BYTES = 512 << 20

# Algorithmic bytes per unit: per query pixel the raycast must write depth (2 B) + colour (4 B)
# and the verification raycast must read D_b (2 B); each touches the distinct scene data its
# samples need. The per-pixel scene-data figures below are the oracle's exact counts of distinct
# voxels (4 B tsdf, 4 B colour) and block-table entries (16 B) touched, averaged over 8 query views
# of this workload (oracle/algorithmic_bytes.py). A verification stage is its raycast plus a
# one-block-per-attempt decision whose bytes are negligible.
# The forest stage reads each query pixel's depth (2 B) and colour (4 B) once and writes T = 5
# leaf ids (10 B); its 2.6 MB of nodes per launch are negligible.
ALG_BYTES_PER_PIXEL = {
    "query_raycast": 50.66,
    "forest_eval": 16.0,
    "forest_verify": 35.87,
    "learned_verify": 35.87,
}
# DRAM bytes (read + write) per attempt of the stage's main kernel: the ncu captures summarised in
# profiles/attempt_dram_house_640x480_batch32.md, profiles/raycast_apron_house_640x480_batch32.md
# and profiles/forest_kernel_house_640x480_batch32.md
# (32 attempts per launch, the current kernels)
# divided by 32; a launch of A attempts is reported as A times that (attempts are independent, so
# the traffic grows with their number; None: not captured for the current code).
PROFILED_TRAFFIC_BYTES_PER_ATTEMPT = {
    "query_raycast": (974674688 + 151929344) / 32,
    "forest_eval": (101758464 + 64701440) / 32,
    "forest_hypotheses": (161393152 + 7238400) / 32,
    "forest_verify": (654187520 + 6215424) / 32,
}
# What limits each stage's main kernel (profiles/attempt_kernels_house_640x480_batch128.md,
# profiles/forest_kernel_house_640x480_batch32.md and profiles/raycast_apron_house_640x480_batch32.md; the roofline fraction divides by DRAM
# bandwidth or an integer-issue peak; these kernels gather from L2 and are bound elsewhere).
PROFILED_LIMITER = {
    "query_raycast": "instruction issue (74 % active at 63 % warps active; 23.5 of 32 lanes per instruction as rays "
                     "end at different steps); DRAM 17 % of peak, L2 hit 51 %",
    "forest_eval": "instruction issue (65 % active at 97 % warps active, about 58 instructions per node "
                   "visit) and dependent node and probe loads (L1 hit 23 %, L2 hit 98 %)",
    "forest_hypotheses": "L2 throughput (63 %, L2 hit 98 %): four random 16-byte gathers per try",
    "forest_verify": "instruction issue (74 % active at 61 % warps active; 23.2 of 32 lanes per instruction); "
                     "DRAM 11 % of peak, L2 hit 54 %",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=256, help="attempts per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fusion-frames", type=int, default=96, help="frames of the TSDF fusion section (0: skip)")
    ap.add_argument("--fragments", type=int, default=1, help="measure the batched 8-fragment configuration (0: skip)")
    ap.add_argument("--tiny", type=int, default=1, help="measure the tiny-room configuration (0: skip)")
    ap.add_argument("--profile-fusion", type=int, default=0, help="(ncu) fuse this many frames and exit, no JSON")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the launch schedule with relo_batch_autotune (default: the default schedule, "
                         "which the tuner matches within noise on this workload)")
    ap.add_argument("--profile-steps", type=int, default=0, help="(ncu) run this many steps and exit, no JSON")
    ap.add_argument("--profile-learned", type=int, default=0,
                    help="(ncu) this many regressor forward passes over 16 house views, then exit, no JSON")
    ap.add_argument("--learned-fragments", type=int, default=0,
                    help="train a regressor on each house fragment for this many steps and relocalise within it "
                         "(0: skip)")
    ap.add_argument("--train-steps", type=int, default=2000,
                    help="online training steps of the learned regressor (0: skip the learned path)")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="seconds per serving operating point (0: skip the serving measurement)")
    return ap.parse_args()


def rank_seeds(rank, set_index, k):
    """Seeds of attempt k of query set set_index on this rank: (query-set seed, noise seed, RANSAC
    seed).  Ranks and sets draw disjoint seeds, so each rank relocalises attempts of its own."""
    return (1000 * (rank + 1) + set_index, 5_000_000 + 100_000 * rank + 10_000 * set_index + k,
            (rank << 40) + (set_index << 20) + k)


def reduce_max(value, world_size, device="cpu"):
    """The largest of the ranks' values (the job's time is its slowest rank's); any backend."""
    if world_size == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(attempts_per_rank_step, steps, world_size, elapsed_s):
    """Whole-job attempts/s: every rank's attempts over the slowest rank's time (weak scaling)."""
    return attempts_per_rank_step * steps * world_size / elapsed_s


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------------
# Workload construction (not timed)
# ------------------------------------------------------------------------------------------------
def build_workload(seed_offset=0):
    from paper_1801_08361_gb300 import synth
    world = synth.house_world(2)
    blocks = synth.sample_scene(world)
    intr = synth.Intrinsics.for_size(W, H, 12.0)
    train = synth.training_poses(world, TRAIN_PER_ROOM, seed=11)
    nodes = synth.random_forest_nodes(T_TREES, DEPTH, seed=5, depth_tau=100, colour_tau=32)
    return world, blocks, intr, train, nodes


def query_set(world, train, n, seed):
    from paper_1801_08361_gb300 import synth
    return synth.query_poses(world, train, n, seed=seed)


def clocks_sampler(local_rank):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--id={local_rank}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def clocks_summary(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def bf16_peaks():
    """(burst, sustained) dense BF16 TFLOP/s: measured, else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "fallback"


# ------------------------------------------------------------------------------------------------
# CPU oracle: whole attempts of the benchmark's own query list
# ------------------------------------------------------------------------------------------------
# The oracle fills its forest's leaves itself, from its own renders of the house at every training
# pose (the GPU's trajectory and noise seeds) but on every 8th pixel of every 8th row (the GPU
# trains on every 2nd): its mean shift on the GPU's reservoirs would take hours.  Nothing it uses
# comes from the CUDA library; the GPU is handed this forest (bench: "precision") to run the same
# attempts on the same modes.
ORACLE_TRAIN_STRIDE = 8


def oracle_setup(blocks, intr, train, nodes, threads):
    """The oracle's scene and forest (untimed inputs of its attempts).  ``threads`` render the
    training views and compute the leaves' modes concurrently (the C calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_1801_08361_gb300 import synth
    sc = oracle.Scene(blocks)

    def render(i):
        return sc.raycast(intr, train[i], noise=synth.depth_noise(H, W, 100 + i))

    with ThreadPoolExecutor(threads) as ex:
        imgs = list(ex.map(render, range(len(train))))
    frames = [(intr, P, d, c) for P, (d, c) in zip(train, imgs)]
    forest = oracle.train_forest(nodes, frames, oracle.LeafParams(capacity=CAPACITY, max_modes=MAX_MODES, seed=7,
                                                                  stride=ORACLE_TRAIN_STRIDE), threads=threads)
    return sc, forest


def attempt_spec(rank, set_index, k, qs):
    """(query pose, noise seed, RANSAC seed) of attempt k of a query set qs: the GPU batch's own."""
    s = rank_seeds(rank, set_index, k)
    return qs[k], s[1], s[2]


def oracle_attempt(sc, forest, intr, pose_b, noise_seed, ransac_seed):
    """One whole attempt by the oracle (Sec. 3.3.1, Fig. 3: render b, forest of a, preemptive
    RANSAC, verification raycast of a): (seconds, result).  The noise image is made before the
    clock starts (it is an input, resident on the GPU side too)."""
    import oracle
    from paper_1801_08361_gb300 import synth
    noise = synth.depth_noise(H, W, noise_seed)
    prm = oracle.RansacParams(n_hyps=K_HYPS, batch=B_PIX, max_tries=10000, seed=ransac_seed)
    t0 = time.perf_counter()
    res = oracle.relocalise(sc, pose_b, forest, sc, intr, prm, noise=noise)
    return time.perf_counter() - t0, res


# state the reference arm's worker processes inherit (forked before any of them starts; the
# reference arm never touches the GPU)
_REF_STATE = {}


def _ref_worker(k):
    st = _REF_STATE
    pose, nseed, rseed = st["specs"][k % len(st["specs"])]
    sec, res = oracle_attempt(st["sc"], st["forest"], st["intr"], pose, nseed, rseed)
    ok = bool(res["verified"]) and oracle_success(res["pose"], pose)
    return sec, ok


def oracle_success(P_est, P_gt):
    import oracle
    dt, dr = oracle.pose_error(P_est, P_gt)
    return dt <= 0.05 and dr <= 5.0


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------------------------
# Reference arm: the CPU oracle on every host core, whole attempts
# ------------------------------------------------------------------------------------------------
def run_reference(args):
    """The oracle on every host core: each step runs one whole attempt per core in parallel
    processes (forked from a parent that never touches the GPU, after the scene and the forest
    are built) on the GPU batch's first query set (pose, noise, RANSAC seed), and its wall clock is
    the step's time."""
    import multiprocessing as mp
    rank, world_size, _ = dist_env()
    if rank != 0:
        return 0
    world, blocks, intr, train, nodes = build_workload()
    cores = cores_used()
    t_setup = time.perf_counter()
    sc, forest = oracle_setup(blocks, intr, train, nodes, cores)
    t_setup = time.perf_counter() - t_setup
    qs = query_set(world, train, args.batch, seed=rank_seeds(0, 0, 0)[0])
    specs = [attempt_spec(0, 0, k, qs) for k in range(args.batch)]
    _REF_STATE.update(sc=sc, forest=forest, intr=intr, specs=specs)
    wall, per_attempt, ok = [], [], 0
    with mp.get_context("fork").Pool(cores) as pool:
        for s in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            out = pool.map(_ref_worker, [s * cores + k for k in range(cores)])
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                wall.append(dt)
                per_attempt += [sec for sec, _ in out]
                ok += sum(int(v) for _, v in out)
    elapsed = sum(wall)
    value = cores * args.steps / elapsed
    sample = (f"whole 640x480 attempts (query raycast, forest, 1024-hypothesis preemptive RANSAC, verification "
              f"raycast) of the GPU batch's first query set (same poses, noise and RANSAC seeds), with a forest the "
              f"oracle filled itself (every training pose, every {ORACLE_TRAIN_STRIDE}th pixel and row); {cores} "
              f"processes, one attempt each per step; value = attempts / wall-clock seconds of the timed steps; "
              f"seconds per attempt in one process {statistics.median(per_attempt):.2f} (median); "
              f"setup {t_setup:.0f} s untimed")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed * 1000.0 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "attempts_per_step": cores,
                       "success_rate": ok / max(1, cores * args.steps)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# Our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_1801_08361_gb300 import binding as B
    from paper_1801_08361_gb300 import synth

    rank, world_size, local = dist_env()
    if world_size > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world_size > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    world, blocks, intr, train, nodes = build_workload()
    scene = B.Scene(blocks, 20)
    if args.profile_fusion:
        # profiler runs of the fusion kernels: the frames sit in an NVTX range named "fusion"
        args.fusion_frames = args.profile_fusion
        fusion_section(args, B, synth, torch, dev, scene, world, intr, train, nvtx="fusion", capacity=1 << 18)
        return 0
    if args.profile_learned:
        # profiler runs of the regressor's forward pass: the passes sit in an NVTX range "learned"
        profile_learned(args, B, synth, torch, dev, scene, world, intr, train)
        return 0
    forest = B.Forest(nodes, max_modes=MAX_MODES)
    # relocaliser training on the GPU: noisy renders along the trajectory, stride 2
    B.forest_train_begin(forest, B.train_params(capacity=CAPACITY, stride=2, seed=7))
    depth = torch.zeros((H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((H, W, 4), dtype=torch.uint8, device=dev)
    for i, P in enumerate(train):
        nz = torch.from_numpy(synth.depth_noise(H, W, 100 + i)).to(dev)
        B.raycast_view(scene, intr, P, depth, rgba, noise_dev=nz)
        B.forest_train_frame(forest, intr, P, depth, rgba)
    B.forest_train_finish(forest)
    del depth, rgba

    A = args.batch
    n_sets = max(1, min(4, args.warmup + args.steps))
    prm = B.ransac_params(n_hyps=K_HYPS, batch=B_PIX, max_tries=10000)
    sets = []
    for si in range(n_sets):
        qs = query_set(world, train, A, seed=rank_seeds(rank, si, 0)[0])
        noise = torch.from_numpy(np.stack([synth.depth_noise(H, W, rank_seeds(rank, si, k)[1])
                                           for k in range(A)])).to(dev)
        items = [dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=qs[k], noise=noise[k],
                      seed=rank_seeds(rank, si, k)[2]) for k in range(A)]
        att = B.make_attempts(items)
        ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
        bt = B.Batch(att, prm, ws)
        bt.enable_timing(True)
        if si == 0:
            # launch schedule: the autotuner's pick on the first set (same shapes in every set)
            schedule = bt.autotune(repeats=2) if args.autotune else bt.schedule()
        else:
            bt.set_schedule(**schedule)
        res = torch.zeros(A * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
        bt.capture(res)            # one CUDA graph per batch; its replays carry the stage events
        sets.append(dict(qs=qs, noise=noise, att=att, ws=ws, batch=bt, res=res))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    if args.profile_steps:
        # profiler runs: the steps sit in an NVTX range named "steps" (ncu --nvtx-include steps/)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("steps")
        for s in range(args.profile_steps):
            sets[s % n_sets]["batch"].run(sets[s % n_sets]["res"])
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return 0

    for s in range(args.warmup):
        flush.zero_()
        sets[s % n_sets]["batch"].replay()
    torch.cuda.synchronize()

    # ---- device-resident timing -----------------------------------------------------------
    if world_size > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks_sampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_tot = {k: 0.0 for k in B.STAGES}
    results = []
    for s in range(args.steps):
        st = sets[(args.warmup + s) % n_sets]
        flush.zero_()
        ev[s][0].record(stream)
        st["batch"].replay()
        ev[s][1].record(stream)
        torch.cuda.synchronize()
        for k, v in st["batch"].stage_ms().items():
            stage_tot[k] += v
        results.append((st, st["res"].cpu()))
    step_ms = [a.elapsed_time(b) for a, b in ev]
    clocks = clocks_summary(clk)
    elapsed = reduce_max(sum(step_ms) / 1000.0, world_size, dev)
    value = job_throughput(A, args.steps, world_size, elapsed)

    # success (the criterion of Sec. 4.2.2: <= 5 cm and <= 5 degrees) and verification rate
    succ = ver = n = 0
    tries_per_step = 0
    for st, raw in results:
        for k in range(A):
            r = B.result_from_bytes(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES])
            succ += int(success(r, st["qs"][k]))
            tries_per_step += r["tries"]
            ver += int(r["verified"])
            n += 1

    # ---- end to end through the public API (host buffers) ----------------------------------
    # Every step copies its query noise from pinned host memory into the device, prepares its batch
    # (relo_batch_prepare: descriptors uploaded), runs it (relo_batch_run), copies its results into
    # pinned host memory and waits for them; the L2 is flushed before each run.  Steps are
    # pipelined on two streams: while step s's kernels run, step s+1's noise is copied in and its
    # batch prepared (its uploads do not wait for the run, which is on a non-blocking stream), so
    # the GPU does not idle between steps.  The one-shot call (relo_relocalise_batch: prepare, run,
    # results into host memory, wait) is also timed step after step, as `serial`.
    host_noise = [torch.empty((A, H, W), dtype=torch.float32, pin_memory=True) for _ in range(n_sets)]
    for si in range(n_sets):
        host_noise[si].copy_(sets[si]["noise"].cpu())
    host_results = (B.PoseResult * A)()
    run_stream, copy_stream = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    res_dev = [torch.empty(A * B.RESULT_BYTES, dtype=torch.uint8, device=dev) for _ in range(2)]
    res_host = [torch.empty(A * B.RESULT_BYTES, dtype=torch.uint8, pin_memory=True) for _ in range(2)]

    def set_of(s):
        return (args.warmup + s) % n_sets

    def copy_noise(s):
        with torch.cuda.stream(copy_stream):
            sets[set_of(s)]["noise"].copy_(host_noise[set_of(s)], non_blocking=True)

    def prepare(s):
        return B.Batch(sets[set_of(s)]["att"], prm, sets[set_of(s)]["ws"])

    def e2e_pipelined(n):
        if world_size > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        copy_noise(0)
        nxt = prepare(0)
        copy_stream.synchronize()
        for s in range(n):
            cur = nxt
            with torch.cuda.stream(run_stream):
                flush.zero_()
                cur.run(res_dev[s & 1], stream=run_stream)
                res_host[s & 1].copy_(res_dev[s & 1], non_blocking=True)
            if s + 1 < n:
                copy_noise(s + 1)
                nxt = prepare(s + 1)
            run_stream.synchronize()
            copy_stream.synchronize()
            del cur
        return reduce_max(time.perf_counter() - t0, world_size, dev)

    def e2e_serial(n):
        if world_size > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(n):
            i = set_of(s)
            sets[i]["noise"].copy_(host_noise[i], non_blocking=True)
            flush.zero_()
            B.relocalise_batch_into(sets[i]["att"], prm, sets[i]["ws"], host_results)
        return reduce_max(time.perf_counter() - t0, world_size, dev)

    e2e_pipelined(min(args.warmup, n_sets))  # untimed warm-up of both forms
    e2e_serial(min(args.warmup, n_sets))
    clk_e2e = clocks_sampler(local)
    e2e_value = job_throughput(A, args.steps, world_size, e2e_pipelined(args.steps))
    e2e_clocks = clocks_summary(clk_e2e)
    e2e_serial_value = job_throughput(A, args.steps, world_size, e2e_serial(args.steps))

    # ---- the RANSAC of each pass in one persistent launch (schedule option), same batch ------
    persistent = None
    if rank == 0:
        persistent = persistent_section(args, B, torch, sets[0], schedule, flush, stream)

    # ---- the learned path (not part of the timed forest steps) -----------------------------
    learned = None
    if args.train_steps > 0 and rank == 0:
        learned = learned_section(args, B, synth, torch, dev, scene, forest, world, intr, train, sets[0], prm,
                                  stream)

    # ---- serving (not part of the timed steps) ----------------------------------------------
    serving = None
    if args.serve_seconds > 0 and rank == 0:
        serving = serving_section(args, B, torch, dev, sets[0], prm)

    # ---- the learned path on each fragment (optional, not part of the timed steps) --------------
    learned_frag = None
    if args.learned_fragments > 0 and rank == 0:
        learned_frag = learned_fragments_section(args, B, synth, torch, dev, stream)

    # ---- the tiny configuration (not part of the timed steps) ---------------------------------
    tiny = None
    if args.tiny and rank == 0:
        tiny = tiny_section(args, B, synth, torch, dev, stream, flush)

    # ---- the batched configuration (not part of the timed steps) ------------------------------
    frag = None
    if args.fragments and rank == 0:
        frag = fragments_section(args, B, torch, dev, stream, flush)

    # ---- TSDF fusion (not part of the timed steps) ------------------------------------------
    fusion = None
    if args.fusion_frames > 0 and rank == 0:
        fusion = fusion_section(args, B, synth, torch, dev, scene, world, intr, train)

    # ---- roofline of the dominant stage ---------------------------------------------------
    dom = max(stage_tot, key=stage_tot.get)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roofs = {k: roofline(k, stage_tot[k] / args.steps, A, tries_per_step / args.steps, clocks, n_sms)
             for k in ("query_raycast", "forest_eval", "forest_hypotheses", "forest_verify") if stage_tot[k] > 0}
    roof = roofs.get(dom) or roofline(dom, stage_tot[dom] / args.steps, A, tries_per_step / args.steps, clocks, n_sms)

    cpu = precision = None
    if rank == 0 and world_size == 1 and not args.no_cpu_baseline:
        cpu, precision = oracle_section(args, B, torch, dev, scene, blocks, intr, train, nodes, sets[0], prm, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world_size, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed * 1000.0 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "attempts_per_step": A, "path": "forest",
                           "l2": "flushed between steps (512 MiB write)",
                           "success_rate": succ / n, "verified_rate": ver / n,
                           "stage_ms_per_step": {k: v / args.steps for k, v in stage_tot.items()},
                           "schedule": dict(schedule, autotuned=bool(args.autotune)),
                           "learned": learned, "serving": serving, "fusion": fusion, "precision": precision,
                           "fragments": frag, "tiny": tiny, "persistent_schedule": persistent,
                           "learned_fragments": learned_frag},
                "e2e": {"value": e2e_value, "unit": UNIT,
                        "h2d_bytes_per_step": A * H * W * 4 + A * ctypes_attempt_bytes(),
                        "d2h_bytes_per_step": A * B.RESULT_BYTES, "clocks": e2e_clocks,
                        "calls": "relo_batch_prepare + relo_batch_run per step, pipelined on two streams",
                        "serial": {"value": e2e_serial_value, "calls": "relo_relocalise_batch, step after step"}},
                "gpu_launches": sets[0]["batch"].launch_count * args.steps,
                "roofline": roof, "roofline_stages": roofs, "cpu_baseline": cpu, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world_size > 1:
        torch.distributed.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------------
# Learned path: online training of the regressor on renders of the house, then the same attempts
# relocalised with it (learned only, and with the forest as fallback)
# ------------------------------------------------------------------------------------------------
TRAIN_BATCH, TRAIN_LR = LEARNED.extra["train_batch"], LEARNED.extra["lr"]
REG_ORIGIN = LEARNED.extra["origin"]   # centre of the house


def regressor_flops_per_view():
    """Multiply-adds x 2 of one 640 x 480 forward pass (padded channel counts, as computed)."""
    chans = [(16, 64, 2), (64, 64, 2), (64, 64, 2)] + [(64, 64, 1)] * 4 + [(64, 8, 1)]
    h, w, fl = H, W, 0
    for cin, cout, st in chans:
        h, w = h // st, w // st
        fl += 2 * h * w * 9 * cin * cout
    return fl


def timed_replays(bt, torch, flush, stream, n):
    """ms per replay of a captured batch over n replays (L2 flushed before each)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        bt.replay()
        e[1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / n


def persistent_section(args, B, torch, st, schedule, flush, stream, n=5):
    """The step's batch with its RANSAC in one persistent launch against the per-stage launches:
    ms per batch (same results, checked), launches per batch."""
    bt = st["batch"]
    ref = st["res"].cpu()
    out = {}
    for name, persistent in (("stage_launches", 0), ("persistent", 1)):
        bt.set_schedule(**dict(schedule, persistent=persistent))
        bt.capture(st["res"])
        bt.replay()
        torch.cuda.synchronize()
        same = bool(torch.equal(st["res"].cpu(), ref))
        ms = timed_replays(bt, torch, flush, stream, n)
        out[name] = {"ms_per_batch": ms, "attempts_per_s": len(st["qs"]) / (ms / 1000.0),
                     "launches": bt.launch_count, "results_equal_default": same}
    bt.set_schedule(**schedule)
    bt.capture(st["res"])
    return out


def profile_learned(args, B, synth, torch, dev, scene, world, intr, train, n=16):
    poses = synth.query_poses(world, train, n, seed=77)
    depth = torch.zeros((n, H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((n, H, W, 4), dtype=torch.uint8, device=dev)
    wsv = torch.empty(B.raycast_views_workspace_size(n), dtype=torch.uint8, device=dev)
    B.raycast_views(scene, intr, poses, depth, rgba, workspace_dev=wsv)
    reg = B.Regressor(seed=3, origin=REG_ORIGIN)
    out = torch.zeros((n, H // 8, W // 8, 4), dtype=torch.float32, device=dev)
    ws = torch.empty(B.regressor_workspace_size(n, W, H, False), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("learned")
    for _ in range(args.profile_learned):
        B.regressor_forward(reg, depth, rgba, out, ws)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()


def learned_section(args, B, synth, torch, dev, scene, forest, world, intr, train, st, prm, stream):
    nb = TRAIN_BATCH
    pool = synth.query_poses(world, train, args.train_steps * nb, seed=77)
    reg = B.Regressor(seed=3, origin=REG_ORIGIN)
    depth = torch.zeros((nb, H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((nb, H, W, 4), dtype=torch.uint8, device=dev)
    ws = torch.empty(B.regressor_workspace_size(nb, W, H, True), dtype=torch.uint8, device=dev)
    ws_views = torch.empty(B.raycast_views_workspace_size(nb), dtype=torch.uint8, device=dev)
    n_noise = 64  # noise images cycled over the renders (a multiple of the batch)
    noise = torch.from_numpy(np.stack([synth.depth_noise(H, W, 9000 + k) for k in range(n_noise)])).to(dev)
    loss = torch.zeros(args.train_steps, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    render_ms = train_ms = 0.0
    for s in range(args.train_steps):
        P = pool[s * nb:(s + 1) * nb]
        ev[0].record(stream)
        q = (s * nb) % n_noise
        B.raycast_views(scene, intr, P, depth, rgba, noise_dev=noise[q:q + nb], workspace_dev=ws_views)
        ev[1].record(stream)
        lr = learning_rate(s, args.train_steps, TRAIN_LR, LEARNED.extra["warmup"])
        B.regressor_train_step(reg, depth, rgba, intr, P, lr, ws, loss[s:s + 1])
        ev[2].record(stream)
        ev[2].synchronize()
        render_ms += ev[0].elapsed_time(ev[1])
        train_ms += ev[1].elapsed_time(ev[2])
    L = loss.cpu().numpy()
    train_step_ms = train_ms / args.train_steps
    # forward + backward-data + backward-weight: about 3 forward passes of work per view
    train_tflops = 3 * regressor_flops_per_view() * nb / (train_step_ms / 1000.0) / 1e12
    burst, sustained, peak_kind = bf16_peaks()
    # the training loop runs for seconds (the sustained peak); a forward runs inside one batch (burst)
    out = {"train_steps": args.train_steps, "train_batch": nb, "lr": TRAIN_LR,
           "train_ms_per_step": train_step_ms, "render_ms_per_step": render_ms / args.train_steps,
           "train_tflops": train_tflops, "train_frac": train_tflops / sustained,
           "bf16_peaks": {"burst": burst, "sustained": sustained, "source": peak_kind},
           "loss_first_last_100": [float(L[:100].mean()), float(L[-100:].mean())]}
    A = len(st["qs"])
    for name, with_forest in (("learned_only", False), ("learned_with_fallback", True)):
        items = [dict(scene_b=scene, forest_a=forest if with_forest else None, scene_a=scene, regressor_a=reg,
                      intr=intr, pose_b=st["qs"][k], noise=st["noise"][k], seed=k) for k in range(A)]
        att = B.make_attempts(items)
        wsb = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
        bt = B.Batch(att, prm, wsb)
        bt.enable_timing(True)
        res = torch.zeros(A * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
        bt.capture(res)
        for _ in range(2):
            bt.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times, stages = [], {}
        for _ in range(3):
            e0.record(stream)
            bt.replay()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            for k, v in bt.stage_ms().items():
                stages[k] = stages.get(k, 0.0) + v / 3
        raw = res.cpu()
        succ = ver = 0
        paths = [0, 0, 0]
        for k in range(A):
            r = B.result_from_bytes(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES])
            succ += int(success(r, st["qs"][k]))
            ver += int(r["verified"])
            paths[r["path"]] += 1
        ms = sorted(times)[1]
        out[name] = {"attempts_per_s": A / (ms / 1000.0), "ms_per_batch": ms, "success_rate": succ / A,
                     "verified_rate": ver / A, "paths_forest_learned_fallback": paths,
                     "learned_forward_ms": stages.get("learned_forward", 0.0),
                     "learned_forward_tflops": regressor_flops_per_view() * A / max(stages.get("learned_forward", 0.0), 1e-9) / 1e9}
        out[name]["learned_forward_frac"] = out[name]["learned_forward_tflops"] / burst
    return out


LEARNED_FRAG_QUERIES = 32


def learned_fragments_section(args, B, synth, torch, dev, stream):
    """The learned regressor on each of the 8 house fragments (1-3 rooms, 13-40 m^2, each in its
    own frame): trained online on noisy 640x480 renders near the fragment's own trajectory
    (args.learned_fragments steps of 16 views, the learned workload's schedule), then relocalising
    32 queries near that trajectory in the same fragment -- the learned path alone, and the
    fragment's forest alone on the same attempts."""
    from paper_1801_08361_gb300 import fragments as F
    world, frags, scenes, forests, _ = F.build(dev)
    intr = synth.Intrinsics.for_size(W, H, 12.0)
    nb, steps = TRAIN_BATCH, args.learned_fragments
    prm = B.ransac_params(n_hyps=K_HYPS, batch=B_PIX, max_tries=10000)
    depth = torch.zeros((nb, H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((nb, H, W, 4), dtype=torch.uint8, device=dev)
    ws = torch.empty(B.regressor_workspace_size(nb, W, H, True), dtype=torch.uint8, device=dev)
    ws_views = torch.empty(B.raycast_views_workspace_size(nb), dtype=torch.uint8, device=dev)
    n_noise = 64
    noise = torch.from_numpy(np.stack([synth.depth_noise(H, W, 9100 + k) for k in range(n_noise)])).to(dev)
    loss = torch.zeros(steps, dtype=torch.float32, device=dev)
    rows = []
    for k, f in enumerate(frags):
        S = f["scene_to_world"]
        centre_w = np.append((f["crop"][:3] + f["crop"][3:]) / 2.0, 1.0)
        reg = B.Regressor(seed=3, origin=tuple(float(x) for x in (np.linalg.inv(S) @ centre_w)[:3]))
        pool = [synth.world_to_scene_pose(P, S) for P in synth.query_poses(world, f["train_w"], steps * nb,
                                                                             seed=500 + k)]
        for s in range(steps):
            q = (s * nb) % n_noise
            B.raycast_views(scenes[k], intr, pool[s * nb:(s + 1) * nb], depth, rgba, noise_dev=noise[q:q + nb],
                            workspace_dev=ws_views)
            B.regressor_train_step(reg, depth, rgba, intr, pool[s * nb:(s + 1) * nb],
                                   learning_rate(s, steps, TRAIN_LR, LEARNED.extra["warmup"]), ws, loss[s:s + 1])
        torch.cuda.synchronize()
        L = loss.cpu().numpy()
        qs = [synth.world_to_scene_pose(P, S) for P in synth.query_poses(world, f["train_w"], LEARNED_FRAG_QUERIES,
                                                                           seed=900 + k)]
        qn = torch.from_numpy(np.stack([synth.depth_noise(H, W, 9500 + 100 * k + i)
                                        for i in range(LEARNED_FRAG_QUERIES)])).to(dev)
        row = {"fragment": k, "rooms": len(f["rooms"]), "loss_first_last_100": [float(L[:100].mean()),
                                                                                 float(L[-100:].mean())]}
        for name, learned in (("learned_only", True), ("forest_only", False)):
            items = [dict(scene_b=scenes[k], forest_a=None if learned else forests[k], scene_a=scenes[k],
                          regressor_a=reg if learned else None, intr=intr, pose_b=qs[i], noise=qn[i], seed=i)
                     for i in range(LEARNED_FRAG_QUERIES)]
            att = B.make_attempts(items)
            wsb = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
            bt = B.Batch(att, prm, wsb)
            res = torch.zeros(len(items) * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
            bt.run(res, stream=stream)
            torch.cuda.synchronize()
            raw = res.cpu()
            rs = [B.result_from_bytes(raw[i * B.RESULT_BYTES:(i + 1) * B.RESULT_BYTES]) for i in range(len(items))]
            row[name] = {"success": sum(int(success(r, qs[i])) for i, r in enumerate(rs)) / len(rs),
                         "verified": sum(int(r["verified"]) for r in rs) / len(rs)}
            del bt
        rows.append(row)
    n = len(rows)
    return {"train_steps": steps, "train_batch": nb, "queries_per_fragment": LEARNED_FRAG_QUERIES, "size": f"{W}x{H}",
            "per_fragment": rows,
            "learned_only_success": sum(r["learned_only"]["success"] for r in rows) / n,
            "forest_only_success": sum(r["forest_only"]["success"] for r in rows) / n}


# ------------------------------------------------------------------------------------------------
# The batched configuration: 8 house fragments, all 56 ordered pairs in one batch (mixed query
# sizes and hypothesis counts), one CUDA graph replay per step; the fragments' voxels exceed L2
# ------------------------------------------------------------------------------------------------
# Algorithmic bytes of one whole batch (python -m oracle.algorithmic_bytes fragments: the oracle's
# exact count of the distinct voxels and hash entries each raycast touches, plus the images read
# and written; the forest stage reads depth and colour and writes 5 leaf ids per pixel).
FRAG_ALG_BYTES = {"query_raycast": 1189722832, "forest_eval": 172339200, "forest_verify": 4181876800}
TINY_STEPS = 20
TINY_ATTEMPTS = 256


def tiny_section(args, B, synth, torch, dev, stream, flush):
    """The tiny configuration: the 4 x 4 x 3 m room with 20 boxes (2^16 buckets), 320 x 240 queries
    near its trajectory (no depth noise), a forest of 5 trees of depth 10 filled on the GPU from 10
    noisy training renders (reservoirs of 64, <= 10 modes), preemptive RANSAC with 64 hypotheses
    and 500 pixels per round, Philox seed 0; 256 attempts per batch, one graph replay per step."""
    from paper_1801_08361_gb300.presets import TINY
    w1, h1 = TINY.sizes[0]
    world = synth.room_world(1)
    scene = B.Scene(synth.sample_scene(world), TINY.log2_buckets)
    intr = synth.Intrinsics.for_size(w1, h1)
    train = synth.training_poses(world, TINY.train_per_room, seed=11)
    nodes = synth.random_forest_nodes(TINY.trees, TINY.depth, seed=5, depth_tau=100, colour_tau=32)
    forest = B.Forest(nodes, max_modes=TINY.max_modes)
    B.forest_train_begin(forest, B.train_params(capacity=TINY.reservoir, stride=1, seed=7))
    depth = torch.zeros((h1, w1), dtype=torch.int16, device=dev)
    rgba = torch.zeros((h1, w1, 4), dtype=torch.uint8, device=dev)
    for i, P in enumerate(train):
        nz = torch.from_numpy(synth.depth_noise(h1, w1, 100 + i)).to(dev)
        B.raycast_view(scene, intr, P, depth, rgba, noise_dev=nz)
        B.forest_train_frame(forest, intr, P, depth, rgba)
    B.forest_train_finish(forest)
    qs = synth.query_poses(world, train, TINY_ATTEMPTS, seed=31)
    prm = B.ransac_params(n_hyps=TINY.hypotheses[0], batch=TINY.batch_pixels, max_tries=TINY.max_tries)
    items = [dict(scene_b=scene, forest_a=forest, scene_a=scene, intr=intr, pose_b=qs[k], noise=None, seed=0)
             for k in range(TINY_ATTEMPTS)]
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
    bt = B.Batch(att, prm, ws)
    bt.enable_timing(True)
    res = torch.zeros(TINY_ATTEMPTS * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
    bt.capture(res)
    for _ in range(3):
        flush.zero_()
        bt.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(TINY_STEPS)]
    stages = {}
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        bt.replay()
        e[1].record(stream)
        torch.cuda.synchronize()
        for k, v in bt.stage_ms().items():
            if v > 0.01:
                stages[k] = stages.get(k, 0.0) + v / TINY_STEPS
    ms = sum(a.elapsed_time(b) for a, b in ev) / TINY_STEPS
    raw = res.cpu()
    ok = ver = 0
    for k in range(TINY_ATTEMPTS):
        r = B.result_from_bytes(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES])
        ok += int(success(r, qs[k]))
        ver += int(r["verified"])
    return {"workload": "room 4x4x3 m + 20 boxes, 5 mm voxels, 2^16 buckets; 320x240 queries (no noise); forest "
                        "T=5 D=10, reservoir 64, <=10 modes, filled on the GPU from 10 noisy renders; preemptive "
                        "RANSAC K=64, B=500, Philox seed 0",
            "attempts_per_batch": TINY_ATTEMPTS, "steps": TINY_STEPS, "l2": "flushed between steps (512 MiB write)",
            "attempts_per_s": TINY_ATTEMPTS / (ms / 1000.0), "ms_per_batch": ms, "stage_ms_per_batch": stages,
            "success_rate": ok / TINY_ATTEMPTS, "verified_rate": ver / TINY_ATTEMPTS,
            "launches": bt.launch_count}


FRAG_STEPS = 20


def fragments_section(args, B, torch, dev, stream, flush):
    from paper_1801_08361_gb300 import fragments as F
    t0 = time.perf_counter()
    world, frags, scenes, forests, _ = F.build(dev)
    items, meta = F.pairs(world, frags, scenes, forests, dev)
    t_build = time.perf_counter() - t0
    prm = B.ransac_params(n_hyps=1024, batch=F.BATCH_PIXELS, max_tries=F.MAX_TRIES)
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
    bt = B.Batch(att, prm, ws)
    bt.enable_timing(True)
    n = len(items)
    res = torch.zeros(n * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
    bt.capture(res)
    for _ in range(3):
        flush.zero_()
        bt.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(FRAG_STEPS)]
    stages = {}
    for e in ev:
        flush.zero_()
        e[0].record(stream)
        bt.replay()
        e[1].record(stream)
        torch.cuda.synchronize()
        for k, v in bt.stage_ms().items():
            stages[k] = stages.get(k, 0.0) + v / FRAG_STEPS
    ms = [a.elapsed_time(b) for a, b in ev]
    raw = res.cpu()
    # the same batch with its RANSAC in one persistent launch
    bt.set_schedule(persistent=1)
    bt.capture(res)
    bt.replay()
    torch.cuda.synchronize()
    pers_same = bool(torch.equal(res.cpu(), raw))
    pers_ms = timed_replays(bt, torch, flush, stream, FRAG_STEPS)
    pers_launches = bt.launch_count
    bt.set_schedule(persistent=0)
    covered = ok = verified = 0
    for k, m in enumerate(meta):
        r = B.result_from_bytes(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES])
        good = success(r, m["pose_a"])
        covered += m["covered"]
        ok += m["covered"] and good
        verified += r["verified"]
    peak, kind = measured_peaks()
    roofs = {}
    for st, key in (("query_raycast", "query_raycast"), ("forest_eval", "forest_eval"),
                    ("forest_verify", "forest_verify")):
        b = FRAG_ALG_BYTES.get(key)
        t = stages.get(st, 0.0)
        if b and t > 0:
            g = b / (t / 1000.0) / 1e9
            roofs[st] = {"bound": "hbm", "achieved": g, "peak": peak, "unit": "GB/s", "frac": g / peak, "ms": t,
                         "algorithmic_bytes": b, "peak_source": kind}
    sizes = {}
    for it in items:
        key = f"{it['intr'].width}x{it['intr'].height}"
        sizes[key] = sizes.get(key, 0) + 1
    return {"workload": "8 fragments of the house (1-3 rooms, 13-40 m^2, own frames), all 56 ordered pairs per batch; "
                        "query sizes drawn from 320x240/480x360/640x480, K from 256-1024, B=64; forests T=5 D=13 "
                        "reservoir 512",
            "attempts_per_batch": n, "sizes": sizes, "hypotheses": sum(int(it["n_hyps"]) for it in items),
            "attempts_per_s": n * FRAG_STEPS / (sum(ms) / 1000.0), "ms_per_batch": sum(ms) / FRAG_STEPS,
            "l2": "flushed between steps (512 MiB write)", "steps": FRAG_STEPS,
            "stage_ms_per_batch": stages, "roofline_stages": roofs,
            "success_covered": f"{ok}/{covered} (pairs whose query room lies in fragment a; <= 5 cm, <= 5 deg "
                               f"of the known aT_b)", "verified": verified, "build_s": t_build,
            "launches": bt.launch_count,
            "persistent_schedule": {"ms_per_batch": pers_ms, "attempts_per_s": n / (pers_ms / 1000.0),
                                    "launches": pers_launches, "results_equal": pers_same}}


# ------------------------------------------------------------------------------------------------
# The oracle beside the GPU: whole attempts timed on one host core (cpu_baseline), and the error
# of every GPU result against the FP64 oracle on the same attempts (precision)
# ------------------------------------------------------------------------------------------------
ORACLE_ATTEMPTS = 2


def oracle_section(args, B, torch, dev, scene, blocks, intr, train, nodes, st, prm, stream):
    import oracle
    cores = cores_used()
    t_setup = time.perf_counter()
    sc_o, forest_o = oracle_setup(blocks, intr, train, nodes, cores)
    t_setup = time.perf_counter() - t_setup
    specs = [attempt_spec(0, 0, k, st["qs"]) for k in range(ORACLE_ATTEMPTS)]
    runs = [oracle_attempt(sc_o, forest_o, intr, *sp) for sp in specs]       # one thread (BLAS too)
    secs = [r[0] for r in runs]
    cpu = {"value": len(runs) / sum(secs), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"attempts 0..{len(runs) - 1} of the GPU batch's first query set, whole (query raycast, forest, "
                     f"1024-hypothesis preemptive RANSAC, verification raycast; same poses, noise and RANSAC seeds), "
                     f"one thread, with a forest the oracle filled itself (every training pose, every "
                     f"{ORACLE_TRAIN_STRIDE}th pixel and row; setup {t_setup:.0f} s on {cores} threads, untimed); "
                     f"seconds per attempt " + ", ".join(f"{x:.2f}" for x in secs)}

    # the GPU on the oracle's forest: the same attempts, the same modes
    gfo = B.Forest(nodes, forest_o.modes, forest_o.n_modes, max_modes=MAX_MODES)
    A = len(st["qs"])
    items = [dict(scene_b=scene, forest_a=gfo, scene_a=scene, intr=intr, pose_b=st["qs"][k], noise=st["noise"][k],
                  seed=rank_seeds(0, 0, k)[2]) for k in range(A)]
    att = B.make_attempts(items)
    ws = torch.empty(B.batch_workspace_size(att, prm), dtype=torch.uint8, device=dev)
    bt = B.Batch(att, prm, ws)
    res = torch.zeros(A * B.RESULT_BYTES, dtype=torch.uint8, device=dev)
    bt.capture(res)
    bt.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(3):
        e0.record(stream)
        bt.replay()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    raw = res.cpu()
    got = [B.result_from_bytes(raw[k * B.RESULT_BYTES:(k + 1) * B.RESULT_BYTES]) for k in range(A)]
    same_forest = {"attempts_per_s": A / (sorted(times)[1] / 1000.0),
                   "success_rate": sum(int(success(r, st["qs"][k])) for k, r in enumerate(got)) / A,
                   "oracle_success": [bool(ro["verified"]) and oracle_success(ro["pose"], sp[0])
                                      for (_, ro), sp in zip(runs, specs)]}

    def pose_diff(a, b):
        return float(np.abs(a[:3, :3] - b[:3, :3]).max()), float(np.abs(a[:3, 3] - b[:3, 3]).max())

    rc, iso, ver, e2e = [], [], [], []
    for k, (_, ro) in enumerate(runs):
        # query raycast (FP32 march) against the oracle's render of the same pose and noise
        dg = bt.attempt_images(k, W, H)[0].cpu().numpy().view(np.uint16)
        do = ro["depth_b"]
        both = (dg > 0) & (do > 0)
        diff = np.abs(dg[both].astype(np.int64) - do[both])
        rc.append((int(diff.max()) if diff.size else 0, float((diff <= 1).mean()) if diff.size else 1.0,
                   float(((dg > 0) != (do > 0)).mean())))
        # stage-isolated: the GPU's forest, RANSAC and verification on the oracle's query image
        dd = torch.from_numpy(np.ascontiguousarray(do).view(np.int16)).to(dev)
        cc = torch.from_numpy(np.ascontiguousarray(ro["rgba_b"])).to(dev)
        lv = torch.zeros((T_TREES, H, W), dtype=torch.int16, device=dev)
        B.forest_eval(gfo, dd, cc, lv)
        p1 = B.ransac_params(n_hyps=K_HYPS, batch=B_PIX, max_tries=10000, seed=specs[k][2])
        wsr = torch.empty(B.ransac_workspace_size(W, H, p1), dtype=torch.uint8, device=dev)
        r1 = torch.zeros(B.RESULT_BYTES, dtype=torch.uint8, device=dev)
        B.ransac_relocalise(gfo, dd, lv, intr, p1, wsr, r1)
        da = torch.zeros_like(dd)
        B.verify(scene, intr, dd, r1, da)
        torch.cuda.synchronize()
        g = B.result_from_bytes(r1)
        mism = int((lv.cpu().numpy().view(np.uint16) != ro["leaves"]).sum())
        dR, dt = pose_diff(g["pose"], ro["pose"])
        iso.append(dict(leaf_mismatches=mism, same_hypothesis=g["hypothesis"] == ro["index"], R_max_abs=dR,
                        t_max_abs_m=dt, energy_rel=abs(g["energy"] - ro["energy"]) / max(abs(ro["energy"]), 1e-30)))
        cnt = [g["omega"], g["omega_a"], g["omega_b"], g["omega_ab"], g["sum_absdiff_mm"]]
        ver.append(dict(count_max_abs_diff=int(np.abs(np.array(cnt, np.int64) - ro["counts"].astype(np.int64)).max()),
                        accept_equal=bool(g["verified"]) == bool(ro["verified"])))
        # the whole GPU attempt (its own FP32 raycasts) against the whole oracle attempt
        dR, dt = pose_diff(got[k]["pose"], ro["pose"])
        e2e.append(dict(same_hypothesis=got[k]["hypothesis"] == ro["index"], R_max_abs=dR, t_max_abs_m=dt,
                        verified_equal=bool(got[k]["verified"]) == bool(ro["verified"])))
    precision = {
        "sample": f"attempts 0..{len(runs) - 1} of the first query set; the FP64 oracle against the GPU run on the "
                  f"oracle's forest (stage-isolated: the GPU's forest, RANSAC and verification on the oracle's "
                  f"query image; end to end: the whole GPU attempt)",
        "query_raycast": {"max_abs_mm": max(x[0] for x in rc), "frac_within_1mm": min(x[1] for x in rc),
                          "validity_mismatch": max(x[2] for x in rc)},
        "forest_leaf_mismatches": sum(x["leaf_mismatches"] for x in iso),
        "ransac_isolated": {"same_hypothesis": [x["same_hypothesis"] for x in iso],
                            "R_max_abs": max(x["R_max_abs"] for x in iso),
                            "t_max_abs_m": max(x["t_max_abs_m"] for x in iso),
                            "energy_max_rel": max(x["energy_rel"] for x in iso)},
        "verification_isolated": {"count_max_abs_diff": max(x["count_max_abs_diff"] for x in ver),
                                  "accept_equal": [x["accept_equal"] for x in ver]},
        "attempt_end_to_end": {"same_hypothesis": [x["same_hypothesis"] for x in e2e],
                               "R_max_abs": max(x["R_max_abs"] for x in e2e),
                               "t_max_abs_m": max(x["t_max_abs_m"] for x in e2e),
                               "verified_equal": [x["verified_equal"] for x in e2e]},
        "gpu_on_oracle_forest": same_forest}
    return cpu, precision


def success(r, P):
    """The success criterion of Sec. 4.2.2: within 5 cm and 5 degrees of the ground-truth pose."""
    dt = float(np.linalg.norm(r["pose"][:3, 3] - P[:3, 3]))
    cang = (np.trace(r["pose"][:3, :3] @ P[:3, :3].T) - 1) / 2
    dr = math.degrees(math.acos(max(-1.0, min(1.0, cang))))
    return r["status"] == 0 and dt <= 0.05 and dr <= 5.0


# ------------------------------------------------------------------------------------------------
# TSDF fusion (Sec. 3.3 (a): each agent's map; Appendix B.3): noisy renders along the house
# trajectory fused into an empty scene, one frame per relo_fuse_frame (four launches)
# ------------------------------------------------------------------------------------------------
FUSION_CAPACITY = 1 << 20          # blocks (5.2 GB of tsdf, colour and weights)
FUSION_BYTES_PER_VOXEL = 2 * (4 + 4 + 2)   # tsdf, colour, weight: read and written


def fusion_section(args, B, synth, torch, dev, scene, world, intr, train, nvtx=None, capacity=FUSION_CAPACITY):
    n = args.fusion_frames
    poses = synth.query_poses(world, train, n, seed=4242)
    depth = torch.zeros((n, H, W), dtype=torch.int16, device=dev)
    rgba = torch.zeros((n, H, W, 4), dtype=torch.uint8, device=dev)
    noise = torch.from_numpy(np.stack([synth.depth_noise(H, W, 5000 + k) for k in range(n)])).to(dev)
    ws = torch.empty(B.raycast_views_workspace_size(n), dtype=torch.uint8, device=dev)
    B.raycast_views(scene, intr, poses, depth, rgba, noise_dev=noise, workspace_dev=ws)
    if nvtx:
        torch.cuda.synchronize()
        scene.__del__()                           # profiler runs keep little on the device
    fs = B.FusionScene(capacity, synth.VOXEL_SIZE, synth.TRUNCATION, log2_buckets=20)
    wsf = torch.empty(B.fuse_workspace_size(W, H), dtype=torch.uint8, device=dev)
    # two timed regions, frames back to back on the stream: the first quarter (most blocks are
    # created there) and the rest (mostly updates of existing blocks)
    q = max(1, n // 4)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    updates = [0]
    if nvtx:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(nvtx)
    for lo, hi, a in ((0, q, 0), (q, n, 2)):
        ev[a].record()
        fs.fuse_many(intr, poses[lo:hi], depth[lo:hi], rgba[lo:hi], workspace_dev=wsf)
        ev[a + 1].record()
        updates.append(fs.block_updates())        # synchronises after the region's end event
    if nvtx:
        torch.cuda.nvtx.range_pop()
    ms_first, ms_rest = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    peak, kind = measured_peaks()
    upd_rest = updates[2] - updates[1]
    steady_bytes = upd_rest * 512 * FUSION_BYTES_PER_VOXEL + (n - q) * H * W * 6
    g = steady_bytes / (ms_rest / 1000.0) / 1e9
    return {"frames": n, "size": f"{W}x{H}", "ms_per_frame": (ms_first + ms_rest) / n,
            "frames_per_s": 1000.0 * n / (ms_first + ms_rest), "steady_ms_per_frame": ms_rest / (n - q),
            "blocks": fs.block_count(), "block_updates_per_frame": updates[2] / n,
            "roofline": {"bound": "hbm", "achieved": g, "peak": peak, "unit": "GB/s", "frac": g / peak,
                         "peak_source": kind, "region": f"frames {q}..{n - 1}",
                         "bytes": "updated blocks x 512 voxels x 20 B (tsdf, colour, weight read and written) "
                                  "+ 6 B per pixel (depth, colour)"}}


# ------------------------------------------------------------------------------------------------
# Serving: agents (threads) submit single attempts at Poisson times to relo_server; the worker
# batches them under the workspace budget; latency = completion - submission
# ------------------------------------------------------------------------------------------------
# (agents, offered requests/s over all agents)
SERVE_POINTS = list(zip(SERVING.extra["agents"], SERVING.extra["offered_per_s"]))
SERVE_MAX_BATCH, SERVE_MAX_WAIT_US, SERVE_SLOTS = (SERVING.extra[k] for k in ("max_batch", "max_wait_us", "slots"))


def serving_section(args, B, torch, dev, st, prm):
    import queue
    import threading
    atts = st["att"]
    A = len(atts)
    ws_bytes = B.batch_workspace_size(B.make_attempts_view(atts, SERVE_MAX_BATCH), prm) + (1 << 20)
    points = []
    for agents, rate in SERVE_POINTS:
        srv = B.Server(prm, workspace_bytes=ws_bytes, max_batch=SERVE_MAX_BATCH, max_wait_us=SERVE_MAX_WAIT_US,
                       slots=SERVE_SLOTS)
        tickets = queue.Queue()
        stop_at = time.perf_counter() + args.serve_seconds
        sent = [0] * agents

        def agent(a):
            rng = np.random.default_rng(1000 + a)
            t = time.perf_counter()
            k = a
            while True:
                t += rng.exponential(agents / rate)
                if t >= stop_at:
                    break
                time.sleep(max(0.0, t - time.perf_counter()))
                try:
                    tickets.put(srv.submit(atts[k % A]))
                    sent[a] += 1
                except B.ReloError as e:
                    if e.status != B.EBUSY:
                        raise
                k += agents
            tickets.put(None)

        def waiter():
            while True:
                tk = tickets.get()
                if tk is None:
                    tickets.put(None)
                    return
                srv.wait(tk)

        t0 = time.perf_counter()
        th = [threading.Thread(target=agent, args=(a,)) for a in range(agents)]
        wt = [threading.Thread(target=waiter) for _ in range(8)]
        for x in th + wt:
            x.start()
        for x in th + wt:
            x.join()
        wall = time.perf_counter() - t0
        stt = srv.stats()
        srv.close()
        points.append({"agents": agents, "offered_per_s": rate, "attempts_per_s": stt["completed"] / wall,
                       "completed": stt["completed"], "discarded": stt["discarded"], "batches": stt["batches"],
                       "mean_batch": stt["mean_batch"], "p50_ms": stt["p50_ms"], "p99_ms": stt["p99_ms"],
                       "max_ms": stt["max_ms"]})
    return {"max_batch": SERVE_MAX_BATCH, "max_wait_us": SERVE_MAX_WAIT_US, "slots": SERVE_SLOTS,
            "workspace_bytes": ws_bytes, "seconds_per_point": args.serve_seconds, "points": points}


# Hypothesis search, ALU view: each try is one Philox4x32-10 block (10 rounds of two 32 x 32 -> 64
# bit products = 40 integer multiply instructions) plus the rigidity and area tests; the peak is
# the integer multiply-add issue rate, 64 per clock per SM (half the 128 FP32 lanes), x the
# device's SMs x the SM clock, i.e. one Philox block per 40 IMAD slots.
IMAD_PER_TRY = 40
IMAD_PER_CLK_SM = 64


def profiled_traffic(kernel, attempts):
    per = PROFILED_TRAFFIC_BYTES_PER_ATTEMPT.get(kernel)
    return None if per is None else per * attempts


def roofline(kernel, avg_ms, attempts, tries_per_launch, clocks, n_sms):
    if kernel in ("forest_hypotheses", "learned_hypotheses"):
        mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = IMAD_PER_CLK_SM * n_sms * mhz * 1e6 / IMAD_PER_TRY / 1e9      # G tries / s
        achieved = tries_per_launch / (avg_ms / 1000.0) / 1e9
        return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gtries/s",
                "frac": achieved / peak, "traffic": profiled_traffic(kernel, attempts), "ms": avg_ms,
                "peak_source": f"derived: 64 IMAD/clk/SM x {n_sms} SMs x max SM clock / 40 IMAD per try",
                "limiter": PROFILED_LIMITER.get(kernel)}
    peak, peak_kind = measured_peaks()
    per_px = ALG_BYTES_PER_PIXEL.get(kernel)
    achieved = None if per_px is None else per_px * W * H * attempts / (avg_ms / 1000.0) / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": None if achieved is None else achieved / peak, "traffic": profiled_traffic(kernel, attempts),
            "ms": avg_ms, "peak_source": peak_kind, "limiter": PROFILED_LIMITER.get(kernel)}


def ctypes_attempt_bytes():
    from paper_1801_08361_gb300 import binding as B
    import ctypes
    return ctypes.sizeof(B.Attempt)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
