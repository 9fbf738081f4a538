"""Seeded synthetic inputs for the relocalisation path (input generation only).

The paper's workloads are live reconstructions from its own dataset (Sec. 5,
"Dataset"), which is not available; these generators stand in for them with
the shapes and sizes the paper reports: voxel sub-scenes of a few rooms
(Sec. 4.3.2 sizes them at about 1 GB each), RGB-D views rendered from poses on
an agent's trajectory (Sec. 3.3.1), depth noise that grows quadratically with
depth (Appendix, "Depth Sensor Noise Characteristics"), and regression forests
with random pixel-pair splits (the relocaliser of Sec. 3.3, trained as in
Cavallari et al.).

This module holds none of the method's arithmetic: it draws random numbers,
lays out boxes, samples an analytic signed distance function into voxel blocks
(scene_sampler.c) and writes camera poses.  The CUDA library and the CPU oracle
both consume what it returns; neither imports the other.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

VOXEL_SIZE = 0.005        # 5 mm voxels
TRUNCATION = 0.02         # mu = 4 voxels
BLOCK = 8


def _lib():
    global _LIB
    if _LIB is None:
        path = os.path.join(_HERE, "_scene_sampler.so")
        if not os.path.exists(path):
            build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.synth_flag_blocks.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, ip, ip,
                                          ctypes.c_void_p]
        lib.synth_fill_blocks.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp,
                                          ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_world_sdf.argtypes = [dp, ctypes.c_int, dp, ctypes.c_long, dp]
        _LIB = lib
    return _LIB


def build(force: bool = False) -> str:
    """Compile scene_sampler.c into _scene_sampler.so next to it (gcc, OpenMP)."""
    import subprocess
    src = os.path.join(_HERE, "scene_sampler.c")
    out = os.path.join(_HERE, "_scene_sampler.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c99", src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------------------------
# World layouts
# --------------------------------------------------------------------------------------------

@dataclass
class World:
    """Boxes of an analytic world: row i = [kind, lo xyz, hi xyz, rgb, texture freqs]."""
    comps: np.ndarray                 # float64 [n, 13]
    free_lo: np.ndarray               # camera-placement region (world)
    free_hi: np.ndarray
    room_centres: list = field(default_factory=list)
    rooms: list = field(default_factory=list)  # (i, j, x0, y0, x1, y1) per room of a house grid

    def sdf(self, pts: np.ndarray) -> np.ndarray:
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.empty(len(pts), dtype=np.float64)
        _lib().synth_world_sdf(_dp(self.comps), len(self.comps), _dp(pts), len(pts), _dp(out))
        return out


def _comp(kind, lo, hi, rng):
    rgb = rng.uniform(0.25, 1.0, 3)
    freq = rng.uniform(0.8, 4.0, 3)
    return [float(kind), *lo, *hi, *rgb, *freq]


def room_world(seed: int = 1, size=(4.0, 4.0, 3.0), n_boxes: int = 20) -> World:
    """A closed axis-aligned room with furniture boxes resting on the floor.

    Boxes have sides U[0.2, 1.0] m and stand in a band next to the walls so the
    room's middle stays free for cameras.
    """
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    comps = [_comp(0, (0.0, 0.0, 0.0), (sx, sy, sz), rng)]
    comps += _furniture(rng, [(0.0, 0.0, sx, sy)], n_boxes, doors=[])
    return World(np.asarray(comps, dtype=np.float64), np.array([1.3, 1.3, 1.0]), np.array([sx - 1.3, sy - 1.3, 2.0]),
                 [np.array([sx / 2, sy / 2])])


def _furniture(rng, rooms, n, doors):
    out = []
    tries = 0
    while len(out) < n and tries < 100000:
        tries += 1
        x0, y0, x1, y1 = rooms[rng.integers(len(rooms))]
        w, d = rng.uniform(0.2, 1.0, 2)
        h = rng.uniform(0.2, 1.6)
        # centre in a band 0.15..1.1 m from one of the room's walls
        side = rng.integers(4)
        off = rng.uniform(0.15, 1.1)
        if side == 0:
            cx, cy = rng.uniform(x0 + 0.3, x1 - 0.3), y0 + off
        elif side == 1:
            cx, cy = rng.uniform(x0 + 0.3, x1 - 0.3), y1 - off
        elif side == 2:
            cx, cy = x0 + off, rng.uniform(y0 + 0.3, y1 - 0.3)
        else:
            cx, cy = x1 - off, rng.uniform(y0 + 0.3, y1 - 0.3)
        if any(math.hypot(cx - dx, cy - dy) < 1.0 for dx, dy in doors):
            continue
        lo = (max(cx - w / 2, x0 + 0.02), max(cy - d / 2, y0 + 0.02), 0.0)
        hi = (min(cx + w / 2, x1 - 0.02), min(cy + d / 2, y1 - 0.02), h)
        out.append(_comp(1, lo, hi, rng))
    return out


def house_world(seed: int = 2, size=(10.0, 8.0, 3.0), grid=(3, 2), n_boxes: int = 200, wall=0.1,
                door_w=1.0, door_h=2.0) -> World:
    """A house of grid[0] x grid[1] rooms: 0.1 m interior walls with 1 x 2 m doorways and furniture."""
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    nx, ny = grid
    comps = [_comp(0, (0.0, 0.0, 0.0), (sx, sy, sz), rng)]
    xs = [sx * i / nx for i in range(nx + 1)]
    ys = [sy * j / ny for j in range(ny + 1)]
    doors = []
    hw = wall / 2
    # walls at x = xs[i] (interior), one doorway per room row
    for i in range(1, nx):
        for j in range(ny):
            y0, y1 = ys[j], ys[j + 1]
            dc = rng.uniform(y0 + 0.8, y1 - 0.8)
            doors.append((xs[i], dc))
            comps.append(_comp(1, (xs[i] - hw, y0, 0.0), (xs[i] + hw, dc - door_w / 2, sz), rng))
            comps.append(_comp(1, (xs[i] - hw, dc + door_w / 2, 0.0), (xs[i] + hw, y1, sz), rng))
            comps.append(_comp(1, (xs[i] - hw, dc - door_w / 2, door_h), (xs[i] + hw, dc + door_w / 2, sz), rng))
    for j in range(1, ny):
        for i in range(nx):
            x0, x1 = xs[i], xs[i + 1]
            dc = rng.uniform(x0 + 0.8, x1 - 0.8)
            doors.append((dc, ys[j]))
            comps.append(_comp(1, (x0, ys[j] - hw, 0.0), (dc - door_w / 2, ys[j] + hw, sz), rng))
            comps.append(_comp(1, (dc + door_w / 2, ys[j] - hw, 0.0), (x1, ys[j] + hw, sz), rng))
            comps.append(_comp(1, (dc - door_w / 2, ys[j] - hw, door_h), (dc + door_w / 2, ys[j] + hw, sz), rng))
    rooms = [(xs[i] + hw, ys[j] + hw, xs[i + 1] - hw, ys[j + 1] - hw) for i in range(nx) for j in range(ny)]
    comps += _furniture(rng, rooms, n_boxes, doors)
    centres = [np.array([(r[0] + r[2]) / 2, (r[1] + r[3]) / 2]) for r in rooms]
    cells = [(i, j, xs[i], ys[j], xs[i + 1], ys[j + 1]) for i in range(nx) for j in range(ny)]
    return World(np.asarray(comps, dtype=np.float64), np.array([0.0, 0.0, 1.0]), np.array([sx, sy, 2.0]), centres,
                 cells)


def house_fragments(world: World, n: int, seed: int, max_rooms: int = 3, max_t: float = 2.0) -> list:
    """n sub-scenes cut from a house, each a rectangle of 1 to max_rooms adjacent rooms (13-40 m^2
    of floor for the 10 x 8 m, 3 x 2-room house) in its own random rigid frame, so that the
    relative transform between any two is known.  Each is a dict: crop (world box, walls
    included), scene_to_world, rooms (indices into world.rooms / world.room_centres)."""
    rng = np.random.default_rng(seed)
    nx = max(r[0] for r in world.rooms) + 1
    ny = max(r[1] for r in world.rooms) + 1
    shapes = [(w, h) for w in range(1, nx + 1) for h in range(1, ny + 1) if w * h <= max_rooms]
    out = []
    for _ in range(n):
        w, h = shapes[rng.integers(len(shapes))]
        i0, j0 = int(rng.integers(nx - w + 1)), int(rng.integers(ny - h + 1))
        idx = [k for k, r in enumerate(world.rooms) if i0 <= r[0] < i0 + w and j0 <= r[1] < j0 + h]
        lo = np.array([min(world.rooms[k][2] for k in idx), min(world.rooms[k][3] for k in idx)])
        hi = np.array([max(world.rooms[k][4] for k in idx), max(world.rooms[k][5] for k in idx)])
        top = world.comps[0][6]
        crop = np.array([lo[0] - 0.15, lo[1] - 0.15, -0.1, hi[0] + 0.15, hi[1] + 0.15, top + 0.1])
        out.append(dict(crop=crop, scene_to_world=random_rigid(rng, max_t=max_t), rooms=idx))
    return out


# --------------------------------------------------------------------------------------------
# Voxel sub-scenes
# --------------------------------------------------------------------------------------------

@dataclass
class SceneBlocks:
    """Voxel blocks of one sub-scene: the input to scene creation on both sides."""
    coords: np.ndarray      # int32 [n, 3] block coordinates, sorted by (bz, by, bx)
    tsdf: np.ndarray        # float32 [n, 512]
    rgba: np.ndarray        # uint8 [n, 512, 4]
    voxel_size: float
    mu: float
    scene_to_world: np.ndarray  # float64 4x4: maps scene-frame points to the world

    @property
    def n_blocks(self) -> int:
        return int(self.coords.shape[0])


def sample_scene(world: World, voxel_size: float = VOXEL_SIZE, mu: float = TRUNCATION,
                 scene_to_world: np.ndarray | None = None, crop: np.ndarray | None = None) -> SceneBlocks:
    """Sample the world's SDF into a voxel-block sub-scene expressed in its own frame."""
    if scene_to_world is None:
        scene_to_world = np.eye(4)
    scene_to_world = np.ascontiguousarray(scene_to_world, dtype=np.float64)
    shell = world.comps[0]
    if crop is None:
        crop = np.concatenate([shell[1:4] - 0.1, shell[4:7] + 0.1])
    crop = np.ascontiguousarray(crop, dtype=np.float64)
    # scene-frame block box covering the crop region
    w2s = np.linalg.inv(scene_to_world)
    corners = np.array([[crop[3 * ((c >> a) & 1) + a] for a in range(3)] for c in range(8)])
    cs = corners @ w2s[:3, :3].T + w2s[:3, 3]
    bsz = BLOCK * voxel_size
    blo = np.floor(cs.min(0) / bsz).astype(np.int32) - 1
    bhi = np.floor(cs.max(0) / bsz).astype(np.int32) + 1
    n = (bhi - blo + 1)
    flags = np.zeros(int(n[0]) * int(n[1]) * int(n[2]), dtype=np.uint8)
    blo_c = np.ascontiguousarray(blo, dtype=np.int32)
    bhi_c = np.ascontiguousarray(bhi, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    rc = _lib().synth_flag_blocks(_dp(world.comps), len(world.comps), voxel_size, mu, _dp(scene_to_world),
                                  _dp(crop), blo_c.ctypes.data_as(ip), bhi_c.ctypes.data_as(ip),
                                  flags.ctypes.data)
    if rc != 0:
        raise MemoryError("scene sampler failed")
    idx = np.nonzero(flags)[0]
    x = idx % n[0]
    y = (idx // n[0]) % n[1]
    z = idx // (n[0] * n[1])
    coords = np.stack([x + blo[0], y + blo[1], z + blo[2]], axis=1).astype(np.int32)
    coords = np.ascontiguousarray(coords)
    tsdf = np.empty((len(coords), 512), dtype=np.float32)
    rgba = np.empty((len(coords), 512, 4), dtype=np.uint8)
    rc = _lib().synth_fill_blocks(_dp(world.comps), len(world.comps), voxel_size, mu, _dp(scene_to_world),
                                  _dp(crop), coords.ctypes.data, len(coords), tsdf.ctypes.data, rgba.ctypes.data)
    if rc != 0:
        raise MemoryError("scene sampler failed")
    return SceneBlocks(coords, tsdf, rgba, voxel_size, mu, scene_to_world)


# --------------------------------------------------------------------------------------------
# Cameras
# --------------------------------------------------------------------------------------------

@dataclass
class Intrinsics:
    """Pinhole camera: fx = fy = 525 * W / 640, principal point at the image centre."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    depth_min: float = 0.1
    depth_max: float = 8.0

    @staticmethod
    def for_size(width: int, height: int, depth_max: float = 8.0) -> "Intrinsics":
        f = 525.0 * width / 640.0
        return Intrinsics(width, height, f, f, (width - 1) / 2.0, (height - 1) / 2.0, 0.1, depth_max)


def look_pose(centre, yaw, pitch) -> np.ndarray:
    """Camera-to-world pose (x right, y down, z forward) at centre looking along yaw/pitch, z up."""
    f = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = r, d, f, centre
    return T


def _free_point(world: World, rng, centre_xy, spread, zr=(1.0, 2.0), clearance=0.3):
    for _ in range(1000):
        p = np.array([centre_xy[0] + rng.uniform(-spread, spread), centre_xy[1] + rng.uniform(-spread, spread),
                      rng.uniform(*zr)])
        if world.sdf(p[None])[0] > clearance:
            return p
    raise RuntimeError("no free camera position")


def training_poses(world: World, n_per_room: int, seed: int, rooms=None) -> list:
    """An agent's trajectory: n_per_room views per room (all rooms, or the given room indices)
    from near its centre, yaw sweeping a full turn."""
    rng = np.random.default_rng(seed)
    out = []
    for c in (world.room_centres if rooms is None else [world.room_centres[k] for k in rooms]):
        for k in range(n_per_room):
            p = _free_point(world, rng, c, 0.35)
            yaw = 2 * math.pi * k / n_per_room + rng.uniform(-0.05, 0.05)
            pitch = rng.uniform(math.radians(-15), math.radians(5))
            out.append(look_pose(p, yaw, pitch))
    return out


def query_poses(world: World, train: list, n: int, seed: int, dpos=0.15, dyaw_deg=10.0, dpitch_deg=5.0) -> list:
    """Query frames near the trajectory: a random training pose perturbed by up to dpos m / dyaw, dpitch degrees."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        T = train[rng.integers(len(train))]
        f = T[:3, 2]
        yaw = math.atan2(f[1], f[0]) + math.radians(rng.uniform(-dyaw_deg, dyaw_deg))
        pitch = math.asin(max(-1.0, min(1.0, f[2]))) + math.radians(rng.uniform(-dpitch_deg, dpitch_deg))
        p = T[:3, 3] + rng.uniform(-dpos, dpos, 3)
        if world.sdf(p[None])[0] < 0.2:
            continue
        out.append(look_pose(p, yaw, pitch))
    return out


def world_to_scene_pose(cam_to_world: np.ndarray, scene_to_world: np.ndarray) -> np.ndarray:
    """Express a camera-to-world pose in a sub-scene's own frame."""
    return np.linalg.inv(scene_to_world) @ cam_to_world


def fragment_trajectories(world: World, frags: list, n_per_room: int = 12) -> None:
    """Each fragment's agent trajectory (camera-to-world poses, n_per_room views in each of its
    rooms, seed 40 + k), stored as frags[k]["train_w"]."""
    for k, f in enumerate(frags):
        f["train_w"] = training_poses(world, n_per_room, seed=40 + k, rooms=f["rooms"])


def fragment_pairs(world: World, frags: list, sizes: list, seed: int = 17) -> list:
    """All ordered pairs (a, b), a != b, of fragments with trajectories: the query of (a, b) is a
    perturbed view of b's trajectory at a size drawn from ``sizes``, with its depth-noise seed, a
    hypothesis count from 256-1024 and a RANSAC seed.  Each pair: a, b, width, height, noise_seed,
    n_hyps, seed, pose_b (in b's frame), pose_a (the same camera in a's frame), covered (the
    query's room lies in fragment a)."""
    rng = np.random.default_rng(seed)
    out = []
    for a in range(len(frags)):
        for b in range(len(frags)):
            if a == b:
                continue
            W, H = sizes[rng.integers(len(sizes))]
            Pw = query_poses(world, frags[b]["train_w"], 1, seed=int(rng.integers(1 << 30)))[0]
            Sa, Sb = frags[a]["scene_to_world"], frags[b]["scene_to_world"]
            noise_seed = int(rng.integers(1 << 30))
            n_hyps = int(rng.integers(256, 1025))
            rseed = int(rng.integers(1 << 40))
            room = int(np.argmin([np.linalg.norm(Pw[:2, 3] - c) for c in world.room_centres]))
            out.append(dict(a=a, b=b, width=int(W), height=int(H), noise_seed=noise_seed, n_hyps=n_hyps, seed=rseed,
                            pose_b=world_to_scene_pose(Pw, Sb), pose_a=world_to_scene_pose(Pw, Sa),
                            covered=room in frags[a]["rooms"]))
    return out


def random_rigid(rng, max_angle=math.pi, max_t=2.0) -> np.ndarray:
    """A random rigid transform: yaw about z up to max_angle and a translation up to max_t per axis."""
    a = rng.uniform(-max_angle, max_angle)
    T = np.eye(4)
    T[:2, :2] = [[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]]
    T[:3, 3] = rng.uniform(-max_t, max_t, 3) * np.array([1.0, 1.0, 0.2])
    return T


def depth_noise(height: int, width: int, seed: int) -> np.ndarray:
    """Standard normal draws per pixel (float32); scaled by 1.5 mm * z^2 where used."""
    return np.random.default_rng(seed).standard_normal((height, width)).astype(np.float32)


# --------------------------------------------------------------------------------------------
# Forest structure (random pixel-pair splits; leaves are filled by the relocaliser's trainer)
# --------------------------------------------------------------------------------------------

NODE_DTYPE = np.dtype([("dx1", "<i2"), ("dy1", "<i2"), ("dx2", "<i2"), ("dy2", "<i2"),
                       ("kind", "u1"), ("c1", "u1"), ("c2", "u1"), ("pad", "u1"), ("tau", "<i4")])
assert NODE_DTYPE.itemsize == 16


def random_forest_nodes(n_trees: int, depth: int, seed: int, offset: int = 130,
                        depth_tau: int = 300, colour_tau: int = 64) -> np.ndarray:
    """Split nodes [n_trees, 2^depth - 1], breadth first (children of n are 2n+1, 2n+2).

    Each node compares two probe pixels offset by (dx, dy) pixel-metres from the
    query pixel: either their depths (kind 0, threshold in mm) or one colour
    channel each (kind 1).  Offsets are uniform integers in [-offset, offset],
    thresholds uniform integers in [-depth_tau, depth_tau] or [-colour_tau, colour_tau].
    """
    rng = np.random.default_rng(seed)
    n_int = (1 << depth) - 1
    nodes = np.zeros((n_trees, n_int), dtype=NODE_DTYPE)
    kind = rng.integers(0, 2, (n_trees, n_int))
    nodes["kind"] = kind
    for k in ("dx1", "dy1", "dx2", "dy2"):
        nodes[k] = rng.integers(-offset, offset + 1, (n_trees, n_int))
    nodes["c1"] = rng.integers(0, 3, (n_trees, n_int))
    nodes["c2"] = rng.integers(0, 3, (n_trees, n_int))
    tau_d = rng.integers(-depth_tau, depth_tau + 1, (n_trees, n_int))
    tau_c = rng.integers(-colour_tau, colour_tau + 1, (n_trees, n_int))
    nodes["tau"] = np.where(kind == 0, tau_d, tau_c)
    return nodes
