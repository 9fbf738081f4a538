"""CPU oracle for the inter-agent relocalisation path (TEST INFRASTRUCTURE ONLY).

Golodetz et al., "Collaborative Large-Scale Dense 3D Reconstruction with Online
Inter-Agent Pose Optimisation", Sec. 3.3.1 and Fig. 3: render a synthetic RGB-D
view of agent b's voxel sub-scene from a frame's pose, relocalise it with agent
a's regression-forest relocaliser (Cavallari et al.), verify the proposed pose
by a depth raycast of a's sub-scene, and form the relative transform sample.

Plain and slow on purpose: FP64 throughout, every step the written-out
definition of what it computes (heavy pixel loops in relo_oracle.c, the
preemptive RANSAC below in numpy).  Only ``tests/``, the smoke check and the
CPU-baseline leg of the benchmark may import this package; it shares no code
with the CUDA library, and the two exchange nothing but seeded inputs from
``paper_1801_08361_gb300.synth``.

Parity is pinned (tests/test_oracle_*.py) for: Philox (published known-answer
vectors), block lookup (a dict), raycast (analytic plane / sphere / box-world
depths, invariance under a shift by whole blocks into negative coordinates),
forest descent (hand-computed trees), verification counts (hand counts), camera
points (pinhole projection back to the pixel), Kabsch (known transforms, Horn's
quaternion method), the energy (scipy's Gaussian density near the modes, the
closed-form single Gaussian), hypotheses (the first all-inlier triple on
constructed data), RANSAC (exact recovery on noise-free data, exhaustive
ranking, ceil(K/2) halving), reservoirs (Algorithm R's inclusion probabilities),
mean shift (Gaussian blobs, the two-cluster merge bound), TSDF fusion (closed-form
plane with its clamp, averages, colour rounding, weight cap), global rendering (a
brute-force depth test) and the count of data a raycast reads (exact colour voxels
on a wall).  The pose graph of Sec. 3.3.2 (``oracle/posegraph.py``) is pinned by
closed-form blends, clustering thresholds, exact recovery and stationarity; the
regressor (``oracle/regressor.py``) by scipy's correlation, central differences and
closed forms.  tests/test_oracle_mutations.py plants plausible mistakes in copies of
this oracle and checks that a pin fails for each.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

TAG_HYP, TAG_PIX, TAG_RES = 1, 2, 3
LOG_EPS = -math.log(1e-30)   # energy of a pixel with no supporting mode


def build(force: bool = False) -> str:
    """Compile relo_oracle.c (plain C99, no FMA contraction) into _relo_oracle.so."""
    src = os.path.join(_HERE, "relo_oracle.c")
    out = os.path.join(_HERE, "_relo_oracle.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", tmp,
                               "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = declare(ctypes.CDLL(build()))
    return _LIB


def declare(lib):
    """Argument and result types of the C oracle's functions on a loaded copy of it."""
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
    lib.orc_philox_many.argtypes = [vp, ctypes.c_long, vp, vp]
    lib.orc_scene_create.restype = vp
    lib.orc_scene_create.argtypes = [vp, vp, vp, ctypes.c_long, ctypes.c_double, ctypes.c_double]
    lib.orc_scene_destroy.argtypes = [vp]
    lib.orc_scene_find_many.argtypes = [vp, vp, ctypes.c_long, vp]
    lib.orc_raycast.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp, vp, vp,
                                ctypes.c_long, vp, vp]
    lib.orc_raycast_touched.restype = ctypes.c_int
    lib.orc_raycast_touched.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp,
                                        ctypes.c_int, vp]
    lib.orc_forest_eval.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    lib.orc_verify_counts.argtypes = [vp, vp, ctypes.c_long, vp]
    lib.orc_reservoirs_create.restype = vp
    lib.orc_reservoirs_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
                                          ctypes.c_uint32]
    lib.orc_reservoirs_destroy.argtypes = [vp]
    lib.orc_reservoirs_add_frame.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
    lib.orc_reservoirs_get.argtypes = [vp, vp, vp]
    lib.orc_mean_shift_leaf.restype = ctypes.c_int
    lib.orc_mean_shift_leaf.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    lib.orc_fill_modes.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, vp, vp]
    lib.orc_fill_modes_range.argtypes = [vp, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp, vp]
    lib.orc_fusion_create.restype = vp
    lib.orc_fusion_create.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.orc_fusion_destroy.argtypes = [vp]
    lib.orc_fusion_frame.restype = ctypes.c_int
    lib.orc_fusion_frame.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp,
                                     vp, vp]
    lib.orc_fusion_count.restype = ctypes.c_long
    lib.orc_fusion_count.argtypes = [vp]
    lib.orc_fusion_export.argtypes = [vp, vp, vp, vp, vp]
    return lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


# ------------------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC 2011)
# ------------------------------------------------------------------------------------------------

def philox(counters, key) -> np.ndarray:
    """Philox4x32-10 of each 4-word counter under a 2-word key -> uint32 [n, 4]."""
    ctr, pc = _c(np.asarray(counters, dtype=np.uint32).reshape(-1, 4), np.uint32)
    k, pk = _c(np.asarray(key, dtype=np.uint32).reshape(2), np.uint32)
    out = np.empty_like(ctr)
    _lib().orc_philox_many(pc, len(ctr), pk, out.ctypes.data)
    return out


def seed_key(seed: int) -> np.ndarray:
    """Reading: the 64-bit seed is the Philox key, low word first."""
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def uniform_below(x, n) -> np.ndarray:
    """Reading: a uniform integer in [0, n) from a 32-bit word x is floor(x * n / 2^32)."""
    return ((np.asarray(x, dtype=np.uint64) * np.asarray(n, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


# ------------------------------------------------------------------------------------------------
# Scene, raycast, forest, verification (C)
# ------------------------------------------------------------------------------------------------

class Scene:
    """A voxel sub-scene (Sec. 3.3: the InfiniTAM map), looked up by binary search."""

    def __init__(self, blocks):
        self.coords = np.ascontiguousarray(blocks.coords, dtype=np.int32)
        self.tsdf = np.ascontiguousarray(blocks.tsdf, dtype=np.float32)
        self.rgba = np.ascontiguousarray(blocks.rgba, dtype=np.uint8)
        self.voxel_size = float(blocks.voxel_size)
        self.mu = float(blocks.mu)
        self._h = _lib().orc_scene_create(self.coords.ctypes.data, self.tsdf.ctypes.data, self.rgba.ctypes.data,
                                          len(self.coords), self.voxel_size, self.mu)
        if not self._h:
            raise MemoryError("oracle scene")

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().orc_scene_destroy(self._h)
            self._h = None

    def find_blocks(self, keys) -> np.ndarray:
        """Input index of each block key (n x 3), -1 where unallocated."""
        k, pk = _c(np.asarray(keys, dtype=np.int32).reshape(-1, 3), np.int32)
        out = np.empty(len(k), dtype=np.int64)
        _lib().orc_scene_find_many(self._h, pk, len(k), out.ctypes.data)
        return out

    def raycast(self, intr, pose, noise=None, pixels=None):
        """Depth (uint16 mm, 0 = invalid) and RGBA (uint8) of a view at camera-to-scene pose.

        With ``pixels`` (indices v*W+u) only those pixels are cast and the outputs are 1-D.
        """
        W, H = intr.width, intr.height
        K = np.array([intr.fx, intr.fy, intr.cx, intr.cy], dtype=np.float64)
        P = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        nz = None
        if noise is not None:
            nz = np.ascontiguousarray(noise, dtype=np.float32).reshape(-1)
        if pixels is None:
            depth = np.zeros((H, W), dtype=np.uint16)
            rgba = np.zeros((H, W, 4), dtype=np.uint8)
            pp, n = None, 0
        else:
            px = np.ascontiguousarray(pixels, dtype=np.int64).reshape(-1)
            depth = np.zeros(len(px), dtype=np.uint16)
            rgba = np.zeros((len(px), 4), dtype=np.uint8)
            pp, n = px.ctypes.data, len(px)
        _lib().orc_raycast(self._h, W, H, _d(K), intr.depth_min, intr.depth_max, _d(P),
                           nz.ctypes.data if nz is not None else None, pp, n, depth.ctypes.data, rgba.ctypes.data)
        return depth, rgba


def render_global(scenes, global_poses, intr, pose_global, pixels=None):
    """Global map rendering (Appendix B.2): each sub-scene a is raycast from its local pose
    (gT_a)^-1 P_g (P_g camera -> global, gT_a scene a -> global); per pixel the scene with the
    smallest depth wins (whole mm as the depth images hold it; ties: the lower index; no hit:
    +inf) and gives the pixel its depth and colour.  Returns (depth, rgba, owner, depths) where
    owner is -1 where no scene is hit and depths [n, ...] holds every scene's own depth image."""
    P_g = np.asarray(pose_global, dtype=np.float64)
    imgs = [sc.raycast(intr, np.linalg.inv(np.asarray(g, dtype=np.float64)) @ P_g, pixels=pixels)
            for sc, g in zip(scenes, global_poses)]
    depths = np.stack([d for d, _ in imgs])
    key = np.where(depths > 0, depths.astype(np.int64), np.iinfo(np.int64).max)
    owner = np.argmin(key, axis=0)                    # first minimum: the lower index wins ties
    hit = np.take_along_axis(depths, owner[None], 0)[0] > 0
    depth = np.where(hit, np.take_along_axis(depths, owner[None], 0)[0], 0).astype(np.uint16)
    cols = np.stack([c for _, c in imgs])
    rgba = np.take_along_axis(cols, owner[None, ..., None], 0)[0]
    rgba = np.where(hit[..., None], rgba, 0).astype(np.uint8)
    return depth, rgba, np.where(hit, owner, -1).astype(np.int8), depths


@dataclass
class FusedBlocks:
    """Blocks of a fused scene (coordinates, tsdf, colour, weights), sorted by (bz, by, bx); has
    the fields oracle.Scene and the library's scene creation read."""
    coords: np.ndarray
    tsdf: np.ndarray
    rgba: np.ndarray
    weight: np.ndarray
    voxel_size: float
    mu: float


class FusionScene:
    """TSDF fusion of depth (+ colour) frames into a growing block scene (Sec. 3.3 (a), Appendix
    B.3; the rules are stated above orc_fusion_frame in relo_oracle.c)."""

    def __init__(self, capacity, voxel_size, mu, max_weight=100):
        self.voxel_size, self.mu = float(voxel_size), float(mu)
        self._h = _lib().orc_fusion_create(int(capacity), self.voxel_size, self.mu, int(max_weight))
        if not self._h:
            raise MemoryError("oracle fusion scene")

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().orc_fusion_destroy(self._h)
            self._h = None

    def fuse(self, intr, pose, depth, rgba=None) -> bool:
        """Fuse one frame (depth uint16 mm [H][W], rgba uint8 [H][W][4] or None) at camera-to-scene
        pose; False if the block capacity ran out."""
        K = np.array([intr.fx, intr.fy, intr.cx, intr.cy], dtype=np.float64)
        d, pd = _c(depth, np.uint16)
        c, pc = (None, None) if rgba is None else _c(rgba, np.uint8)
        rc = _lib().orc_fusion_frame(self._h, intr.width, intr.height, _d(K), intr.depth_min, intr.depth_max,
                                     _d(np.asarray(pose, dtype=np.float64).reshape(16)), pd, pc)
        return rc == 0

    def blocks(self) -> FusedBlocks:
        n = _lib().orc_fusion_count(self._h)
        coords = np.empty((n, 3), dtype=np.int32)
        tsdf = np.empty((n, 512), dtype=np.float32)
        rgba = np.empty((n, 512, 4), dtype=np.uint8)
        weight = np.empty((n, 512), dtype=np.uint16)
        if n:
            _lib().orc_fusion_export(self._h, coords.ctypes.data, tsdf.ctypes.data, rgba.ctypes.data,
                                     weight.ctypes.data)
        order = np.lexsort((coords[:, 0], coords[:, 1], coords[:, 2]))
        return FusedBlocks(coords[order], tsdf[order], rgba[order], weight[order], self.voxel_size, self.mu)


def raycast_touched(scene: Scene, intr, pose, with_colour: bool) -> dict:
    """Distinct data one view's raycast reads: tsdf voxels, colour voxels (query renders only)
    and block keys looked up -- the algorithmic input bytes of that raycast."""
    K = np.array([intr.fx, intr.fy, intr.cx, intr.cy], dtype=np.float64)
    out = np.zeros(3, dtype=np.int64)
    rc = _lib().orc_raycast_touched(scene._h, intr.width, intr.height, _d(K), intr.depth_min, intr.depth_max,
                                    _d(np.asarray(pose, dtype=np.float64).reshape(16)), int(with_colour),
                                    out.ctypes.data)
    if rc != 0:
        raise MemoryError("raycast_touched")
    return dict(tsdf_voxels=int(out[0]), colour_voxels=int(out[1]), block_keys=int(out[2]))


def forest_eval(nodes, depth_img, rgba_img) -> np.ndarray:
    """Leaf index per (tree, pixel) -> uint16 [T, H, W]; 0xFFFF where the pixel has no depth."""
    nodes = np.ascontiguousarray(nodes)
    T, n_int = nodes.shape
    D = int(round(math.log2(n_int + 1)))
    H, W = depth_img.shape
    d, pd = _c(depth_img, np.uint16)
    c, pc = _c(rgba_img, np.uint8)
    out = np.empty((T, H, W), dtype=np.uint16)
    _lib().orc_forest_eval(nodes.ctypes.data, T, D, pd, pc, W, H, out.ctypes.data)
    return out


def verify_counts(depth_a, depth_b) -> np.ndarray:
    """[|Omega|, |Omega_a|, |Omega_b|, |Omega_ab|, sum over Omega_ab of |D_a - D_b|] (Sec. 3.3.1)."""
    a, pa = _c(np.asarray(depth_a).reshape(-1), np.uint16)
    b, pb = _c(np.asarray(depth_b).reshape(-1), np.uint16)
    out = np.zeros(5, dtype=np.uint64)
    _lib().orc_verify_counts(pa, pb, len(a), out.ctypes.data)
    return out


def verify_accept(counts, valid_fraction=0.5, max_mean_mm=50) -> bool:
    """Sec. 3.3.1: accept iff |Omega_a| / |Omega| > 0.5 and the mean |D_a - D_b| over Omega_ab is
    below 5 cm.  Reading: an empty Omega_ab rejects."""
    n, oa, _, oab, s = (int(x) for x in counts)
    if not oa > valid_fraction * n:
        return False
    if oab == 0:
        return False
    return s < max_mean_mm * oab


# ------------------------------------------------------------------------------------------------
# Relocaliser training: reservoirs + mean shift (Cavallari et al., as used in Sec. 3.3 (b))
# ------------------------------------------------------------------------------------------------

@dataclass
class LeafParams:
    capacity: int = 64
    max_modes: int = 10
    bandwidth: float = 0.05
    tol: float = 1e-5
    max_iter: int = 50
    merge_dist: float = 0.025
    cov_floor: float = 1e-4
    stride: int = 1
    seed: int = 0


@dataclass
class Forest:
    nodes: np.ndarray        # NODE_DTYPE [T, 2^D - 1]
    modes: np.ndarray        # float32 [T, 2^D, M, 12]
    n_modes: np.ndarray      # uint8 [T, 2^D]

    @property
    def n_trees(self):
        return self.nodes.shape[0]

    @property
    def depth(self):
        return int(round(math.log2(self.nodes.shape[1] + 1)))


class Reservoirs:
    def __init__(self, nodes, p: LeafParams):
        self.nodes = np.ascontiguousarray(nodes)
        self.p = p
        T, n_int = self.nodes.shape
        self.T, self.D = T, int(round(math.log2(n_int + 1)))
        key = seed_key(p.seed)
        self._h = _lib().orc_reservoirs_create(T, self.D, p.capacity, int(key[0]), int(key[1]))
        if not self._h:
            raise MemoryError("oracle reservoirs")

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().orc_reservoirs_destroy(self._h)
            self._h = None

    def add_frame(self, intr, pose, depth_img, rgba_img):
        d, pd = _c(depth_img, np.uint16)
        c, pc = _c(rgba_img, np.uint8)
        K = np.array([intr.fx, intr.fy, intr.cx, intr.cy])
        _lib().orc_reservoirs_add_frame(self._h, self.nodes.ctypes.data, pd, pc, intr.width, intr.height, _d(K),
                                        _d(np.asarray(pose).reshape(16)), self.p.stride)

    def contents(self):
        L = 1 << self.D
        samples = np.zeros((self.T, L, self.p.capacity, 3), dtype=np.float32)
        count = np.zeros((self.T, L), dtype=np.int32)
        _lib().orc_reservoirs_get(self._h, samples.ctypes.data, count.ctypes.data)
        return samples, count

    def modes(self, threads: int = 1) -> Forest:
        """Mean-shift modes of every leaf.  With threads > 1 the leaves are split into ranges that
        threads fill concurrently (the C call releases the GIL; every leaf is computed exactly as
        in the one-thread call, only the order in which leaves are visited differs)."""
        L = 1 << self.D
        modes = np.zeros((self.T, L, self.p.max_modes, 12), dtype=np.float32)
        n_modes = np.zeros((self.T, L), dtype=np.uint8)
        p = self.p
        total = self.T * L

        def fill(lo, hi):
            _lib().orc_fill_modes_range(self._h, lo, hi, p.bandwidth, p.tol, p.max_iter, p.merge_dist, p.cov_floor,
                                        p.max_modes, modes.ctypes.data, n_modes.ctypes.data)

        if threads <= 1:
            fill(0, total)
        else:
            from concurrent.futures import ThreadPoolExecutor
            step = max(1, total // (64 * threads))
            with ThreadPoolExecutor(threads) as ex:
                list(ex.map(lambda lo: fill(lo, min(total, lo + step)), range(0, total, step)))
        return Forest(self.nodes, modes, n_modes)


def mean_shift_leaf(samples, p: LeafParams) -> np.ndarray:
    """Modes of one leaf's samples (float32 [k, 12], see relo_oracle.c for the row layout)."""
    x, px = _c(np.asarray(samples, dtype=np.float32).reshape(-1, 3), np.float32)
    out = np.zeros((max(p.max_modes, 1), 12), dtype=np.float32)
    k = _lib().orc_mean_shift_leaf(px, len(x), p.bandwidth, p.tol, p.max_iter, p.merge_dist, p.cov_floor,
                                   p.max_modes, out.ctypes.data)
    return out[:k]


def train_forest(nodes, frames, p: LeafParams, threads: int = 1) -> Forest:
    """Fill the leaves of a forest from training frames [(intr, pose, depth, rgba), ...] in order
    (``threads``: how many threads compute the leaves' modes)."""
    r = Reservoirs(nodes, p)
    for intr, pose, depth, rgba in frames:
        r.add_frame(intr, pose, depth, rgba)
    return r.modes(threads)


# ------------------------------------------------------------------------------------------------
# Preemptive RANSAC (after Cavallari et al. / Valentin et al.; readings stated inline)
# ------------------------------------------------------------------------------------------------

@dataclass
class RansacParams:
    n_hyps: int = 64             # K
    batch: int = 500             # B pixels added per round
    max_tries: int = 10000       # draws per hypothesis before it is declared invalid
    rigidity: float = 0.05       # |dist_cam - dist_scene| tolerance (m)
    min_area: float = 1e-3       # |cross| of the correspondence triangle (m^2)
    inlier_dist: float = 0.1     # refinement inlier radius (m)
    seed: int = 0


def camera_points(depth_img, intr, pixels) -> np.ndarray:
    """Back-projected camera points (FP64) of pixel indices v*W+u: z (u-cx)/fx, z (v-cy)/fy, z; z = d/1000."""
    W = intr.width
    pixels = np.asarray(pixels, dtype=np.int64)
    u = (pixels % W).astype(np.float64)
    v = (pixels // W).astype(np.float64)
    z = depth_img.reshape(-1)[pixels].astype(np.float64) / 1000.0
    return np.stack([z * (u - intr.cx) / intr.fx, z * (v - intr.cy) / intr.fy, z], axis=-1)


def kabsch(c, w):
    """Least-squares rigid transform w ~ R c + t (Kabsch 1976): returns R (3x3), t (3)."""
    c = np.asarray(c, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    cb, wb = c.mean(0), w.mean(0)
    Hm = (c - cb).T @ (w - wb)
    U, S, Vt = np.linalg.svd(Hm)
    V = Vt.T
    d = np.sign(np.linalg.det(V @ U.T))
    if d == 0:
        d = 1.0
    R = V @ np.diag([1.0, 1.0, d]) @ U.T
    return R, wb - R @ cb


def _dist(a, b):
    d0, d1, d2 = a[..., 0] - b[..., 0], a[..., 1] - b[..., 1], a[..., 2] - b[..., 2]
    return np.sqrt(d0 * d0 + d1 * d1 + d2 * d2)


def _cross_norm(p0, p1, p2):
    e1 = p1 - p0
    e2 = p2 - p0
    x = e1[..., 1] * e2[..., 2] - e1[..., 2] * e2[..., 1]
    y = e1[..., 2] * e2[..., 0] - e1[..., 0] * e2[..., 2]
    z = e1[..., 0] * e2[..., 1] - e1[..., 1] * e2[..., 0]
    return np.sqrt(x * x + y * y + z * z)


def valid_pixels(depth_img) -> np.ndarray:
    """Pixel indices with depth > 0, in raster order."""
    return np.nonzero(np.asarray(depth_img).reshape(-1) > 0)[0].astype(np.int64)


def generate_hypotheses(depth_img, intr, leaves, forest: Forest, p: RansacParams):
    """Pose hypotheses from three sampled correspondences each.

    Reading: hypothesis h tries j = 0, 1, ... max_tries-1; try j is the Philox block
    at counter (1, h, j, 0): words 0..2 pick three pixels uniformly among the valid
    pixels, byte k of word 3 picks the tree of correspondence k as floor(byte * T / 256),
    and each correspondence takes its leaf's most supported mode (mode 0).  The try is
    kept when every leaf has a mode, the three pixels differ, every pair's camera-space
    and scene-space distances agree within ``rigidity`` and both triangles have
    |cross| >= ``min_area`` (all tests in FP64 in the order written in _dist and
    _cross_norm).  The pose is Kabsch on the three pairs.
    Returns (poses [K,4,4] camera->scene, valid [K] bool, tries [K] int: index of the kept try).
    """
    key = seed_key(p.seed)
    valid = valid_pixels(depth_img)
    T = forest.n_trees
    K = p.n_hyps
    poses = np.tile(np.eye(4), (K, 1, 1))
    ok = np.zeros(K, dtype=bool)
    tries = np.full(K, p.max_tries, dtype=np.int64)
    if len(valid) == 0:
        return poses, ok, tries
    leaves_flat = leaves.reshape(T, -1)
    chunk = 512
    for h in range(K):
        for j0 in range(0, p.max_tries, chunk):
            js = np.arange(j0, min(j0 + chunk, p.max_tries))
            ctr = np.zeros((len(js), 4), dtype=np.uint32)
            ctr[:, 0] = TAG_HYP
            ctr[:, 1] = h
            ctr[:, 2] = js
            x = philox(ctr, key)
            pix = valid[uniform_below(x[:, :3], len(valid))]                          # [n,3]
            tbytes = np.stack([(x[:, 3] >> np.uint32(8 * k)) & np.uint32(0xFF) for k in range(3)], 1)
            tree = (tbytes.astype(np.int64) * T) >> 8
            leaf = leaves_flat[tree, pix].astype(np.int64)
            nm = forest.n_modes[tree, leaf].astype(np.int64)
            has = (nm > 0).all(1)
            distinct = (pix[:, 0] != pix[:, 1]) & (pix[:, 0] != pix[:, 2]) & (pix[:, 1] != pix[:, 2])
            cam = camera_points(depth_img, intr, pix.reshape(-1)).reshape(len(js), 3, 3)
            wld = forest.modes[tree, leaf, 0, :3].astype(np.float64)
            rigid = np.ones(len(js), dtype=bool)
            for a, b in ((0, 1), (0, 2), (1, 2)):
                rigid &= np.abs(_dist(cam[:, a], cam[:, b]) - _dist(wld[:, a], wld[:, b])) <= p.rigidity
            area = (_cross_norm(cam[:, 0], cam[:, 1], cam[:, 2]) >= p.min_area) & (
                _cross_norm(wld[:, 0], wld[:, 1], wld[:, 2]) >= p.min_area)
            good = has & distinct & rigid & area
            if good.any():
                i = int(np.argmax(good))
                R, t = kabsch(cam[i], wld[i])
                poses[h, :3, :3], poses[h, :3, 3] = R, t
                ok[h] = True
                tries[h] = int(js[i])
                break
    return poses, ok, tries


def pixel_energies(pose, cam, pix, leaves, forest: Forest):
    """Per-pixel energy and best mode under one pose.

    Reading (Gaussian-mode likelihood of Valentin et al.): for x = R c + t,
    e = -log(max(1e-30, max over trees t and modes m of w_m N(x; mu_m, Sigma_m)))
    evaluated in the log domain as min(-log 1e-30, -max(logw_m - 0.5 log det(2 pi Sigma_m)
    - 0.5 (x-mu)^T Sigma^-1 (x-mu))).  Returns (e [n], best score mu [n,3] or nan, best found [n]).
    """
    R, t = pose[:3, :3], pose[:3, 3]
    x = cam @ R.T + t                                           # [n,3]
    T = forest.n_trees
    lf = leaves.reshape(T, -1)[:, pix].astype(np.int64).T      # [n,T]
    M = forest.modes.shape[2]
    md = forest.modes[np.arange(T)[None, :], lf].astype(np.float64)   # [n,T,M,12]
    nm = forest.n_modes[np.arange(T)[None, :], lf].astype(np.int64)   # [n,T]
    present = np.arange(M)[None, None, :] < nm[..., None]            # [n,T,M]
    dlt = x[:, None, None, :] - md[..., :3]
    i00, i01, i02, i11, i12, i22 = (md[..., k] for k in range(3, 9))
    q = (dlt[..., 0] * (i00 * dlt[..., 0] + i01 * dlt[..., 1] + i02 * dlt[..., 2]) +
         dlt[..., 1] * (i01 * dlt[..., 0] + i11 * dlt[..., 1] + i12 * dlt[..., 2]) +
         dlt[..., 2] * (i02 * dlt[..., 0] + i12 * dlt[..., 1] + i22 * dlt[..., 2]))
    score = np.where(present, md[..., 9] - 0.5 * q, -np.inf).reshape(len(pix), -1)
    best = score.argmax(1)          # first maximum in (tree, mode) order
    best_score = score[np.arange(len(pix)), best]
    e = np.minimum(LOG_EPS, -best_score)
    mu = md[..., :3].reshape(len(pix), -1, 3)[np.arange(len(pix)), best]
    found = np.isfinite(best_score)
    return e, mu, found, x


def decision_margins(pose, cam, pix, leaves, forest: Forest, inlier_dist: float):
    """Distance of each pixel's discrete decisions from their thresholds under one pose:
    (| |x - mu_best| - inlier_dist |, best score - second best score).  Used by the parity
    tests to tell genuine disagreements from near-ties that FP32 may resolve either way."""
    R, t = pose[:3, :3], pose[:3, 3]
    x = cam @ R.T + t
    T = forest.n_trees
    lf = leaves.reshape(T, -1)[:, pix].astype(np.int64).T
    M = forest.modes.shape[2]
    md = forest.modes[np.arange(T)[None, :], lf].astype(np.float64)
    nm = forest.n_modes[np.arange(T)[None, :], lf].astype(np.int64)
    present = np.arange(M)[None, None, :] < nm[..., None]
    dlt = x[:, None, None, :] - md[..., :3]
    i00, i01, i02, i11, i12, i22 = (md[..., k] for k in range(3, 9))
    q = (dlt[..., 0] * (i00 * dlt[..., 0] + i01 * dlt[..., 1] + i02 * dlt[..., 2]) +
         dlt[..., 1] * (i01 * dlt[..., 0] + i11 * dlt[..., 1] + i12 * dlt[..., 2]) +
         dlt[..., 2] * (i02 * dlt[..., 0] + i12 * dlt[..., 1] + i22 * dlt[..., 2]))
    score = np.where(present, md[..., 9] - 0.5 * q, -np.inf).reshape(len(pix), -1)
    srt = np.sort(score, axis=1)
    best = srt[:, -1]
    second = srt[:, -2] if srt.shape[1] > 1 else np.full(len(pix), -np.inf)
    arg = score.argmax(1)
    mu = md[..., :3].reshape(len(pix), -1, 3)[np.arange(len(pix)), arg]
    dist = np.where(np.isfinite(best), _dist(x, mu), np.inf)
    dm = np.abs(dist - inlier_dist)
    am = np.where(np.isfinite(second), best - second, np.inf)
    return dm, am


@dataclass
class RansacTrace:
    poses0: np.ndarray                       # hypotheses [K,4,4]
    valid0: np.ndarray                       # [K]
    rounds: list = field(default_factory=list)   # per round: dict(pixels, energy, alive_before, survivors, poses, inliers)


def preemptive_ransac(depth_img, intr, leaves, forest: Forest, p: RansacParams, trace: bool = False,
                      hypotheses=None):
    """Preemptive RANSAC (reading, after Cavallari et al.):

    hypotheses from generate_hypotheses; K_0 = K; while K_r > 1: draw B pixels
    uniformly (with replacement) from the valid pixels at counters (2, r, i, 0)
    word 0; add each alive hypothesis's summed pixel energies to its energy
    E(h) (invalid hypotheses keep E = +inf); sort alive hypotheses by (E, h) and
    keep the first ceil(K_r / 2); re-fit every survivor by Kabsch on its inliers
    among all pixels drawn so far (pixel inlier when its best mode lies within
    ``inlier_dist`` of R c + t), keeping the pose when fewer than 3 inliers.
    ``hypotheses`` = (poses [K,4,4], valid [K]) skips generation and starts the rounds from them.
    Returns dict(pose [4,4], energy, inliers, valid, trace).
    """
    key = seed_key(p.seed)
    valid = valid_pixels(depth_img)
    if hypotheses is None:
        poses, ok, _ = generate_hypotheses(depth_img, intr, leaves, forest, p)
    else:
        poses, ok = np.array(hypotheses[0], dtype=np.float64), np.array(hypotheses[1], dtype=bool)
    K = p.n_hyps
    E = np.where(ok, 0.0, np.inf)
    alive = np.arange(K)
    tr = RansacTrace(poses.copy(), ok.copy()) if trace else None
    drawn = np.zeros(0, dtype=np.int64)
    inl = np.zeros(K, dtype=np.int64)
    r = 0
    while len(alive) > 1 and len(valid) > 0:
        ctr = np.zeros((p.batch, 4), dtype=np.uint32)
        ctr[:, 0] = TAG_PIX
        ctr[:, 1] = r
        ctr[:, 2] = np.arange(p.batch)
        x = philox(ctr, key)
        pix = valid[uniform_below(x[:, 0], len(valid))]
        drawn = np.concatenate([drawn, pix])
        cam = camera_points(depth_img, intr, pix)
        for h in alive:
            if ok[h]:
                e, _, _, _ = pixel_energies(poses[h], cam, pix, leaves, forest)
                E[h] += e.sum()
        alive_before = alive.copy()
        order = sorted(alive.tolist(), key=lambda h: (E[h], h))
        keep = int(math.ceil(len(alive) / 2))
        alive = np.array(order[:keep], dtype=np.int64)
        cam_all = camera_points(depth_img, intr, drawn)
        for h in alive:
            if not ok[h]:
                continue
            _, mu, found, x3 = pixel_energies(poses[h], cam_all, drawn, leaves, forest)
            d = np.where(found, _dist(x3, mu), np.inf)
            m = d < p.inlier_dist
            inl[h] = int(m.sum())
            if inl[h] >= 3:
                R, t = kabsch(cam_all[m], mu[m])
                poses[h, :3, :3], poses[h, :3, 3] = R, t
        if trace:
            tr.rounds.append(dict(pixels=pix.copy(), energy=E.copy(), alive_before=alive_before,
                                  survivors=alive.copy(), poses=poses.copy(), inliers=inl.copy()))
        r += 1
    best = int(alive[0]) if len(alive) else 0
    return dict(pose=poses[best].copy(), energy=float(E[best]), inliers=int(inl[best]), valid=bool(ok[best]),
                index=best, trace=tr)


# ------------------------------------------------------------------------------------------------
# One relocalisation attempt (Sec. 3.3.1, Fig. 3)
# ------------------------------------------------------------------------------------------------

def relocalise(scene_b: Scene, pose_b, forest_a: Forest, scene_a: Scene, intr, p: RansacParams, noise=None):
    """Render b at pose_b, relocalise in a, verify by a depth raycast of a.

    Returns dict with the proposed camera->a pose, the verification counts and
    decision, and the relative transform sample a_T_b = P_a P_b^-1 (Sec. 3.3.1,
    with P = camera->scene, the inverse of the paper's f_T_s).
    """
    depth_b, rgba_b = scene_b.raycast(intr, pose_b, noise=noise)
    leaves = forest_eval(forest_a.nodes, depth_b, rgba_b)
    res = preemptive_ransac(depth_b, intr, leaves, forest_a, p)
    depth_a, _ = scene_a.raycast(intr, res["pose"])
    counts = verify_counts(depth_a, depth_b)
    res.update(depth_b=depth_b, rgba_b=rgba_b, leaves=leaves, depth_a=depth_a, counts=counts,
               verified=bool(res["valid"]) and verify_accept(counts),
               rel_a_b=res["pose"] @ np.linalg.inv(pose_b))
    return res


def pose_error(P_est, P_gt):
    """(translation error m, rotation error degrees) between two camera->scene poses."""
    dt = float(np.linalg.norm(P_est[:3, 3] - P_gt[:3, 3]))
    c = (np.trace(P_est[:3, :3] @ P_gt[:3, :3].T) - 1.0) / 2.0
    return dt, math.degrees(math.acos(max(-1.0, min(1.0, c))))
