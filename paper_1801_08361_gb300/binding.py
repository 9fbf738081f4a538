"""ctypes binding of include/relo.h (argument marshalling only).

Every function keeps the C name without its ``relo_`` prefix and takes torch CUDA tensors
for device buffers (their ``data_ptr()`` is passed through) and a CUDA stream (default: the
current torch stream).  All arithmetic happens in the sm_103a kernels of ``librelo.so``;
``lib()`` raises if the library has not been built, and there is no other code path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RELO_CHECKED=1 in the environment loads the bounds-checked build (build.build_cuda(checked=True))
LIB_PATH = os.path.join(_HERE, "librelo_checked.so" if os.environ.get("RELO_CHECKED") == "1" else "librelo.so")
_LIB = None

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDEVICE, ENOTFOUND, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "RELO_OK", -1: "RELO_EINVAL", -2: "RELO_ENOMEM", -3: "RELO_ECUDA", -4: "RELO_ETIMEOUT",
                -5: "RELO_EDEVICE", -6: "RELO_ENOTFOUND", -7: "RELO_EBUSY"}

c_i32, c_i64, c_u64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class ReloError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Intrinsics(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("fx", c_dbl), ("fy", c_dbl), ("cx", c_dbl), ("cy", c_dbl),
                ("depth_min", c_dbl), ("depth_max", c_dbl)]


class TrainParams(ctypes.Structure):
    _fields_ = [("capacity", c_i32), ("stride", c_i32), ("max_iter", c_i32), ("pad", c_i32), ("seed", c_u64),
                ("bandwidth", c_dbl), ("tol", c_dbl), ("merge_dist", c_dbl), ("cov_floor", c_dbl)]


class RansacParams(ctypes.Structure):
    _fields_ = [("n_hyps", c_i32), ("batch", c_i32), ("max_tries", c_i32), ("pad", c_i32), ("rigidity", c_dbl),
                ("min_area", c_dbl), ("inlier_dist", c_dbl), ("seed", c_u64)]


class PoseResult(ctypes.Structure):
    _fields_ = [("pose_c2s", c_dbl * 16), ("rel_a_b", c_dbl * 16), ("energy", c_dbl), ("n_inliers", c_i32),
                ("status", c_i32), ("verified", c_i32), ("n_valid", c_i32), ("hypothesis", c_i32),
                ("n_rounds", c_i32), ("omega", c_u64), ("omega_a", c_u64), ("omega_b", c_u64),
                ("omega_ab", c_u64), ("sum_absdiff_mm", c_u64), ("tries", c_u64), ("path", c_i32), ("pad", c_i32)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pose_c2s", "rel_a_b")}
        d["pose"] = np.array(self.pose_c2s[:], dtype=np.float64).reshape(4, 4)
        d["rel_a_b"] = np.array(self.rel_a_b[:], dtype=np.float64).reshape(4, 4)
        return d


class Attempt(ctypes.Structure):
    _fields_ = [("scene_b", c_vp), ("forest_a", c_vp), ("scene_a", c_vp), ("intr", Intrinsics),
                ("pose_b", c_dbl * 16), ("noise_dev", c_vp), ("n_hyps", c_i32), ("pad", c_i32), ("seed", c_u64),
                ("regressor_a", c_vp)]


RESULT_BYTES = ctypes.sizeof(PoseResult)


# relo_set_allocator's callbacks: alloc(bytes, ctx) -> device pointer or NULL; free(ptr, ctx)
ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_vp)


class Schedule(ctypes.Structure):
    _fields_ = [("ray_warp_width", c_i32), ("forest_threads", c_i32), ("forest_tiles", c_i32),
                ("search_ctas_per_sm", c_i32), ("refit_per", c_i32), ("persistent", c_i32),
                ("forest_smem_levels", c_i32)]

    def to_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class ServerParams(ctypes.Structure):
    _fields_ = [("max_batch", c_i32), ("max_wait_us", c_i32), ("slots", c_i32), ("pad", c_i32),
                ("workspace_bytes", c_u64), ("ransac", RansacParams)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", c_u64), ("discarded", c_u64), ("batches", c_u64), ("mean_batch", c_dbl),
                ("p50_ms", c_dbl), ("p99_ms", c_dbl), ("max_ms", c_dbl)]

_SIGS = {
    "relo_last_error": (ctypes.c_char_p, []),
    "relo_create_scene": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_dbl, c_dbl, c_i32, ctypes.POINTER(c_vp)]),
    "relo_destroy_scene": (None, [c_vp]),
    "relo_create_fusion_scene": (c_i32, [c_i64, c_dbl, c_dbl, c_i32, c_i32, ctypes.POINTER(c_vp)]),
    "relo_fuse_workspace_size": (ctypes.c_size_t, [c_i32, c_i32]),
    "relo_fuse_frame": (c_i32, [c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(c_dbl), c_vp, c_vp, c_vp,
                                ctypes.c_size_t, c_vp]),
    "relo_fuse_frames": (c_i32, [c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(c_dbl), c_i32, c_vp, c_vp, c_vp,
                                 ctypes.c_size_t, c_vp]),
    "relo_scene_block_count": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "relo_fuse_stats": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32)]),
    "relo_scene_fusion_updates": (c_i32, [c_vp, ctypes.POINTER(c_u64)]),
    "relo_scene_export": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64)]),
    "relo_scene_lookup": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "relo_scene_use_grid": (c_i32, [c_vp, c_i32]),
    "relo_scene_use_apron": (c_i32, [c_vp, c_i32]),
    "relo_raycast_view": (c_i32, [c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(c_dbl), c_vp, c_vp, c_vp, c_vp]),
    "relo_create_forest": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_i32, ctypes.POINTER(c_vp)]),
    "relo_destroy_forest": (None, [c_vp]),
    "relo_forest_get_modes": (c_i32, [c_vp, c_vp, c_vp]),
    "relo_forest_eval": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_vp, c_vp]),
    "relo_forest_train_begin": (c_i32, [c_vp, ctypes.POINTER(TrainParams)]),
    "relo_forest_train_frame": (c_i32, [c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(c_dbl), c_vp, c_vp, c_vp]),
    "relo_forest_train_finish": (c_i32, [c_vp, c_vp]),
    "relo_forest_train_reservoirs": (c_i32, [c_vp, c_vp, c_vp]),
    "relo_ransac_workspace_size": (ctypes.c_size_t, [c_i32, c_i32, ctypes.POINTER(RansacParams)]),
    "relo_ransac_relocalise": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(RansacParams),
                                       c_vp, ctypes.c_size_t, c_vp, c_vp]),
    "relo_ransac_relocalise_noalloc": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(Intrinsics),
                                               ctypes.POINTER(RansacParams), c_vp, c_vp]),
    "relo_ransac_hypotheses": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(RansacParams),
                                       c_vp, ctypes.c_size_t, c_vp, c_vp, c_vp, c_vp]),
    "relo_ransac_round": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(RansacParams), c_i32,
                                  c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "relo_verify": (c_i32, [c_vp, ctypes.POINTER(Intrinsics), c_vp, c_vp, c_vp, c_vp]),
    "relo_batch_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Attempt), c_i32, ctypes.POINTER(RansacParams)]),
    "relo_relocalise_batch": (c_i32, [ctypes.POINTER(Attempt), c_i32, ctypes.POINTER(RansacParams), c_vp,
                                      ctypes.c_size_t, ctypes.POINTER(PoseResult), c_vp]),
    "relo_batch_prepare": (c_i32, [ctypes.POINTER(Attempt), c_i32, ctypes.POINTER(RansacParams), c_vp,
                                   ctypes.c_size_t, ctypes.POINTER(c_vp)]),
    "relo_batch_run": (c_i32, [c_vp, c_vp, c_vp]),
    "relo_batch_launch_count": (c_i32, [c_vp]),
    "relo_batch_destroy": (None, [c_vp]),
    "relo_regressor_param_count": (c_i64, []),
    "relo_create_regressor": (c_i32, [c_vp, c_u64, ctypes.POINTER(c_dbl), ctypes.POINTER(c_vp)]),
    "relo_destroy_regressor": (None, [c_vp]),
    "relo_regressor_get_params": (c_i32, [c_vp, c_vp, c_vp]),
    "relo_regressor_workspace_size": (ctypes.c_size_t, [c_i32, c_i32, c_i32, c_i32]),
    "relo_regressor_forward": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "relo_regressor_gradients": (c_i32, [c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(Intrinsics), c_vp, c_vp, c_vp,
                                         ctypes.c_size_t, c_vp]),
    "relo_regressor_train_step": (c_i32, [c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(Intrinsics), c_vp, ctypes.c_float,
                                          c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "relo_regressor_relocalise_workspace_size": (ctypes.c_size_t, [c_i32, c_i32, ctypes.POINTER(RansacParams)]),
    "relo_regressor_relocalise": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(Intrinsics), ctypes.POINTER(RansacParams),
                                          c_vp, ctypes.c_size_t, c_vp, c_vp]),
    "relo_regressor_relocalise_cells": (c_i32, [c_vp, ctypes.POINTER(ctypes.c_double), c_vp, ctypes.POINTER(Intrinsics),
                                                ctypes.POINTER(RansacParams), c_vp, ctypes.c_size_t, c_vp, c_vp]),
    "relo_batch_enable_timing": (c_i32, [c_vp, c_i32]),
    "relo_batch_stage_ms": (c_i32, [c_vp, ctypes.POINTER(ctypes.c_float), c_i32]),
    "relo_batch_stage_name": (ctypes.c_char_p, [c_i32]),
    "relo_server_create": (c_i32, [ctypes.POINTER(ServerParams), ctypes.POINTER(c_vp)]),
    "relo_server_submit": (c_i32, [c_vp, ctypes.POINTER(Attempt), ctypes.POINTER(c_u64)]),
    "relo_server_wait": (c_i32, [c_vp, c_u64, ctypes.POINTER(PoseResult), ctypes.POINTER(c_dbl)]),
    "relo_server_stats_get": (c_i32, [c_vp, ctypes.POINTER(ServerStats)]),
    "relo_server_destroy": (None, [c_vp]),
    "relo_raycast_views_workspace_size": (ctypes.c_size_t, [c_i32]),
    "relo_raycast_views": (c_i32, [c_vp, ctypes.POINTER(Intrinsics), c_vp, c_i32, c_vp, c_vp, c_vp, c_vp,
                                   ctypes.c_size_t, c_vp]),
    "relo_batch_capture": (c_i32, [c_vp, c_vp]),
    "relo_batch_replay": (c_i32, [c_vp, c_vp]),
    "relo_batch_attempt_images": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp),
                                          ctypes.POINTER(c_vp)]),
    "relo_set_allocator": (c_i32, [ALLOC_FN, FREE_FN, c_vp]),
    "relo_debug_fail_allocations": (None, [c_i32]),
    "relo_debug_conv_path": (None, [c_i32]),
    "relo_debug_conv_stall": (None, [c_i32, c_i32]),
    "relo_debug_persistent_stall": (None, [c_i32, c_i32]),
    "relo_debug_check_failures": (c_i64, []),
    "relo_debug_corrupt_scene": (c_i32, [c_vp]),
    "relo_regressor_get_state": (c_i32, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(c_i64)]),
    "relo_regressor_set_state": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64]),
    "relo_render_global_workspace_size": (ctypes.c_size_t, [c_i32]),
    "relo_render_global": (c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(c_dbl), c_i32, ctypes.POINTER(Intrinsics),
                                   ctypes.POINTER(c_dbl), c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "relo_batch_get_schedule": (c_i32, [c_vp, ctypes.POINTER(Schedule)]),
    "relo_batch_set_schedule": (c_i32, [c_vp, ctypes.POINTER(Schedule)]),
    "relo_batch_autotune": (c_i32, [c_vp, c_i32, ctypes.POINTER(Schedule), c_vp]),
    "relo_pose_graph_create": (c_i32, [c_i32, ctypes.POINTER(c_vp)]),
    "relo_pose_graph_destroy": (None, [c_vp]),
    "relo_pose_graph_add_sample": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_dbl), ctypes.POINTER(c_i32)]),
    "relo_pose_graph_optimise": (c_i32, [c_vp, ctypes.POINTER(c_dbl), ctypes.POINTER(c_i32), ctypes.POINTER(c_dbl)]),
    "relo_pose_graph_mark_tried": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_dbl)]),
    "relo_pose_graph_score": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl)]),
    "relo_pose_graph_cluster_count": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_i32), c_i32]),
    "relo_pose_graph_cluster_blend": (c_i32, [c_vp, c_i32, c_i32, c_i32, ctypes.POINTER(c_dbl)]),
}

STAGES = ["query_raycast", "learned_forward", "learned_hypotheses", "learned_rounds", "learned_verify", "forest_eval",
          "forest_hypotheses", "forest_rounds", "forest_verify", "merge"]
PATH_FOREST, PATH_LEARNED, PATH_FALLBACK = 0, 1, 2

EXPORTED = sorted(_SIGS)


def lib():
    """The loaded library; raises if it is missing (there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1801_08361_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(status):
    if status != OK:
        raise ReloError(status, lib().relo_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        import torch
        return c_vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_vp(stream)
    return c_vp(stream.cuda_stream)


def _ptr(t):
    return None if t is None else c_vp(t.data_ptr())


def intrinsics(intr) -> Intrinsics:
    """From any object with width, height, fx, fy, cx, cy, depth_min, depth_max."""
    return Intrinsics(int(intr.width), int(intr.height), float(intr.fx), float(intr.fy), float(intr.cx),
                      float(intr.cy), float(intr.depth_min), float(intr.depth_max))


def _pose(p):
    a = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(16))
    return (c_dbl * 16)(*a.tolist())


def ransac_params(n_hyps=64, batch=500, max_tries=10000, rigidity=0.05, min_area=1e-3, inlier_dist=0.1, seed=0):
    return RansacParams(int(n_hyps), int(batch), int(max_tries), 0, float(rigidity), float(min_area),
                        float(inlier_dist), int(seed))


def train_params(capacity=64, stride=1, max_iter=50, seed=0, bandwidth=0.05, tol=1e-5, merge_dist=0.025,
                 cov_floor=1e-4):
    return TrainParams(int(capacity), int(stride), int(max_iter), 0, int(seed), float(bandwidth), float(tol),
                       float(merge_dist), float(cov_floor))


# ------------------------------------------------------------------------------------------------
# Handles
# ------------------------------------------------------------------------------------------------

class Scene:
    """Device-resident voxel sub-scene (relo_create_scene)."""

    def __init__(self, blocks, log2_buckets: int = 20):
        self._keep = (np.ascontiguousarray(blocks.coords, dtype=np.int32),
                      np.ascontiguousarray(blocks.tsdf, dtype=np.float32),
                      np.ascontiguousarray(blocks.rgba, dtype=np.uint8))
        h = c_vp()
        _check(lib().relo_create_scene(self._keep[0].ctypes.data, self._keep[1].ctypes.data,
                                       self._keep[2].ctypes.data, len(self._keep[0]), float(blocks.voxel_size),
                                       float(blocks.mu), int(log2_buckets), ctypes.byref(h)))
        self._keep = None
        self.handle = h.value

    def use_grid(self, enable: bool):
        _check(lib().relo_scene_use_grid(self.handle, 1 if enable else 0))

    def use_apron(self, enable: bool):
        _check(lib().relo_scene_use_apron(self.handle, 1 if enable else 0))

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.relo_destroy_scene(self.handle)
            self.handle = None


def fuse_workspace_size(width, height) -> int:
    return int(lib().relo_fuse_workspace_size(int(width), int(height)))


class FusionScene(Scene):
    """A scene that grows by TSDF fusion (relo_create_fusion_scene / relo_fuse_frame); raycasts,
    verification and global rendering take it like any scene."""

    def __init__(self, capacity, voxel_size, mu, log2_buckets: int = 20, max_weight: int = 100):
        h = c_vp()
        _check(lib().relo_create_fusion_scene(int(capacity), float(voxel_size), float(mu), int(log2_buckets),
                                              int(max_weight), ctypes.byref(h)))
        self.handle = h.value
        self.capacity = int(capacity)
        self._ws = None

    def fuse(self, intr, pose, depth_dev, rgba_dev=None, workspace_dev=None, stream=None):
        """Fuse one frame (depth u16 mm [H][W] as int16 bits, rgba u8 [H][W][4] or None)."""
        if workspace_dev is None:
            need = fuse_workspace_size(intr.width, intr.height)
            if self._ws is None or self._ws.numel() < need:
                import torch
                self._ws = torch.empty(need, dtype=torch.uint8, device=depth_dev.device)
            workspace_dev = self._ws
        ci = intrinsics(intr)
        ph, pp = _poses_host([pose])
        _check(lib().relo_fuse_frame(self.handle, ctypes.byref(ci), ctypes.cast(pp, ctypes.POINTER(c_dbl)),
                                     _ptr(depth_dev), _ptr(rgba_dev), _ptr(workspace_dev), workspace_dev.numel(),
                                     _stream(stream)))

    def fuse_many(self, intr, poses, depth_dev, rgba_dev=None, workspace_dev=None, stream=None):
        """Fuse n frames in order in one call (depth [n][H][W], rgba [n][H][W][4] or None)."""
        if workspace_dev is None:
            need = fuse_workspace_size(intr.width, intr.height)
            if self._ws is None or self._ws.numel() < need:
                import torch
                self._ws = torch.empty(need, dtype=torch.uint8, device=depth_dev.device)
            workspace_dev = self._ws
        ci = intrinsics(intr)
        ph, pp = _poses_host(poses)
        _check(lib().relo_fuse_frames(self.handle, ctypes.byref(ci), ctypes.cast(pp, ctypes.POINTER(c_dbl)),
                                      len(ph), _ptr(depth_dev), _ptr(rgba_dev), _ptr(workspace_dev),
                                      workspace_dev.numel(), _stream(stream)))

    def last_frame_stats(self, intr, workspace_dev=None):
        """(blocks updated, blocks created) by the last frame fused with the workspace."""
        ws = self._ws if workspace_dev is None else workspace_dev
        vis, new = c_i32(), c_i32()
        _check(lib().relo_fuse_stats(_ptr(ws), intr.width, intr.height, ctypes.byref(vis), ctypes.byref(new)))
        return int(vis.value), int(new.value)

    def block_updates(self) -> int:
        """Blocks updated, summed over every frame fused so far."""
        n = c_u64()
        _check(lib().relo_scene_fusion_updates(self.handle, ctypes.byref(n)))
        return int(n.value)

    def block_count(self) -> int:
        n = c_i64()
        _check(lib().relo_scene_block_count(self.handle, ctypes.byref(n)))
        return int(n.value)

    def export(self):
        """(coords [n, 3], tsdf [n, 512], rgba [n, 512, 4], weight [n, 512]) sorted by (bz, by, bx)."""
        n = c_i64()
        _check(lib().relo_scene_block_count(self.handle, ctypes.byref(n)))
        k = int(n.value)
        coords = np.empty((k, 3), np.int32)
        tsdf = np.empty((k, 512), np.float32)
        rgba = np.empty((k, 512, 4), np.uint8)
        weight = np.empty((k, 512), np.uint16)
        _check(lib().relo_scene_export(self.handle, coords.ctypes.data, tsdf.ctypes.data, rgba.ctypes.data,
                                       weight.ctypes.data, k, ctypes.byref(n)))
        order = np.lexsort((coords[:, 0], coords[:, 1], coords[:, 2]))
        return coords[order], tsdf[order], rgba[order], weight[order]


class Forest:
    """Device-resident regression forest (relo_create_forest)."""

    def __init__(self, nodes, modes=None, n_modes=None, max_modes: int = 10):
        nodes = np.ascontiguousarray(nodes)
        T, n_int = nodes.shape
        self.n_trees, self.depth, self.max_modes = T, int(round(np.log2(n_int + 1))), int(max_modes)
        m = None if modes is None else np.ascontiguousarray(modes, dtype=np.float32)
        nm = None if n_modes is None else np.ascontiguousarray(n_modes, dtype=np.uint8)
        h = c_vp()
        _check(lib().relo_create_forest(nodes.ctypes.data, T, self.depth, None if m is None else m.ctypes.data,
                                        None if nm is None else nm.ctypes.data, self.max_modes, ctypes.byref(h)))
        self.handle = h.value

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.relo_destroy_forest(self.handle)
            self.handle = None

    def get_modes(self):
        L = 1 << self.depth
        modes = np.zeros((self.n_trees, L, self.max_modes, 12), np.float32)
        nm = np.zeros((self.n_trees, L), np.uint8)
        _check(lib().relo_forest_get_modes(self.handle, modes.ctypes.data, nm.ctypes.data))
        return modes, nm


# ------------------------------------------------------------------------------------------------
# Entry points
# ------------------------------------------------------------------------------------------------

def scene_lookup(scene, keys_dev, out_dev, stream=None):
    _check(lib().relo_scene_lookup(scene.handle, _ptr(keys_dev), int(keys_dev.shape[0]), _ptr(out_dev),
                                   _stream(stream)))


def raycast_view(scene, intr, pose, depth_dev, rgba_dev=None, noise_dev=None, stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_raycast_view(scene.handle, ctypes.byref(ci), _pose(pose), _ptr(noise_dev), _ptr(depth_dev),
                                   _ptr(rgba_dev), _stream(stream)))


def raycast_views_workspace_size(n) -> int:
    return int(lib().relo_raycast_views_workspace_size(int(n)))


def raycast_views(scene, intr, poses, depth_dev, rgba_dev=None, noise_dev=None, workspace_dev=None, stream=None):
    """n views in one launch: depth_dev [n][H][W], rgba_dev [n][H][W][4], noise_dev [n][H][W]."""
    n = int(depth_dev.shape[0])
    ci = intrinsics(intr)
    ph, pp = _poses_host(poses)
    _check(lib().relo_raycast_views(scene.handle, ctypes.byref(ci), pp, n, _ptr(noise_dev), _ptr(depth_dev),
                                    _ptr(rgba_dev), _ptr(workspace_dev),
                                    0 if workspace_dev is None else workspace_dev.numel(), _stream(stream)))


def render_global_workspace_size(n) -> int:
    return int(lib().relo_render_global_workspace_size(int(n)))


def render_global(scenes, global_poses, intr, pose_global, depth_dev, rgba_dev=None, owner_dev=None, err_dev=None,
                  workspace_dev=None, stream=None):
    """Global map rendering: the scenes placed by global_poses [n][4][4] (gT_a), seen from the
    camera -> global pose pose_global; per pixel the nearest scene wins (owner_dev: its index)."""
    n = len(scenes)
    hs = (c_vp * n)(*[sc.handle for sc in scenes])
    g = np.ascontiguousarray(np.asarray(global_poses, dtype=np.float64).reshape(n, 16))
    pg = np.ascontiguousarray(np.asarray(pose_global, dtype=np.float64).reshape(16))
    ci = intrinsics(intr)
    if workspace_dev is None:
        import torch
        workspace_dev = torch.empty(render_global_workspace_size(n), dtype=torch.uint8, device=depth_dev.device)
    _check(lib().relo_render_global(hs, g.ctypes.data_as(ctypes.POINTER(c_dbl)), n, ctypes.byref(ci),
                                    pg.ctypes.data_as(ctypes.POINTER(c_dbl)), _ptr(depth_dev), _ptr(rgba_dev),
                                    _ptr(owner_dev), _ptr(err_dev), _ptr(workspace_dev), workspace_dev.numel(),
                                    _stream(stream)))


def forest_eval(forest, depth_dev, rgba_dev, leaves_dev, stream=None):
    H, W = depth_dev.shape[-2:]
    _check(lib().relo_forest_eval(forest.handle, _ptr(depth_dev), _ptr(rgba_dev), int(W), int(H), _ptr(leaves_dev),
                                  _stream(stream)))


def forest_train_begin(forest, params: TrainParams):
    _check(lib().relo_forest_train_begin(forest.handle, ctypes.byref(params)))


def forest_train_frame(forest, intr, pose, depth_dev, rgba_dev, stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_forest_train_frame(forest.handle, ctypes.byref(ci), _pose(pose), _ptr(depth_dev),
                                         _ptr(rgba_dev), _stream(stream)))


def forest_train_finish(forest, stream=None):
    _check(lib().relo_forest_train_finish(forest.handle, _stream(stream)))


def forest_train_reservoirs(forest, capacity):
    L = 1 << forest.depth
    samples = np.zeros((forest.n_trees, L, capacity, 3), np.float32)
    count = np.zeros((forest.n_trees, L), np.int32)
    _check(lib().relo_forest_train_reservoirs(forest.handle, samples.ctypes.data, count.ctypes.data))
    return samples, count


def ransac_workspace_size(width, height, params: RansacParams) -> int:
    return int(lib().relo_ransac_workspace_size(int(width), int(height), ctypes.byref(params)))


def ransac_relocalise(forest, depth_dev, leaves_dev, intr, params, workspace_dev, result_dev, stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_ransac_relocalise(forest.handle, _ptr(depth_dev), _ptr(leaves_dev), ctypes.byref(ci),
                                        ctypes.byref(params), _ptr(workspace_dev), workspace_dev.numel(),
                                        _ptr(result_dev), _stream(stream)))


STATIC_SCRATCH_BYTES = 8 << 20


def ransac_relocalise_noalloc(forest, depth_dev, leaves_dev, intr, params, result_dev, stream=None):
    """relo_ransac_relocalise_noalloc: no workspace; the library's fixed scratch array is used."""
    ci = intrinsics(intr)
    _check(lib().relo_ransac_relocalise_noalloc(forest.handle, _ptr(depth_dev), _ptr(leaves_dev), ctypes.byref(ci),
                                                ctypes.byref(params), _ptr(result_dev), _stream(stream)))


def ransac_hypotheses(forest, depth_dev, leaves_dev, intr, params, workspace_dev, poses_dev, valid_dev, tries_dev,
                      stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_ransac_hypotheses(forest.handle, _ptr(depth_dev), _ptr(leaves_dev), ctypes.byref(ci),
                                        ctypes.byref(params), _ptr(workspace_dev), workspace_dev.numel(),
                                        _ptr(poses_dev), _ptr(valid_dev), _ptr(tries_dev), _stream(stream)))


def ransac_round(forest, depth_dev, leaves_dev, intr, params, rnd, alive_dev, valid_dev, poses_dev, energy_dev,
                 drawn_dev, survivors_dev, inliers_dev, workspace_dev, stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_ransac_round(forest.handle, _ptr(depth_dev), _ptr(leaves_dev), ctypes.byref(ci),
                                   ctypes.byref(params), int(rnd), _ptr(alive_dev), int(alive_dev.numel()),
                                   _ptr(valid_dev), _ptr(poses_dev), _ptr(energy_dev), _ptr(drawn_dev),
                                   _ptr(survivors_dev), _ptr(inliers_dev), _ptr(workspace_dev),
                                   workspace_dev.numel(), _stream(stream)))


def verify(scene_a, intr, depth_b_dev, result_dev, depth_a_dev=None, stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_verify(scene_a.handle, ctypes.byref(ci), _ptr(depth_b_dev), _ptr(result_dev),
                             _ptr(depth_a_dev), _stream(stream)))


def result_from_bytes(t) -> dict:
    """Decode a relo_pose_result held in a (CPU) uint8 tensor / bytes."""
    raw = bytes(t.cpu().numpy().tobytes()) if hasattr(t, "cpu") else bytes(t)
    return PoseResult.from_buffer_copy(raw[:RESULT_BYTES]).to_dict()


def make_attempts(items) -> "ctypes.Array":
    """items: dicts with scene_b, scene_a, forest_a and/or regressor_a, intr, pose_b, noise (tensor or
    None), n_hyps, seed."""
    arr = (Attempt * len(items))()
    for i, it in enumerate(items):
        a = arr[i]
        a.scene_b, a.scene_a = it["scene_b"].handle, it["scene_a"].handle
        a.forest_a = None if it.get("forest_a") is None else it["forest_a"].handle
        a.regressor_a = None if it.get("regressor_a") is None else it["regressor_a"].handle
        a.intr = intrinsics(it["intr"])
        a.pose_b = _pose(it["pose_b"])
        a.noise_dev = None if it.get("noise") is None else it["noise"].data_ptr()
        a.n_hyps = int(it.get("n_hyps", 0))
        a.seed = int(it.get("seed", 0))
    return arr


def make_attempts_view(attempts, n):
    """The first n attempts of a relo_attempt array, as an array of their own."""
    arr = (Attempt * n)()
    for k in range(n):
        arr[k] = attempts[k]
    return arr


def batch_workspace_size(attempts, params) -> int:
    return int(lib().relo_batch_workspace_size(attempts, len(attempts), ctypes.byref(params)))


def relocalise_batch_into(attempts, params, workspace_dev, results, stream=None):
    """relo_relocalise_batch into a caller-owned host array of PoseResult (no conversion)."""
    _check(lib().relo_relocalise_batch(attempts, len(attempts), ctypes.byref(params), _ptr(workspace_dev),
                                       workspace_dev.numel(), results, _stream(stream)))
    return results


def relocalise_batch(attempts, params, workspace_dev, stream=None):
    res = relocalise_batch_into(attempts, params, workspace_dev, (PoseResult * len(attempts))(), stream)
    return [r.to_dict() for r in res]


class Batch:
    """Prepared batch (relo_batch_prepare / run / launch_count / destroy)."""

    def __init__(self, attempts, params, workspace_dev):
        h = c_vp()
        _check(lib().relo_batch_prepare(attempts, len(attempts), ctypes.byref(params), _ptr(workspace_dev),
                                        workspace_dev.numel(), ctypes.byref(h)))
        self.handle = h.value
        self.n = len(attempts)
        self._ws = workspace_dev

    def run(self, results_dev, stream=None):
        _check(lib().relo_batch_run(self.handle, _ptr(results_dev), _stream(stream)))

    def capture(self, results_dev=None):
        """Record one run into the batch's CUDA graph (relo_batch_capture)."""
        _check(lib().relo_batch_capture(self.handle, _ptr(results_dev)))

    def replay(self, stream=None):
        _check(lib().relo_batch_replay(self.handle, _stream(stream)))

    def attempt_images(self, k, width, height, trees=0):
        """Views into the workspace of attempt k's query depth (int16 bits of u16 [H][W]), colour
        (u8 [H][W][4]) and forest leaves (int16 bits of u16 [T][H][W], None without a forest)."""
        d, c, lv = c_vp(), c_vp(), c_vp()
        _check(lib().relo_batch_attempt_images(self.handle, int(k), ctypes.byref(d), ctypes.byref(c),
                                               ctypes.byref(lv)))
        base, n = self._ws.data_ptr(), width * height

        def view(addr, nbytes):
            off = addr - base
            if off < 0 or off + nbytes > self._ws.numel():
                raise ReloError(EINVAL, "attempt image outside the workspace")
            return self._ws[off:off + nbytes]

        import torch
        depth = view(d.value, 2 * n).view(torch.int16).view(height, width)
        rgba = view(c.value, 4 * n).view(height, width, 4)
        leaves = None if not lv.value else view(lv.value, 2 * n * trees).view(torch.int16).view(trees, height, width)
        return depth, rgba, leaves

    @property
    def launch_count(self) -> int:
        return int(lib().relo_batch_launch_count(self.handle))

    def enable_timing(self, on: bool = True):
        _check(lib().relo_batch_enable_timing(self.handle, 1 if on else 0))

    def stage_ms(self) -> dict:
        buf = (ctypes.c_float * len(STAGES))()
        n = lib().relo_batch_stage_ms(self.handle, buf, len(STAGES))
        return {lib().relo_batch_stage_name(k).decode(): float(buf[k]) for k in range(n)}

    def schedule(self) -> dict:
        sc = Schedule()
        _check(lib().relo_batch_get_schedule(self.handle, ctypes.byref(sc)))
        return sc.to_dict()

    def set_schedule(self, **fields):
        """Change schedule fields (relo_schedule); drops a captured graph."""
        sc = Schedule(**{**self.schedule(), **fields})
        _check(lib().relo_batch_set_schedule(self.handle, ctypes.byref(sc)))

    def autotune(self, repeats=2, stream=None) -> dict:
        """Pick the fastest schedule on this batch's own inputs (relo_batch_autotune)."""
        sc = Schedule()
        _check(lib().relo_batch_autotune(self.handle, int(repeats), ctypes.byref(sc), _stream(stream)))
        return sc.to_dict()

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.relo_batch_destroy(self.handle)
            self.handle = None


# ------------------------------------------------------------------------------------------------
# Learned regressor
# ------------------------------------------------------------------------------------------------

def regressor_param_count() -> int:
    return int(lib().relo_regressor_param_count())


class Regressor:
    """Device-resident scene-coordinate regressor (relo_create_regressor)."""

    def __init__(self, params=None, seed: int = 0, origin=(0.0, 0.0, 0.0)):
        h = c_vp()
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        if p is not None and p.size != regressor_param_count():
            raise ValueError("parameter count mismatch")
        org = (c_dbl * 3)(*[float(x) for x in origin])
        _check(lib().relo_create_regressor(None if p is None else p.ctypes.data, int(seed), org, ctypes.byref(h)))
        self.handle = h.value
        self.origin = tuple(float(x) for x in origin)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.relo_destroy_regressor(self.handle)
            self.handle = None

    def params(self):
        p = np.zeros(regressor_param_count(), np.float32)
        _check(lib().relo_regressor_get_params(self.handle, p.ctypes.data, None))
        return p

    def grads(self):
        g = np.zeros(regressor_param_count(), np.float32)
        _check(lib().relo_regressor_get_params(self.handle, None, g.ctypes.data))
        return g


def regressor_state(reg) -> dict:
    """Training checkpoint: {"params", "m", "v"} float32 arrays and the Adam "step"."""
    n = regressor_param_count()
    out = {k: np.empty(n, dtype=np.float32) for k in ("params", "m", "v")}
    step = c_i64()
    _check(lib().relo_regressor_get_state(reg.handle, out["params"].ctypes.data, out["m"].ctypes.data,
                                          out["v"].ctypes.data, ctypes.byref(step)))
    out["step"] = int(step.value)
    return out


def regressor_set_state(reg, state):
    a = {k: np.ascontiguousarray(state[k], dtype=np.float32) for k in ("params", "m", "v")}
    _check(lib().relo_regressor_set_state(reg.handle, a["params"].ctypes.data, a["m"].ctypes.data,
                                          a["v"].ctypes.data, int(state["step"])))


def regressor_workspace_size(n, width, height, training) -> int:
    return int(lib().relo_regressor_workspace_size(int(n), int(width), int(height), 1 if training else 0))


def regressor_forward(reg, depth_dev, rgba_dev, out_dev, workspace_dev, stream=None):
    n, H, W = depth_dev.shape
    _check(lib().relo_regressor_forward(reg.handle, _ptr(depth_dev), _ptr(rgba_dev), int(n), int(W), int(H),
                                        _ptr(out_dev), _ptr(workspace_dev), workspace_dev.numel(), _stream(stream)))


def _poses_host(poses):
    a = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 16))
    return a, a.ctypes.data


def regressor_gradients(reg, depth_dev, rgba_dev, intr, poses, workspace_dev, loss_dev=None, stream=None):
    ci = intrinsics(intr)
    ph, pp = _poses_host(poses)
    _check(lib().relo_regressor_gradients(reg.handle, _ptr(depth_dev), _ptr(rgba_dev), int(depth_dev.shape[0]),
                                          ctypes.byref(ci), pp, _ptr(loss_dev), _ptr(workspace_dev),
                                          workspace_dev.numel(), _stream(stream)))


def regressor_train_step(reg, depth_dev, rgba_dev, intr, poses, lr, workspace_dev, loss_dev=None, stream=None):
    ci = intrinsics(intr)
    ph, pp = _poses_host(poses)
    _check(lib().relo_regressor_train_step(reg.handle, _ptr(depth_dev), _ptr(rgba_dev), int(depth_dev.shape[0]),
                                           ctypes.byref(ci), pp, ctypes.c_float(lr), _ptr(loss_dev),
                                           _ptr(workspace_dev), workspace_dev.numel(), _stream(stream)))


def regressor_relocalise_workspace_size(width, height, params) -> int:
    return int(lib().relo_regressor_relocalise_workspace_size(int(width), int(height), ctypes.byref(params)))


def regressor_relocalise(reg, depth_dev, rgba_dev, intr, params, workspace_dev, result_dev, stream=None):
    ci = intrinsics(intr)
    _check(lib().relo_regressor_relocalise(reg.handle, _ptr(depth_dev), _ptr(rgba_dev), ctypes.byref(ci),
                                           ctypes.byref(params), _ptr(workspace_dev), workspace_dev.numel(),
                                           _ptr(result_dev), _stream(stream)))


def regressor_relocalise_cells(cells_dev, origin, depth_dev, intr, params, workspace_dev, result_dev, stream=None):
    """The cell-grid RANSAC of the learned path on given cell outputs cells_dev [H/8][W/8][4]
    (scene coordinate - origin, log-variance)."""
    ci = intrinsics(intr)
    o = (ctypes.c_double * 3)(*[float(x) for x in origin])
    _check(lib().relo_regressor_relocalise_cells(_ptr(cells_dev), o, _ptr(depth_dev), ctypes.byref(ci),
                                                 ctypes.byref(params), _ptr(workspace_dev), workspace_dev.numel(),
                                                 _ptr(result_dev), _stream(stream)))


# ------------------------------------------------------------------------------------------------
# Serving
# ------------------------------------------------------------------------------------------------

class Server:
    """Batched serving of single attempts (relo_server_*): submit returns a ticket, wait blocks
    until its result is ready.  Attempts are relo_attempt structs (make_attempts(...)[k])."""

    def __init__(self, ransac, workspace_bytes, max_batch=64, max_wait_us=2000, slots=256):
        prm = ServerParams(int(max_batch), int(max_wait_us), int(slots), 0, int(workspace_bytes), ransac)
        h = c_vp()
        _check(lib().relo_server_create(ctypes.byref(prm), ctypes.byref(h)))
        self.handle = h.value

    def submit(self, attempt) -> int:
        """Ticket of the queued attempt; raises ReloError(EBUSY) when it is discarded."""
        t = c_u64()
        _check(lib().relo_server_submit(self.handle, ctypes.byref(attempt), ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket):
        res, lat = PoseResult(), c_dbl()
        _check(lib().relo_server_wait(self.handle, int(ticket), ctypes.byref(res), ctypes.byref(lat)))
        return res.to_dict(), float(lat.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().relo_server_stats_get(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.relo_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


# Pose graph (host)
# ------------------------------------------------------------------------------------------------

def _mat16(T):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))
    return a, a.ctypes.data_as(ctypes.POINTER(c_dbl))


class PoseGraph:
    """Clusters of relative transform samples per pair of scenes, the pose graph of scene 0's
    component and the candidate score (relo_pose_graph_*).  Transforms are 4x4 arrays; aT_b maps
    scene b's coordinates into scene a's."""

    def __init__(self, n_scenes):
        h = c_vp()
        _check(lib().relo_pose_graph_create(int(n_scenes), ctypes.byref(h)))
        self.handle = h.value
        self.n = int(n_scenes)

    def add_sample(self, a, b, aTb) -> int:
        """Size of the cluster the sample joined."""
        m, p = _mat16(aTb)
        size = c_i32()
        _check(lib().relo_pose_graph_add_sample(self.handle, int(a), int(b), p, ctypes.byref(size)))
        return int(size.value)

    def optimise(self):
        """(global poses [n, 4, 4], in-graph flags [n] bool, epsilon)."""
        poses = np.zeros((self.n, 16), dtype=np.float64)
        flags = np.zeros(self.n, dtype=np.int32)
        eps = c_dbl()
        _check(lib().relo_pose_graph_optimise(self.handle, poses.ctypes.data_as(ctypes.POINTER(c_dbl)),
                                              flags.ctypes.data_as(ctypes.POINTER(c_i32)), ctypes.byref(eps)))
        return poses.reshape(self.n, 4, 4), flags.astype(bool), float(eps.value)

    def mark_tried(self, a, b, pose_in_b):
        m, p = _mat16(pose_in_b)
        _check(lib().relo_pose_graph_mark_tried(self.handle, int(a), int(b), p))

    def score(self, a, b, pose_in_b) -> float:
        m, p = _mat16(pose_in_b)
        out = c_dbl()
        _check(lib().relo_pose_graph_score(self.handle, int(a), int(b), p, ctypes.byref(out)))
        return float(out.value)

    def cluster_sizes(self, a, b):
        n = lib().relo_pose_graph_cluster_count(self.handle, int(a), int(b), None, 0)
        if n < 0:
            raise ReloError(EINVAL, "bad scene pair")
        sizes = (c_i32 * max(n, 1))()
        lib().relo_pose_graph_cluster_count(self.handle, int(a), int(b), sizes, n)
        return [int(sizes[k]) for k in range(n)]

    def cluster_blend(self, a, b, c):
        """Blend of cluster c of the pair, as aT_b (4x4)."""
        out = np.zeros(16, dtype=np.float64)
        _check(lib().relo_pose_graph_cluster_blend(self.handle, int(a), int(b), int(c),
                                                   out.ctypes.data_as(ctypes.POINTER(c_dbl))))
        return out.reshape(4, 4)

    def close(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.relo_pose_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


# Device memory (relo_set_allocator)
# ------------------------------------------------------------------------------------------------
# Every callback pair handed to the library stays referenced for the life of the process: blocks
# go back to the functions that gave them, even after the allocator changed.
_ALLOCATORS = []


def set_allocator(alloc=None, free=None):
    """Route the library's device allocations through alloc(nbytes) -> int device pointer (0 or an
    exception: the allocation fails) and free(ptr), both Python callables; set_allocator() goes
    back to cudaMalloc / cudaFree.  Blocks allocated earlier go back to the allocator that gave
    them; the library synchronises the device before it calls free."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        _check(lib().relo_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def _alloc(nbytes, _ctx):
        try:
            return int(alloc(int(nbytes))) or None
        except Exception:     # noqa: BLE001 -- reported to the library as a failed allocation
            return None

    def _free(ptr, _ctx):
        free(int(ptr))

    pair = (ALLOC_FN(_alloc), FREE_FN(_free))
    _ALLOCATORS.append(pair)
    _check(lib().relo_set_allocator(pair[0], pair[1], None))


def use_torch_allocator(device=None):
    """The library's device memory from torch's caching allocator (torch.cuda.memory_allocated
    then counts scenes, forests, regressors and servers)."""
    import torch
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n, device), torch.cuda.caching_allocator_delete)


# Fault injection (tests of the error paths)
# ------------------------------------------------------------------------------------------------

def debug_conv_path(use_tcgen05: bool):
    lib().relo_debug_conv_path(1 if use_tcgen05 else 0)


def debug_conv_stall(tile: int, timeout_ms: int = 0):
    lib().relo_debug_conv_stall(int(tile), int(timeout_ms))


def debug_persistent_stall(stall: bool, timeout_ms: int = 0):
    lib().relo_debug_persistent_stall(1 if stall else 0, int(timeout_ms))


def debug_fail_allocations(n):
    """The library's next n device allocations fail (RELO_ENOMEM); 0 cancels."""
    lib().relo_debug_fail_allocations(int(n))


def debug_corrupt_scene(scene):
    """Every hash chain of the scene ends in a cycle: hash walks hit their bound (RELO_EDEVICE)."""
    _check(lib().relo_debug_corrupt_scene(scene.handle))
