"""Save and load the state an agent's mapping component builds, as .npz files: a forest (split
nodes, leaf modes and counts), the learned regressor's training state (parameters, Adam moments
and step, origin), and a scene (its voxel blocks; a fused scene is saved through relo_scene_export
and loads as a static scene).  The paper keeps each agent's sequence and global pose so that the
sub-scenes can be fused again later (Appendix B.3); these files keep the built state itself.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def save_forest(path, nodes, forest):
    modes, n_modes = forest.get_modes()
    np.savez(path, kind="forest", nodes=np.asarray(nodes), modes=modes, n_modes=n_modes,
             max_modes=np.int32(forest.max_modes))


def load_forest(path):
    """(nodes, forest)."""
    z = np.load(path, allow_pickle=False)
    assert str(z["kind"]) == "forest", "not a forest checkpoint"
    nodes = z["nodes"]
    return nodes, B.Forest(nodes, z["modes"], z["n_modes"], max_modes=int(z["max_modes"]))


def save_regressor(path, reg):
    st = B.regressor_state(reg)
    np.savez(path, kind="regressor", params=st["params"], m=st["m"], v=st["v"], step=np.int64(st["step"]),
             origin=np.asarray(reg.origin, dtype=np.float64))


def load_regressor(path):
    z = np.load(path, allow_pickle=False)
    assert str(z["kind"]) == "regressor", "not a regressor checkpoint"
    reg = B.Regressor(params=z["params"], origin=tuple(float(x) for x in z["origin"]))
    B.regressor_set_state(reg, {"params": z["params"], "m": z["m"], "v": z["v"], "step": int(z["step"])})
    return reg


def save_fused_scene(path, scene, voxel_size, mu):
    coords, tsdf, rgba, weight = scene.export()
    np.savez(path, kind="scene", coords=coords, tsdf=tsdf, rgba=rgba, weight=weight,
             voxel_size=np.float64(voxel_size), mu=np.float64(mu))


class _Blocks:
    def __init__(self, z):
        self.coords, self.tsdf, self.rgba = z["coords"], z["tsdf"], z["rgba"]
        self.voxel_size, self.mu = float(z["voxel_size"]), float(z["mu"])


def load_scene(path, log2_buckets=20):
    """A static scene (raycasts through its dense grid) from a saved scene."""
    z = np.load(path, allow_pickle=False)
    assert str(z["kind"]) == "scene", "not a scene checkpoint"
    return B.Scene(_Blocks(z), log2_buckets)
