"""Hand-built voxel scenes for pins: an analytic SDF sampled at voxel centres by the test itself."""
import numpy as np

from paper_1801_08361_gb300.synth import SceneBlocks


def blocks_from_sdf(sdf, colour, lo, hi, voxel=0.005, mu=0.02):
    """Blocks of 8^3 voxels covering [lo, hi] whose voxels include |sdf| < mu.

    sdf(points [n,3]) -> [n]; colour(points) -> uint8 [n,3].
    """
    bs = 8 * voxel
    blo = np.floor(np.asarray(lo) / bs).astype(int) - 1
    bhi = np.floor(np.asarray(hi) / bs).astype(int) + 1
    g = np.stack(np.meshgrid(*[np.arange(a, b + 1) for a, b in zip(blo, bhi)], indexing="ij"), -1).reshape(-1, 3)
    loc = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    loc = loc[np.lexsort((loc[:, 0], loc[:, 1], loc[:, 2]))]          # local index x + 8y + 64z
    coords, tsdf, rgba = [], [], []
    for i in range(0, len(g), 4096):
        gb = g[i:i + 4096]
        vox = (gb[:, None, :] * 8 + loc[None, :, :]) * voxel            # [nb,512,3]
        d = sdf(vox.reshape(-1, 3)).reshape(len(gb), 512)
        keep = (np.abs(d) < mu).any(1)
        if keep.any():
            coords.append(gb[keep])
            tsdf.append(np.clip(d[keep] / mu, -1, 1).astype(np.float32))
            c = colour(vox[keep].reshape(-1, 3)).reshape(-1, 512, 3)
            rgba.append(np.concatenate([c, np.full(c.shape[:2] + (1,), 255, np.uint8)], -1))
    coords = np.concatenate(coords).astype(np.int32)
    order = np.lexsort((coords[:, 0], coords[:, 1], coords[:, 2]))
    return SceneBlocks(np.ascontiguousarray(coords[order]), np.ascontiguousarray(np.concatenate(tsdf)[order]),
                       np.ascontiguousarray(np.concatenate(rgba)[order]), voxel, mu, np.eye(4))


def empty_blocks(voxel=0.005, mu=0.02):
    return SceneBlocks(np.zeros((0, 3), np.int32), np.zeros((0, 512), np.float32), np.zeros((0, 512, 4), np.uint8),
                       voxel, mu, np.eye(4))


def ray_dirs(intr, pose):
    """World ray directions with camera-z = 1 for every pixel, [H, W, 3], and the centre."""
    v, u = np.mgrid[0:intr.height, 0:intr.width].astype(np.float64)
    dc = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, np.ones_like(u)], -1)
    return dc @ pose[:3, :3].T, pose[:3, 3]


def ray_box_entry(C, d, lo, hi):
    """Slab-method entry parameter of rays C + l d into box [lo, hi] (inf if missed / behind)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - C) / d
        t2 = (hi - C) / d
    tmin = np.nanmax(np.minimum(t1, t2), -1)
    tmax = np.nanmin(np.maximum(t1, t2), -1)
    hit = (tmax >= tmin) & (tmax > 0)
    return np.where(hit & (tmin > 0), tmin, np.inf)


def ray_box_exit(C, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - C) / d
        t2 = (hi - C) / d
    return np.nanmin(np.maximum(t1, t2), -1)
