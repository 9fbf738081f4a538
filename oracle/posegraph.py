"""Plain FP64 oracle of the inter-agent pose optimisation (Sec. 3.3.2) and the candidate score
(Sec. 3.3.1).  Test infrastructure: only tests/ may use it.  It shares no code with the library.

Transforms are 4x4 numpy arrays; aT_b maps scene b's coordinates into scene a's.  Readings (the
paper gives the rules, not every detail), stated identically in the library's header:
- samples of (a, b) and (b, a) share the unordered pair's clusters, kept as aT_b with a < b;
- "within 20 degrees and 10 cm" (Sec. 4.2.4): the rotation angle of R1 R2^T and the distance of
  the translations; a sample joins the first cluster with such a member, else opens a new one;
- confident pair: largest cluster >= N = 2 (Sec. 3.3.1);
- the blend of a cluster: dual quaternion linear blending (Kavan et al. 2006) with equal weights,
  quaternion signs aligned with the first sample's;
- G: the confident pairs of scene 0's connected component; scene 0's global pose is the identity;
- v(T) = (imaginary part of T's rotation quaternion with w >= 0, translation of T); the
  optimisation minimises the sum of squared components of v(gT_b^-1 gT_a aT_b) over the edges,
  epsilon(G) is the sum of their norms as printed (Sec. 3.3.2);
- Phi = phi_new - phi_conf - phi_homog with N = 2 and a penalty of 5 within 5 cm / 5 degrees.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np
from scipy.optimize import least_squares
from scipy.spatial.transform import Rotation

N_CONFIDENT = 2
CLUSTER_DEG, CLUSTER_M = 20.0, 0.10
HOMOG_DEG, HOMOG_M, HOMOG_PENALTY = 5.0, 0.05, 5.0


def rot_angle(R1, R2) -> float:
    """Angle of the rotation R1 R2^T, radians."""
    c = (np.trace(R1 @ R2.T) - 1.0) / 2.0
    return math.acos(max(-1.0, min(1.0, c)))


def close(T1, T2, deg, metres) -> bool:
    return rot_angle(T1[:3, :3], T2[:3, :3]) <= math.radians(deg) and \
        np.linalg.norm(T1[:3, 3] - T2[:3, 3]) <= metres


def quat_wxyz(R) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of R with w >= 0."""
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    q = np.array([w, x, y, z])
    return -q if q[0] < 0 else q


def qmul(a, b) -> np.ndarray:
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def dq_blend(samples) -> np.ndarray:
    """Dual quaternion linear blending with equal weights (Kavan et al. 2006, Sec. 3.3.2)."""
    real = np.zeros(4)
    dual = np.zeros(4)
    q0 = None
    for T in samples:
        q = quat_wxyz(T[:3, :3])
        if q0 is None:
            q0 = q
        if q @ q0 < 0:
            q = -q
        real += q
        dual += 0.5 * qmul(np.concatenate([[0.0], T[:3, 3]]), q)
    n = np.linalg.norm(real)
    real, dual = real / n, dual / n
    out = np.eye(4)
    w, x, y, z = real
    out[:3, :3] = Rotation.from_quat([x, y, z, w]).as_matrix()
    out[:3, 3] = 2.0 * qmul(dual, real * np.array([1, -1, -1, -1]))[1:]
    return out


def vee(T) -> np.ndarray:
    return np.concatenate([quat_wxyz(T[:3, :3])[1:], T[:3, 3]])


class PoseGraph:
    """Clusters per unordered pair, optimisation and scoring, step by step as Sec. 3.3.1-3.3.2."""

    def __init__(self, n: int):
        self.n = n
        self.clusters = {}            # (a, b), a < b -> list of clusters (lists of aT_b)
        self.tried = {}               # (a, b) -> local poses of b's frames tried against a
        self.optimised = [False] * n

    def add_sample(self, a, b, aTb) -> int:
        T = np.asarray(aTb, dtype=np.float64)
        if a > b:
            a, b, T = b, a, np.linalg.inv(T)
        cl = self.clusters.setdefault((a, b), [])
        for c in cl:
            if any(close(s, T, CLUSTER_DEG, CLUSTER_M) for s in c):
                c.append(T)
                return len(c)
        cl.append([T])
        return 1

    def confident_edges(self):
        out = []
        for (a, b), cl in sorted(self.clusters.items()):
            sizes = [len(c) for c in cl]
            if max(sizes) >= N_CONFIDENT:
                out.append((a, b, dq_blend(cl[sizes.index(max(sizes))])))
        return out

    def optimise(self):
        """Returns (global poses [n][4][4], in-graph flags, epsilon)."""
        edges = self.confident_edges()
        adj = {s: [] for s in range(self.n)}
        for e in edges:
            adj[e[0]].append(e)
            adj[e[1]].append(e)
        g = {0: np.eye(4)}
        order = [0]
        dq = deque([0])
        while dq:                                      # connected component of scene 0
            u = dq.popleft()
            for a, b, T in adj[u]:
                v, Tv = (b, g[u] @ T) if a == u else (a, g[u] @ np.linalg.inv(T))
                if v not in g:
                    g[v] = Tv
                    order.append(v)
                    dq.append(v)
        inside = [e for e in edges if e[0] in g and e[1] in g]
        free = order[1:]

        def unpack(x):
            G = {0: np.eye(4)}
            for i, s in enumerate(free):
                T = np.eye(4)
                T[:3, :3] = Rotation.from_rotvec(x[6 * i:6 * i + 3]).as_matrix()
                T[:3, 3] = x[6 * i + 3:6 * i + 6]
                G[s] = T
            return G

        def residuals(x):
            G = unpack(x)
            return np.concatenate([vee(np.linalg.inv(G[b]) @ G[a] @ T) for a, b, T in inside]) if inside \
                else np.zeros(0)

        if free and inside:
            x0 = np.concatenate([np.concatenate([Rotation.from_matrix(g[s][:3, :3]).as_rotvec(), g[s][:3, 3]])
                                 for s in free])
            sol = least_squares(residuals, x0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
            g = unpack(sol.x)
        poses = np.stack([g.get(s, np.eye(4)) for s in range(self.n)])
        flags = [s in g for s in range(self.n)]
        self.optimised = flags
        eps = sum(float(np.linalg.norm(vee(np.linalg.inv(poses[b]) @ poses[a] @ T))) for a, b, T in inside)
        return poses, flags, eps

    def mark_tried(self, a, b, pose_in_b):
        self.tried.setdefault((a, b), []).append(np.asarray(pose_in_b, dtype=np.float64))

    def score(self, a, b, pose_in_b) -> float:
        """Phi of candidate (a, (b, frame)) (Sec. 3.3.1)."""
        phi_new = 1.0 if self.optimised[a] != self.optimised[b] else 0.0
        cl = self.clusters.get((min(a, b), max(a, b)), [])
        phi_conf = max(0.0, max((len(c) for c in cl), default=0) - N_CONFIDENT)
        P = np.asarray(pose_in_b, dtype=np.float64)
        phi_homog = HOMOG_PENALTY if any(close(t, P, HOMOG_DEG, HOMOG_M) for t in self.tried.get((a, b), [])) else 0.0
        return phi_new - phi_conf - phi_homog
