"""FP64 CPU oracle of the learned scene-coordinate regressor (TEST INFRASTRUCTURE ONLY).

The paper relocalises with a regression forest (Sec. 3.3 (b)); the workload adds a small
fully-convolutional network as an alternative relocaliser for a scene, trained online on views
rendered from the scene's own voxel map and used inside the same preemptive RANSAC.  Nothing in
the paper fixes its details; the readings here are implemented identically by the CUDA library:

- input: 4 channels per pixel, centred and scaled: (depth in metres - 3) / 2 (depth 0 where
  invalid) and (R, G, B / 255 - 1/2) x 4;
- layers: eight 3x3 convolutions with zero padding 1, 64 channels; the first three have stride
  2 (so the output grid has one cell per 8 x 8 pixels), the rest stride 1; ReLU after layers
  1-7; layer 8 outputs 4 channels per cell: a scene coordinate relative to a fixed origin o and
  a log-variance s;
- target of cell (cx, cy): the scene coordinate of its centre pixel (8 cx + 4, 8 cy + 4),
  P * backproject(depth) - o, when that pixel has depth (else the cell is not scored);
- loss: mean over scored cells of rho(e) + 1/2 e^2 exp(-s) + 3/2 s, e = |y - y_hat|,
  rho(e) = sqrt(e^2 + 1e-6 m^2): the coordinates are fitted by their (smoothed) Euclidean error,
  which no value of s can discount, and s by the negative log-likelihood of an isotropic
  Gaussian with the error held fixed (that term's gradient does not reach y_hat);
- optimiser: Adam (Kingma and Ba 2015), beta = (0.9, 0.999), eps = 1e-8, FP64 here.

Every operation is the plain definition: a convolution is im2col (a gather) followed by a matrix
product, its gradients the transposed products.  Pinned in tests/test_oracle_regressor.py by
central finite differences and by scipy's correlation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

STRIDES = (2, 2, 2, 1, 1, 1, 1, 1)
CHANNELS = 64
DEPTH_CENTRE, DEPTH_SCALE = 3.0, 0.5       # input channel 0: (depth m - 3) x 0.5
COLOUR_CENTRE, COLOUR_SCALE = 0.5, 4.0     # input channels 1-3: (colour / 255 - 0.5) x 4
RHO_EPS2 = 1e-6                            # m^2: smoothing of the Euclidean coordinate error


def out_size(n: int, stride: int) -> int:
    """Output length of a 3-tap convolution with zero padding 1."""
    return (n - 1) // stride + 1


def im2col(x, stride):
    """x [B, H, W, C] -> columns [B, H', W', 9, C]: tap (ky, kx) of output (oy, ox) reads input
    (stride oy + ky - 1, stride ox + kx - 1), zero outside the image."""
    B, H, W, C = x.shape
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    xp = np.zeros((B, H + 2, W + 2, C), dtype=x.dtype)
    xp[:, 1:H + 1, 1:W + 1] = x
    cols = np.empty((B, Ho, Wo, 9, C), dtype=x.dtype)
    for ky in range(3):
        for kx in range(3):
            cols[:, :, :, 3 * ky + kx] = xp[:, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
    return cols


def col2im(cols, shape, stride):
    """Adjoint of im2col: scatter-add columns [B, H', W', 9, C] back to an image of ``shape``."""
    B, H, W, C = shape
    Ho, Wo = cols.shape[1], cols.shape[2]
    xp = np.zeros((B, H + 2, W + 2, C), dtype=cols.dtype)
    for ky in range(3):
        for kx in range(3):
            xp[:, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride] += cols[:, :, :, 3 * ky + kx]
    return xp[:, 1:H + 1, 1:W + 1]


def conv3x3(x, w, b, stride):
    """x [B, H, W, Cin], w [3, 3, Cin, Cout], b [Cout] -> [B, H', W', Cout]."""
    cols = im2col(x, stride)
    B, Ho, Wo = cols.shape[:3]
    y = cols.reshape(B * Ho * Wo, -1) @ w.reshape(-1, w.shape[-1]) + b
    return y.reshape(B, Ho, Wo, -1)


@dataclass
class Params:
    w: list       # 8 arrays [3, 3, Cin, Cout]
    b: list       # 8 arrays [Cout]

    def flat(self):
        return [p for pair in zip(self.w, self.b) for p in pair]


def init_params(seed: int, channels: int = CHANNELS, in_ch: int = 4, out_ch: int = 4, n_layers: int = 8):
    """He-uniform weights (bound sqrt(6 / fan_in)) from a seeded generator, zero biases; the head's
    weights are scaled by 0.1 so the first log-variances start near 0."""
    rng = np.random.default_rng(seed)
    w, b = [], []
    for l in range(n_layers):
        cin = in_ch if l == 0 else channels
        cout = out_ch if l == n_layers - 1 else channels
        bound = math.sqrt(6.0 / (9 * cin))
        wl = rng.uniform(-bound, bound, (3, 3, cin, cout))
        if l == n_layers - 1:
            wl *= 0.1
        w.append(wl)
        b.append(np.zeros(cout))
    return Params(w, b)


def forward(params: Params, x, strides=STRIDES):
    """Returns (output [B, H/8, W/8, 4], cache of layer inputs / post-activations)."""
    acts = [x]
    h = x
    n = len(params.w)
    for l in range(n):
        z = conv3x3(h, params.w[l], params.b[l], strides[l])
        h = np.maximum(z, 0.0) if l < n - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad_output(out, target, mask):
    """Mean over scored cells of rho(e) + 1/2 e^2 exp(-s) + 3/2 s and the gradient the training
    follows: d rho / d y_hat for the coordinates, the NLL's derivative for s (the error in the
    variance term held fixed).  That gradient is the exact gradient of surrogate_loss at
    sq_fixed = the current squared errors."""
    n = max(int(mask.sum()), 1)
    s = out[..., 3]
    err = out[..., :3] - target
    sq = (err * err).sum(-1)
    rho = np.sqrt(sq + RHO_EPS2)
    e = np.exp(-s)
    per = rho + 0.5 * sq * e + 1.5 * s
    loss = float((per * mask).sum() / n)
    g = np.zeros_like(out)
    g[..., :3] = err * (mask / (n * rho))[..., None]
    g[..., 3] = (-0.5 * sq * e + 1.5) * mask / n
    return loss, g


def surrogate_loss(out, target, mask, sq_fixed):
    """The loss with the squared error of the variance term held at sq_fixed: a plain function of
    the output whose gradient at sq_fixed = the current squared errors is the training gradient."""
    n = max(int(mask.sum()), 1)
    s = out[..., 3]
    err = out[..., :3] - target
    rho = np.sqrt((err * err).sum(-1) + RHO_EPS2)
    return float(((rho + 0.5 * sq_fixed * np.exp(-s) + 1.5 * s) * mask).sum() / n)


def backward(params: Params, acts, g_out, strides=STRIDES):
    """Gradients of the loss with respect to every weight and bias (same layout as params)."""
    n = len(params.w)
    gw, gb = [None] * n, [None] * n
    g = g_out
    for l in reversed(range(n)):
        if l < n - 1:
            g = g * (acts[l + 1] > 0)                 # ReLU of layer l's output
        x = acts[l]
        cols = im2col(x, strides[l])
        B, Ho, Wo = cols.shape[:3]
        g2 = g.reshape(B * Ho * Wo, -1)
        gw[l] = (cols.reshape(B * Ho * Wo, -1).T @ g2).reshape(params.w[l].shape)
        gb[l] = g2.sum(0)
        if l > 0:
            gcols = (g2 @ params.w[l].reshape(-1, params.w[l].shape[-1]).T).reshape(cols.shape)
            g = col2im(gcols, x.shape, strides[l])
    return Params(gw, gb)


@dataclass
class Adam:
    lr: float = 1e-3
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: list = None
    v: list = None

    def step(self, params: Params, grads: Params):
        """theta -= lr * mhat / (sqrt(vhat) + eps), with bias-corrected first and second moments."""
        ps, gs = params.flat(), grads.flat()
        if self.m is None:
            self.m = [np.zeros_like(p) for p in ps]
            self.v = [np.zeros_like(p) for p in ps]
        self.t += 1
        for p, g, m, v in zip(ps, gs, self.m, self.v):
            m *= self.b1
            m += (1 - self.b1) * g
            v *= self.b2
            v += (1 - self.b2) * g * g
            mh = m / (1 - self.b1 ** self.t)
            vh = v / (1 - self.b2 ** self.t)
            p -= self.lr * mh / (np.sqrt(vh) + self.eps)


def network_input(depth_mm, rgba):
    """[H, W] uint16 depth and [H, W, 4] uint8 colour -> [H, W, 4] float input channels, centred
    and scaled to about [-2, 2]."""
    x = np.zeros(depth_mm.shape + (4,), dtype=np.float64)
    x[..., 0] = (depth_mm.astype(np.float64) / 1000.0 - DEPTH_CENTRE) * DEPTH_SCALE
    x[..., 1:] = (rgba[..., :3].astype(np.float64) / 255.0 - COLOUR_CENTRE) * COLOUR_SCALE
    return x


def cell_targets(depth_mm, intr, pose, origin, cell=8):
    """Scene coordinate (minus origin) of each cell's centre pixel, and the mask of cells whose
    centre pixel has depth."""
    H, W = depth_mm.shape
    Hc, Wc = H // cell, W // cell
    v = np.arange(Hc) * cell + cell // 2
    u = np.arange(Wc) * cell + cell // 2
    uu, vv = np.meshgrid(u, v)
    d = depth_mm[vv, uu].astype(np.float64)
    z = d / 1000.0
    c = np.stack([z * (uu - intr.cx) / intr.fx, z * (vv - intr.cy) / intr.fy, z], -1)
    y = c @ pose[:3, :3].T + pose[:3, 3] - np.asarray(origin)
    return y, d > 0


def cell_view(depth_mm, intr, cell=8):
    """The coarse view RANSAC sees on the learned path: the centre pixels' depths and the
    intrinsics of that grid (fx / 8, cy' = (cy - 4) / 8, ...)."""
    H, W = depth_mm.shape
    d = depth_mm[cell // 2::cell, cell // 2::cell][: H // cell, : W // cell]
    from types import SimpleNamespace
    ci = SimpleNamespace(width=W // cell, height=H // cell, fx=intr.fx / cell, fy=intr.fy / cell,
                         cx=(intr.cx - cell // 2) / cell, cy=(intr.cy - cell // 2) / cell,
                         depth_min=intr.depth_min, depth_max=intr.depth_max)
    return np.ascontiguousarray(d), ci


def cell_forest(out, origin, valid, max_modes: int = 1):
    """One-tree 'forest' over the cell grid: leaf = cell index, one Gaussian mode per scored cell
    with mean y_hat + o and covariance exp(s) I (log weight 0), so the forest RANSAC runs
    unchanged on the regressor's output."""
    from . import Forest
    from paper_1801_08361_gb300.synth import NODE_DTYPE
    Hc, Wc = out.shape[:2]
    n = Hc * Wc
    D = max(1, int(math.ceil(math.log2(max(n, 2)))))
    L = 1 << D
    modes = np.zeros((1, L, max_modes, 12), np.float32)
    nm = np.zeros((1, L), np.uint8)
    o = out.reshape(n, 4).astype(np.float64)
    s = o[:, 3]
    modes[0, :n, 0, :3] = o[:, :3] + np.asarray(origin)
    inv = np.exp(-s)
    modes[0, :n, 0, 3] = inv
    modes[0, :n, 0, 6] = inv
    modes[0, :n, 0, 8] = inv
    modes[0, :n, 0, 9] = -1.5 * math.log(2 * math.pi) - 1.5 * s
    modes[0, :n, 0, 10] = 1.0
    nm[0, :n] = valid.reshape(n).astype(np.uint8)
    leaves = np.arange(n, dtype=np.uint16).reshape(1, Hc, Wc)
    return Forest(np.zeros((1, L - 1), dtype=NODE_DTYPE), modes, nm), leaves
