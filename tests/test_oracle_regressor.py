"""Pins of the regressor oracle: convolution against scipy's correlation, gradients against
central finite differences, Adam against its closed-form first step, and the cell geometry
against direct back-projection."""
import math

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import regressor as R
from paper_1801_08361_gb300 import synth


@pytest.mark.parametrize("stride", [1, 2])
@pytest.mark.parametrize("shape", [(9, 7), (8, 8), (5, 12)])
def test_conv_matches_scipy_correlation(stride, shape):
    rng = np.random.default_rng(0)
    H, W = shape
    x = rng.normal(size=(2, H, W, 3))
    w = rng.normal(size=(3, 3, 3, 2))
    b = rng.normal(size=2)
    y = R.conv3x3(x, w, b, stride)
    for n in range(2):
        for co in range(2):
            want = b[co] + sum(correlate2d(x[n, :, :, ci], w[:, :, ci, co], mode="same") for ci in range(3))
            assert np.allclose(y[n, :, :, co], want[::stride, ::stride], atol=1e-12)
    assert y.shape[1:3] == (R.out_size(H, stride), R.out_size(W, stride))


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(1)
    for stride in (1, 2):
        x = rng.normal(size=(2, 7, 6, 3))
        c = rng.normal(size=R.im2col(x, stride).shape)
        lhs = (R.im2col(x, stride) * c).sum()
        rhs = (x * R.col2im(c, x.shape, stride)).sum()
        assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    strides = (2, 1, 1)
    params = R.init_params(3, channels=4, in_ch=4, out_ch=4, n_layers=3)
    for p in params.b:
        p += rng.normal(0, 0.1, p.shape)                   # non-zero biases exercise their gradient
    x = rng.normal(size=(2, 8, 8, 4))
    out, _ = R.forward(params, x, strides)
    target = rng.normal(size=out.shape[:3] + (3,))
    mask = rng.random(out.shape[:3]) < 0.8

    out, acts = R.forward(params, x, strides)
    _, g = R.loss_and_grad_output(out, target, mask)
    sq_fixed = ((out[..., :3] - target) ** 2).sum(-1)

    def f():
        o, _ = R.forward(params, x, strides)
        return R.surrogate_loss(o, target, mask, sq_fixed)

    grads = R.backward(params, acts, g, strides)
    h = 1e-6
    for p, gp in zip(params.flat(), grads.flat()):
        flat, gflat = p.reshape(-1), gp.reshape(-1)
        for i in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[i]
            flat[i] = old + h
            fp = f()
            flat[i] = old - h
            fm = f()
            flat[i] = old
            num = (fp - fm) / (2 * h)
            assert abs(num - gflat[i]) <= 1e-6 * max(1.0, abs(num)) + 1e-8, (num, gflat[i])


def test_loss_closed_form():
    out = np.zeros((1, 1, 2, 4))
    out[0, 0, 0] = [1.0, 2.0, 3.0, 0.5]
    out[0, 0, 1] = [0.0, 0.0, 0.0, -1.0]
    target = np.zeros((1, 1, 2, 3))
    mask = np.array([[[True, False]]])
    loss, g = R.loss_and_grad_output(out, target, mask)
    rho = math.sqrt(14 + 1e-6)
    assert loss == pytest.approx(rho + 0.5 * 14 * math.exp(-0.5) + 0.75)
    assert np.allclose(g[0, 0, 1], 0)
    assert g[0, 0, 0, 3] == pytest.approx(-0.5 * 14 * math.exp(-0.5) + 1.5)
    assert np.allclose(g[0, 0, 0, :3], np.array([1.0, 2.0, 3.0]) / rho)


def test_coordinate_gradient_ignores_the_variance():
    """The coordinates follow the Euclidean error alone: a unit vector along the error for errors
    well above the smoothing, whatever the predicted log-variance."""
    rng = np.random.default_rng(5)
    out = rng.normal(size=(1, 3, 4, 4))
    target = out[..., :3] + rng.normal(size=(1, 3, 4, 3))
    mask = np.ones((1, 3, 4), bool)
    _, g1 = R.loss_and_grad_output(out, target, mask)
    out2 = out.copy()
    out2[..., 3] += 3.0
    _, g2 = R.loss_and_grad_output(out2, target, mask)
    assert np.allclose(g1[..., :3], g2[..., :3], atol=1e-15)
    unit = (out[..., :3] - target) / np.linalg.norm(out[..., :3] - target, axis=-1, keepdims=True) / 12
    assert np.allclose(g1[..., :3], unit, atol=1e-6)


def test_network_input_centres_and_scales():
    d = np.array([[0, 3000, 5000]], np.uint16)
    c = np.zeros((1, 3, 4), np.uint8)
    c[0, 1, :3] = 255
    c[0, 2, :3] = [0, 51, 204]
    x = R.network_input(d, c)
    assert np.allclose(x[0, :, 0], [-1.5, 0.0, 1.0])
    assert np.allclose(x[0, 0, 1:], -2.0) and np.allclose(x[0, 1, 1:], 2.0)
    assert np.allclose(x[0, 2, 1:], [-2.0, -1.2, 1.2])


def test_adam_first_step_closed_form():
    p = R.Params([np.array([1.0, -2.0, 0.0])], [np.array([0.5])])
    g = R.Params([np.array([0.3, -4.0, 0.0])], [np.array([1e-3])])
    opt = R.Adam(lr=0.01)
    opt.step(p, g)
    # first step: mhat = g, vhat = g^2, update = lr g / (|g| + eps)
    want = np.array([1.0, -2.0, 0.0]) - 0.01 * np.array([0.3, -4.0, 0.0]) / (np.abs([0.3, -4.0, 0.0]) + 1e-8)
    assert np.allclose(p.w[0], want, atol=1e-12)
    assert p.b[0][0] == pytest.approx(0.5 - 0.01 * 1e-3 / (1e-3 + 1e-8))


def test_cell_geometry():
    intr = synth.Intrinsics.for_size(64, 48)
    rng = np.random.default_rng(3)
    d = rng.integers(500, 4000, (48, 64)).astype(np.uint16)
    d[4, 12] = 0                                            # centre pixel of cell (1, 0) invalid
    P = np.eye(4)
    P[:3, 3] = [0.5, -1.0, 2.0]
    y, mask = R.cell_targets(d, intr, P, origin=(0.5, 0.0, 0.0))
    assert y.shape == (6, 8, 3) and not mask[0, 1] and mask.sum() == 47
    u, v = 8 * 3 + 4, 8 * 2 + 4
    z = d[v, u] / 1000.0
    want = np.array([z * (u - intr.cx) / intr.fx, z * (v - intr.cy) / intr.fy, z]) + [0.5, -1.0, 2.0] - [0.5, 0, 0]
    assert np.allclose(y[2, 3], want, atol=1e-12)
    # the coarse view's intrinsics back-project each cell to its centre pixel's camera point
    dl, ci = R.cell_view(d, intr)
    assert dl.shape == (6, 8) and dl[2, 3] == d[v, u]
    zc = dl[2, 3] / 1000.0
    assert np.allclose([zc * (3 - ci.cx) / ci.fx, zc * (2 - ci.cy) / ci.fy],
                       [z * (u - intr.cx) / intr.fx, z * (v - intr.cy) / intr.fy], atol=1e-12)
