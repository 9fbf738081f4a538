"""Planted mistakes: each test swaps one oracle function for a copy with one plausible error (a
dropped term, a wrong sign, a transposed operand, an off-by-one comparison) and checks that one of
the oracle's pins then fails.  The mistakes live only here, on the CPU, for the length of a test
(monkeypatch restores the oracle); they show that the pins can tell a wrong oracle from a right one."""
import dataclasses

import numpy as np
import pytest

import oracle
import oracle.posegraph as PG
from oracle import regressor as R

import test_oracle_forest_verify as pins_verify
import test_oracle_posegraph as pins_pg
import test_oracle_render_global as pins_global
import test_oracle_ransac as pins_ransac
import test_oracle_regressor as pins_reg


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# -- Kabsch ----------------------------------------------------------------------------------------

def test_kabsch_without_the_reflection_fix(monkeypatch):
    def kabsch(c, w):
        c, w = np.asarray(c, np.float64), np.asarray(w, np.float64)
        cb, wb = c.mean(0), w.mean(0)
        U, _, Vt = np.linalg.svd((c - cb).T @ (w - wb))
        Rm = Vt.T @ U.T                       # mistake: det(R) may be -1
        return Rm, wb - Rm @ cb
    monkeypatch.setattr(oracle, "kabsch", kabsch)
    _fails(pins_ransac.test_kabsch_returns_proper_rotation_for_mirrored_points)


def test_kabsch_with_a_transposed_rotation(monkeypatch):
    right = oracle.kabsch

    def kabsch(c, w):
        Rm, _ = right(c, w)
        c, w = np.asarray(c, np.float64), np.asarray(w, np.float64)
        return Rm.T, w.mean(0) - Rm.T @ c.mean(0)   # mistake: R^T for R
    monkeypatch.setattr(oracle, "kabsch", kabsch)
    _fails(pins_ransac.test_kabsch_recovers_known_transform)


# -- pixel energy ----------------------------------------------------------------------------------

def test_energy_without_the_covariance_cross_terms(monkeypatch):
    right = oracle.pixel_energies

    def pixel_energies(pose, cam, pix, leaves, forest):
        modes = forest.modes.copy()
        modes[..., [4, 5, 7]] = 0.0           # mistake: the off-diagonal inverse-covariance terms dropped
        return right(pose, cam, pix, leaves, dataclasses.replace(forest, modes=modes))
    monkeypatch.setattr(oracle, "pixel_energies", pixel_energies)
    _fails(pins_ransac.test_pixel_energy_matches_gaussian_density)


def test_energy_with_the_wrong_floor(monkeypatch):
    monkeypatch.setattr(oracle, "LOG_EPS", -np.log(1e-20))     # mistake: a density floor of 1e-20
    _fails(pins_ransac.test_pixel_energy_single_isotropic_gaussian_closed_form)


def test_distance_without_its_z_term(monkeypatch):
    def dist(a, b):
        return np.sqrt((a[..., 0] - b[..., 0]) ** 2 + (a[..., 1] - b[..., 1]) ** 2)   # mistake: no z term
    monkeypatch.setattr(oracle, "_dist", dist)
    _fails(pins_ransac.test_first_passing_try_is_the_first_triple_of_distinct_inliers)


def test_uniform_draw_by_modulo(monkeypatch):
    monkeypatch.setattr(oracle, "uniform_below",                   # mistake: x mod n for floor(x n / 2^32)
                        lambda x, n: (np.asarray(x, np.uint64) % np.asarray(n, np.uint64)).astype(np.int64))
    _fails(pins_ransac.test_hypotheses_use_first_passing_try)


def test_camera_points_with_swapped_principal_point(monkeypatch):
    def camera_points(depth_img, intr, pixels):
        W = intr.width
        pixels = np.asarray(pixels, dtype=np.int64)
        u = (pixels % W).astype(np.float64)
        v = (pixels // W).astype(np.float64)
        z = depth_img.reshape(-1)[pixels].astype(np.float64) / 1000.0
        return np.stack([z * (u - intr.cy) / intr.fx, z * (v - intr.cx) / intr.fy, z], axis=-1)   # mistake
    monkeypatch.setattr(oracle, "camera_points", camera_points)
    _fails(pins_ransac.test_camera_points_project_back_to_their_pixels)


# -- verification ----------------------------------------------------------------------------------

def test_verification_accepting_half_valid(monkeypatch):
    def verify_accept(counts, valid_fraction=0.5, max_mean_mm=50):
        n, oa, _, oab, s = (int(x) for x in counts)
        if not oa >= valid_fraction * n:     # mistake: >= where the paper's test is strict
            return False
        return oab > 0 and s < max_mean_mm * oab
    monkeypatch.setattr(oracle, "verify_accept", verify_accept)
    _fails(pins_verify.test_verification_decision_rules)


def test_verification_with_an_inclusive_mean_bound(monkeypatch):
    def verify_accept(counts, valid_fraction=0.5, max_mean_mm=50):
        n, oa, _, oab, s = (int(x) for x in counts)
        if not oa > valid_fraction * n:
            return False
        return oab > 0 and s <= max_mean_mm * oab   # mistake: mean <= 5 cm accepted
    monkeypatch.setattr(oracle, "verify_accept", verify_accept)
    _fails(pins_verify.test_verification_decision_rules)


# -- pose graph ------------------------------------------------------------------------------------

def test_blend_without_quaternion_sign_alignment(monkeypatch):
    def dq_blend(samples):
        real, dual = np.zeros(4), np.zeros(4)
        for T in samples:
            q = PG.quat_wxyz(T[:3, :3])      # mistake: q and -q not brought to one hemisphere
            real += q
            dual += 0.5 * PG.qmul(np.concatenate([[0.0], T[:3, 3]]), q)
        n = np.linalg.norm(real)
        real, dual = real / n, dual / n
        out = np.eye(4)
        w, x, y, z = real
        from scipy.spatial.transform import Rotation
        out[:3, :3] = Rotation.from_quat([x, y, z, w]).as_matrix()
        out[:3, 3] = 2.0 * PG.qmul(dual, real * np.array([1, -1, -1, -1]))[1:]
        return out
    monkeypatch.setattr(PG, "dq_blend", dq_blend)
    _fails(pins_pg.test_blend_aligns_quaternion_signs)


def test_quaternion_product_with_a_flipped_cross_term(monkeypatch):
    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 - y1 * z2 + z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    monkeypatch.setattr(PG, "qmul", qmul)   # mistake: y1 z2 - z1 y2 with the wrong sign
    _fails(pins_pg.test_blend_of_opposite_rotations_about_an_offset_axis_is_the_identity)


def test_clustering_with_a_tighter_rotation_threshold(monkeypatch):
    monkeypatch.setattr(PG, "CLUSTER_DEG", 10.0)                 # mistake: 10 degrees for 20
    _fails(pins_pg.test_clustering_thresholds_and_chains)


def test_clustering_with_a_looser_translation_threshold(monkeypatch):
    monkeypatch.setattr(PG, "CLUSTER_M", 0.2)                    # mistake: 20 cm for 10 cm
    _fails(pins_pg.test_clustering_thresholds_and_chains)


def test_candidate_score_with_the_wrong_penalty(monkeypatch):
    monkeypatch.setattr(PG, "HOMOG_PENALTY", 1.0)                # mistake: a penalty of 1 for 5
    _fails(pins_pg.test_phi_terms)


def test_halving_that_keeps_the_floor(monkeypatch):
    import math
    import types
    monkeypatch.setattr(oracle, "math", types.SimpleNamespace(**{**vars(math), "ceil": math.floor}))   # mistake
    _fails(pins_ransac.test_halving_keeps_the_ceiling_of_half)


# -- regressor -------------------------------------------------------------------------------------

def test_convolution_instead_of_correlation(monkeypatch):
    right = R.conv3x3
    monkeypatch.setattr(R, "conv3x3", lambda x, w, b, stride: right(x, w[::-1, ::-1], b, stride))
    _fails(pins_reg.test_conv_matches_scipy_correlation, 1, (9, 7))


def test_loss_gradient_that_ignores_the_mask(monkeypatch):
    def loss_and_grad_output(out, target, mask):
        n = max(int(mask.sum()), 1)
        s = out[..., 3]
        err = out[..., :3] - target
        sq = (err * err).sum(-1)
        rho = np.sqrt(sq + R.RHO_EPS2)
        e = np.exp(-s)
        loss = float(((rho + 0.5 * sq * e + 1.5 * s) * mask).sum() / n)
        g = np.zeros_like(out)
        g[..., :3] = err / (n * rho)[..., None]        # mistake: unscored cells get a gradient
        g[..., 3] = (-0.5 * sq * e + 1.5) * mask / n
        return loss, g
    monkeypatch.setattr(R, "loss_and_grad_output", loss_and_grad_output)
    _fails(pins_reg.test_gradients_match_central_differences)


def test_variance_term_that_pulls_the_coordinates(monkeypatch):
    def loss_and_grad_output(out, target, mask):
        n = max(int(mask.sum()), 1)
        s = out[..., 3]
        err = out[..., :3] - target
        sq = (err * err).sum(-1)
        rho = np.sqrt(sq + R.RHO_EPS2)
        e = np.exp(-s)
        loss = float(((rho + 0.5 * sq * e + 1.5 * s) * mask).sum() / n)
        g = np.zeros_like(out)
        g[..., :3] = err * (mask * (1.0 / rho + e) / n)[..., None]    # mistake: the NLL's pull on y_hat kept
        g[..., 3] = (-0.5 * sq * e + 1.5) * mask / n
        return loss, g
    monkeypatch.setattr(R, "loss_and_grad_output", loss_and_grad_output)
    _fails(pins_reg.test_coordinate_gradient_ignores_the_variance)


def test_network_input_without_its_centring(monkeypatch):
    monkeypatch.setattr(R, "DEPTH_CENTRE", 0.0)                    # mistake: depth not centred
    _fails(pins_reg.test_network_input_centres_and_scales)


def test_adam_without_bias_correction(monkeypatch):
    def step(self, params, grads):
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
            p -= self.lr * m / (np.sqrt(v) + self.eps)    # mistake: raw moments
    monkeypatch.setattr(R.Adam, "step", step)
    _fails(pins_reg.test_adam_first_step_closed_form)


def test_backward_data_that_drops_a_stride_offset(monkeypatch):
    right = R.col2im

    def col2im(cols, shape, stride):
        g = right(cols, shape, stride)
        return np.roll(g, 1, axis=1)           # mistake: the input gradient lands one row off
    monkeypatch.setattr(R, "col2im", col2im)
    _fails(pins_reg.test_gradients_match_central_differences)


def test_global_render_where_the_farther_surface_wins(monkeypatch):
    right = oracle.render_global

    class Reversed:
        def __init__(self, sc):
            self.sc = sc

        def raycast(self, intr, pose, pixels=None):
            d, c = self.sc.raycast(intr, pose, pixels=pixels)
            return np.where(d > 0, 65535 - d, 0).astype(np.uint16), c

    def render_global(scenes, global_poses, intr, pose_global, pixels=None):
        # mistake: the per-pixel depth test keeps the farthest hit
        d, c, o, ds = right([Reversed(sc) for sc in scenes], global_poses, intr, pose_global, pixels)
        back = lambda x: np.where(x > 0, 65535 - x.astype(np.int64), 0).astype(np.uint16)   # noqa: E731
        return back(d), c, o, back(ds)
    monkeypatch.setattr(oracle, "render_global", render_global)
    _fails(pins_global.test_depth_test_against_a_brute_force_loop)


def test_vee_with_the_quaternion_sign_left_free(monkeypatch):
    monkeypatch.setattr(PG, "vee", lambda T: np.concatenate([-PG.quat_wxyz(T[:3, :3])[1:], T[:3, 3]]))   # mistake
    _fails(pins_pg.test_vee_takes_the_quaternion_with_nonnegative_w, 30.0)


# -- the C part of the oracle ----------------------------------------------------------------------
# Each case compiles a copy of relo_oracle.c with one edit into a temporary library, points the
# oracle at it for the test, and runs a pin that must then fail.

import ctypes                                    # noqa: E402
import os                                        # noqa: E402
import subprocess                                # noqa: E402

import test_oracle_fusion as pins_fusion        # noqa: E402
import test_oracle_leaves as pins_leaves        # noqa: E402
import test_oracle_philox as pins_philox        # noqa: E402
import test_oracle_scene as pins_scene          # noqa: E402

C_SOURCE = os.path.join(os.path.dirname(oracle.__file__), "relo_oracle.c")

C_MUTATIONS = [
    # (name, original text, mistaken text, pin that must fail)
    ("trilinear corner by truncation", "base[a] = (long)floor(q[a]);", "base[a] = (long)q[a];",
     pins_scene.test_shift_by_whole_blocks_into_negative_coordinates),
    ("secant root with a wrong sign", "f_prev / (f_prev - f);", "f_prev / (f_prev + f);",
     pins_scene.test_plane_depth_exact_to_rounding),
    ("depth rounded down", "double zr = round_half_up(z_mm);", "double zr = floor(z_mm);",
     pins_scene.test_plane_depth_exact_to_rounding),
    ("colour channel off by one", "rgb[c] = (double)s->rgba[(b * 512 + li) * 4 + c];",
     "rgb[c] = (double)s->rgba[(b * 512 + li) * 4 + (c + 1) % 3];", pins_scene.test_linear_colour_is_reproduced),
    ("forest children swapped", "? 2 * n + 1 : 2 * n + 2;", "? 2 * n + 2 : 2 * n + 1;",
     pins_verify.test_depth_split_by_hand),
    ("forest split not strict", "n = (a - b < nd->tau)", "n = (a - b <= nd->tau)",
     pins_verify.test_offset_truncates_toward_zero_and_invalid_probe_reads_zero),
    ("forest offset rounded down", "int q1x = clampi(u + (int)(((int32_t)nd->dx1 * 1000) / d), 0, W - 1);",
     "int q1x = clampi(u + (int)floor(((double)nd->dx1 * 1000) / d), 0, W - 1);",
     pins_verify.test_offset_truncates_toward_zero_and_invalid_probe_reads_zero),
    ("verification difference one-sided", "sum += (uint64_t)(da[i] > db[i] ? da[i] - db[i] : db[i] - da[i]);",
     "sum += (uint64_t)(da[i] > db[i] ? da[i] - db[i] : 0);", pins_verify.test_verification_counts_by_hand),
    ("Philox key schedule", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE87u;", pins_philox.test_known_answer_vectors),
    ("reservoir draw over [0, n)", "uint64_t j = ((uint64_t)o[0] * (uint64_t)(n + 1)) >> 32;",
     "uint64_t j = ((uint64_t)o[0] * (uint64_t)n) >> 32;",
     pins_leaves.test_reservoir_of_one_keeps_the_second_of_two_samples_half_the_time),
    ("mode weight over n + 1 samples", "double weight = (double)cnt / n;", "double weight = (double)cnt / (n + 1);",
     pins_leaves.test_mean_shift_recovers_blob_centres_and_weights),
    ("fusion without the truncation clamp", "const float fn = fminf(1.0f, eta / mu);", "const float fn = eta / mu;",
     pins_fusion.test_plane_closed_form),
    ("free-space restart 3 cm past the block exit", "lam = lam_prev + 1e-5;", "lam = lam_prev + 3e-2;",
     pins_scene.test_sphere_depth_within_interpolation_bound),
    ("mean-shift kernel twice as narrow", "double k = exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * h * h));",
     "double k = exp(-(dx * dx + dy * dy + dz * dz) / (h * h));",
     pins_leaves.test_mean_shift_bandwidth_decides_when_two_clusters_merge),
    ("fusion colour rounded down", "float r = floorf(cc + 0.5f);", "float r = floorf(cc);",
     pins_fusion.test_colour_average_rounds_half_up),
    ("fusion weight without its cap",
     "f->weight[at] = (uint16_t)(f->weight[at] + 1 < f->max_weight ? f->weight[at] + 1 : f->max_weight);",
     "f->weight[at] = (uint16_t)(f->weight[at] + 1);",
     pins_fusion.test_equal_frames_average_to_themselves_and_weights_stop_at_the_cap),
]


@pytest.mark.parametrize("name,right,wrong,pin", C_MUTATIONS, ids=[m[0] for m in C_MUTATIONS])
def test_c_oracle_mistake_is_caught(name, right, wrong, pin, tmp_path, monkeypatch):
    src = open(C_SOURCE).read()
    assert src.count(right) == 1, name
    c_file = tmp_path / "mutant.c"
    c_file.write_text(src.replace(right, wrong))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", str(c_file), "-o",
                           str(so), "-lm"])
    monkeypatch.setattr(oracle, "_LIB", oracle.declare(ctypes.CDLL(str(so))))
    _fails(pin)
