"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/scan_work.json), closed forms, invariants, library
routines (numpy's corrcoef), brute-force search and exactness properties of
the two image models (bilinear interpolation; the quadratic B-spline model of
the nonrigid energy).  A dropped term, a wrong sign, a transposed operand or
a wrong index in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2010_12478_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "scan_work.json")


def rand_img(H, W, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(H, W))


# ---------------------------------------------------------------- pyramid
def test_downsample_by_hand_with_odd_clamp():
    a = np.arange(15, dtype=np.float64).reshape(3, 5)       # rows 0..2, cols 0..4
    d = O.downsample(a)
    assert d.shape == (2, 3)
    # (0,0): rows 0-1, cols 0-1 ; (0,2): cols 4,4 (clamped) ; (1,*): rows 2,2 (clamped)
    exp = np.array([[(0 + 1 + 5 + 6) / 4, (2 + 3 + 7 + 8) / 4, (4 + 4 + 9 + 9) / 4],
                    [(10 + 11 + 10 + 11) / 4, (12 + 13 + 12 + 13) / 4, (14 + 14 + 14 + 14) / 4]])
    np.testing.assert_array_equal(d, exp)


def test_pyramid_of_linear_ramp_is_centre_consistent():
    # f(x, y) = 3x - 2y + 1 on an even grid: the box average of level l sits at
    # x_l = 2 x_{l+1} + 0.5, i.e. level l+1 equals f(2x + 0.5, 2y + 0.5).
    H, W = 16, 24
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    p = O.pyramid(3 * x - 2 * y + 1, 3)
    y1, x1 = np.mgrid[0:H // 2, 0:W // 2].astype(np.float64)
    np.testing.assert_allclose(p[1], 3 * (2 * x1 + 0.5) - 2 * (2 * y1 + 0.5) + 1, atol=1e-12)
    y2, x2 = np.mgrid[0:H // 4, 0:W // 4].astype(np.float64)
    np.testing.assert_allclose(p[2], 3 * (4 * x2 + 1.5) - 2 * (4 * y2 + 1.5) + 1, atol=1e-12)


# ---------------------------------------------------------------- sampling
def test_sample_exact_at_pixels_and_on_bilinear_functions():
    H, W = 7, 9
    T = rand_img(H, W, 1)
    for r in range(H):
        for c in range(W):
            assert O.sample(T, c, r)[0] == T[r, c]
    # bilinear interpolation reproduces span{1, x, y, xy} exactly, with exact derivatives
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    F = 0.5 + 2.0 * x - 3.0 * y + 0.25 * x * y
    rng = np.random.default_rng(2)
    for _ in range(50):
        px, py = rng.uniform(0, W - 1), rng.uniform(0, H - 1)
        v, dx, dy = O.sample(F, px, py)
        assert v == pytest.approx(0.5 + 2 * px - 3 * py + 0.25 * px * py, abs=1e-12)
        assert dx == pytest.approx(2.0 + 0.25 * py, abs=1e-12)
        assert dy == pytest.approx(-3.0 + 0.25 * px, abs=1e-12)


def test_sample_clamps_to_edge_with_zero_derivative_along_clamped_axis():
    H, W = 5, 6
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    F = 1.0 + x + 10.0 * y
    v, dx, dy = O.sample(F, -3.0, 2.5)          # x clamped to 0
    assert (v, dx, dy) == (pytest.approx(1 + 25.0), 0.0, pytest.approx(10.0))
    v, dx, dy = O.sample(F, 2.25, H + 4.0)      # y clamped to H-1
    assert (v, dx, dy) == (pytest.approx(1 + 2.25 + 40.0), pytest.approx(1.0), 0.0)
    v, dx, dy = O.sample(F, W - 1.0, H - 1.0)   # exactly on the last pixel: not clamped
    assert v == F[-1, -1] and dx == pytest.approx(1.0) and dy == pytest.approx(10.0)


# ---------------------------------------------------------------- NCC energy
def smooth_1_8_3_4_1_8(img, outside=None):
    """The separable filter (1/8, 3/4, 1/8), samples beyond the frame equal to ``outside`` (default
    the frame's mean) (numpy, by hand)."""
    p = np.pad(img, 1, mode="constant", constant_values=img.mean() if outside is None else outside)
    rows = 0.125 * p[:-2, :] + 0.75 * p[1:-1, :] + 0.125 * p[2:, :]
    return 0.125 * rows[:, :-2] + 0.75 * rows[:, 1:-1] + 0.125 * rows[:, 2:]


def test_ncc_energy_equals_corrcoef_at_identity():
    R, T = rand_img(12, 10, 3), rand_img(12, 10, 4)
    E = O.rigid_energy(R, T, [0.0, 0.0, 0.0], grad=False)
    assert E == pytest.approx(1.0 - np.corrcoef(R.ravel(), T.ravel())[0, 1], abs=1e-13)
    # the nonrigid energy takes both frames through the B-spline model: at the zero field that is
    # the correlation of the two filtered frames
    g = O.grid_for(10, 12, 4)
    Eg = O.grid_energy(R, T, 0, g, np.zeros((2, g.ny, g.nx)), 5.0, grad=False)
    Rf, Tf = smooth_1_8_3_4_1_8(R), smooth_1_8_3_4_1_8(T)
    assert Eg == pytest.approx(1.0 - np.corrcoef(Rf.ravel(), Tf.ravel())[0, 1], abs=1e-13)


# ---------------------------------------------------------------- quadratic B-spline image model
def test_bspline_model_at_pixel_centres_is_the_filter_and_central_difference():
    T = rand_img(9, 11, 81)
    Tf = smooth_1_8_3_4_1_8(T, outside=0.37)
    p = np.pad(T, 1, mode="constant", constant_values=0.37)
    # d/dx at a centre: central difference along x, filtered (1/8, 3/4, 1/8) along y; and vice versa
    cx = 0.5 * (p[:, 2:] - p[:, :-2])
    dx = 0.125 * cx[:-2, :] + 0.75 * cx[1:-1, :] + 0.125 * cx[2:, :]
    cy = 0.5 * (p[2:, :] - p[:-2, :])
    dy = 0.125 * cy[:, :-2] + 0.75 * cy[:, 1:-1] + 0.125 * cy[:, 2:]
    for r in range(9):
        for c in range(11):
            v, gx, gy = O.sample_q(T, float(c), float(r), outside=0.37)
            assert v == pytest.approx(Tf[r, c], abs=1e-15)
            assert gx == pytest.approx(dx[r, c], abs=1e-15) and gy == pytest.approx(dy[r, c], abs=1e-15)


def test_bspline_model_reproduces_affine_images():
    H, W = 12, 15
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    T = 0.3 + 0.7 * x - 0.45 * y
    rng = np.random.default_rng(82)
    for px, py in rng.uniform(1.5, [W - 2.5, H - 2.5], size=(20, 2)):
        v, gx, gy = O.sample_q(T, px, py)
        assert v == pytest.approx(0.3 + 0.7 * px - 0.45 * py, abs=1e-13)
        assert gx == pytest.approx(0.7, abs=1e-13) and gy == pytest.approx(-0.45, abs=1e-13)
    # a constant image stays constant with zero derivative anywhere, inside or outside
    for px, py in ((-7.3, 2.2), (3.4, 40.0), (5.5, 5.5)):
        v, gx, gy = O.sample_q(np.full((6, 7), 0.25), px, py)
        assert v == pytest.approx(0.25, abs=1e-15) and abs(gx) <= 1e-15 and abs(gy) <= 1e-15


def test_bspline_model_is_continuously_differentiable():
    # value and derivatives agree on both sides of a knot (half-integer), where the tap set changes
    T = rand_img(10, 10, 83)
    e = 1e-9
    for px, py in ((3.5, 4.2), (6.1, 2.5), (0.5, 0.5), (-0.5, 7.3), (9.5, 9.5)):
        for dx, dy in ((e, 0.0), (0.0, e)):
            a = O.sample_q(T, px - dx, py - dy)
            b = O.sample_q(T, px + dx, py + dy)
            np.testing.assert_allclose(a, b, atol=1e-8)


def test_bspline_model_takes_the_outside_value_beyond_the_frame():
    T = rand_img(7, 8, 84)
    out = 0.42
    # far outside every tap is the outside value: the model is that constant, with zero derivative
    for px, py in ((-6.0, 3.0), (100.0, 100.0), (3.2, -4.0)):
        v, gx, gy = O.sample_q(T, px, py, outside=out)
        assert v == pytest.approx(out, abs=1e-15) and abs(gx) <= 1e-15 and abs(gy) <= 1e-15
    # at x = -1 (a pixel centre outside) the x taps are -2, -1 (outside) and 0 (column 0), weights
    # 1/8, 3/4, 1/8; at y = 3 the y taps are rows 2, 3, 4 with the same weights
    v, gx, gy = O.sample_q(T, -1.0, 3.0, outside=out)
    col = 0.125 * T[2, 0] + 0.75 * T[3, 0] + 0.125 * T[4, 0]
    assert v == pytest.approx(0.875 * out + 0.125 * col, abs=1e-15)
    assert gx == pytest.approx(0.5 * (col - out), abs=1e-15)


def test_bspline_derivative_matches_central_differences():
    T = rand_img(16, 16, 85)
    h = 1e-6
    for px, py in np.random.default_rng(86).uniform(-1.0, 16.0, size=(25, 2)):
        v, gx, gy = O.sample_q(T, px, py)
        fx = (O.sample_q(T, px + h, py)[0] - O.sample_q(T, px - h, py)[0]) / (2 * h)
        fy = (O.sample_q(T, px, py + h)[0] - O.sample_q(T, px, py - h)[0]) / (2 * h)
        assert gx == pytest.approx(fx, abs=1e-7) and gy == pytest.approx(fy, abs=1e-7)


def test_image_models_equal_scipy_spline_evaluation():
    # an independent implementation of both image models: scipy.ndimage evaluates a B-spline of
    # order 2 with the samples as its coefficients (prefilter=False) and the constant beyond the
    # frame ("grid-constant"), and bilinear interpolation with the edge replicated ("nearest"), at
    # positions inside the frame, on its border and well outside it
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(87)
    T = rng.uniform(0.0, 1.0, (9, 12))
    out = 0.37
    h = 1e-6

    def q(x, y):
        return nd.map_coordinates(T, [[y], [x]], order=2, prefilter=False, mode="grid-constant", cval=out)[0]

    for px, py in rng.uniform([-4.0, -4.0], [15.0, 12.0], size=(200, 2)):
        v, gx, gy = O.sample_q(T, float(px), float(py), outside=out)
        assert v == pytest.approx(q(px, py), abs=1e-14)
        assert gx == pytest.approx((q(px + h, py) - q(px - h, py)) / (2 * h), abs=1e-8)
        assert gy == pytest.approx((q(px, py + h) - q(px, py - h)) / (2 * h), abs=1e-8)
        b = nd.map_coordinates(T, [[py], [px]], order=1, mode="nearest")[0]
        assert O.sample(T, float(px), float(py))[0] == pytest.approx(b, abs=1e-14)


def test_ncc_by_hand_on_2x2():
    R = np.array([[0.0, 1.0], [2.0, 3.0]])
    T = np.array([[1.0, 0.0], [3.0, 2.0]])
    # centred: r = (-1.5, -0.5, 0.5, 1.5), t = (-0.5, -1.5, 1.5, 0.5); r.t = 0.75+0.75+0.75+0.75 = 3
    # |r|^2 = |t|^2 = 5  ->  NCC = 3/5
    assert O.rigid_energy(R, T, [0, 0, 0], grad=False) == pytest.approx(1.0 - 0.6, abs=1e-15)


def test_ncc_invariances_and_self_match():
    R, T = rand_img(16, 16, 5), rand_img(16, 16, 6)
    th = [0.02, 0.3, -0.4]
    E = O.rigid_energy(R, T, th, grad=False)
    assert O.rigid_energy(R, 3.0 * T + 7.0, th, grad=False) == pytest.approx(E, abs=1e-12)
    assert O.rigid_energy(0.5 * R - 2.0, T, th, grad=False) == pytest.approx(E, abs=1e-12)
    assert O.rigid_energy(R, R, [0, 0, 0], grad=False) == 0.0
    assert O.rigid_energy(R, -R, [0, 0, 0], grad=False) == pytest.approx(2.0, abs=1e-13)


def test_constant_image_is_degenerate():
    R = np.full((8, 8), 0.3)
    E, g = O.rigid_energy(R, rand_img(8, 8, 7), [0, 0.1, 0.2])
    assert E == 1.0 and not g.any()


# ---------------------------------------------------------------- gradients
def test_rigid_gradient_matches_central_differences():
    R, T = synth.rigid_pair(48, 40, 0.01, (0.6, -0.9), noise_snr=8.0, seed=11)
    th = np.array([0.013, 0.37, -0.61])
    E, g = O.rigid_energy(R, T, th)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3); e[k] = h
        fd = (O.rigid_energy(R, T, th + e, grad=False) - O.rigid_energy(R, T, th - e, grad=False)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


@pytest.mark.parametrize("level", [0, 1])
def test_grid_gradient_matches_central_differences(level):
    R0, T0 = synth.translated_pair(40, 36, (0.4, -0.3), noise_snr=8.0, seed=12)
    pr, pt = O.pyramid(R0, 2), O.pyramid(T0, 2)
    R, T = pr[level], pt[level]
    g = O.grid_for(36, 40, 8)
    rng = np.random.default_rng(13)
    c = rng.uniform(-0.4, 0.4, size=(2, g.ny, g.nx)) + np.array([0.3, -0.2])[:, None, None]
    lam = 3.0
    E, gr = O.grid_energy(R, T, level, g, c, lam)
    h = 1e-6
    for (cmp, jy, jx) in [(0, 0, 0), (1, 2, 3), (0, g.ny - 1, g.nx - 1), (1, 0, g.nx - 1), (0, 3, 1)]:
        cp, cm = c.copy(), c.copy()
        cp[cmp, jy, jx] += h; cm[cmp, jy, jx] -= h
        fd = (O.grid_energy(R, T, level, g, cp, lam, grad=False) - O.grid_energy(R, T, level, g, cm, lam, grad=False)) / (2 * h)
        assert gr[cmp, jy, jx] == pytest.approx(fd, rel=1e-5, abs=1e-10), (cmp, jy, jx)


def test_grid_regulariser_closed_form_on_ramp():
    # c_x = a * jx, c_y = b * jy: every horizontal edge of c_x differs by a, every vertical edge of c_y by b
    g = O.grid_for(57, 41, 8)
    a, b, lam, P = 0.3, -0.7, 2.5, 57 * 41
    jy, jx = np.mgrid[0:g.ny, 0:g.nx].astype(np.float64)
    c = np.stack([a * jx, b * jy])
    exp = 0.5 * lam / P * (a * a * (g.nx - 1) * g.ny + b * b * (g.ny - 1) * g.nx)
    assert O.grid_regulariser(g, c, lam, P) == pytest.approx(exp, rel=1e-14)


def test_grid_field_interpolates_control_points_and_affine_fields():
    g = O.grid_for(50, 34, 8)           # points at 0, 8, .., 56 > 49: the last cell extends past the frame
    rng = np.random.default_rng(14)
    c = rng.uniform(-1, 1, size=(2, g.ny, g.nx))
    u = O.grid_dense(g, c)
    for jy in range(g.ny):
        for jx in range(g.nx):
            if jy * 8 < 34 and jx * 8 < 50:
                np.testing.assert_allclose(u[:, jy * 8, jx * 8], c[:, jy, jx], atol=1e-14)
    # affine field u(X) = A X + b is reproduced exactly, at level 0 and at level 1 where pixel x sits at
    # X = 2x + 1/2 and the level's values are halved
    A = np.array([[0.01, -0.02], [0.03, 0.005]]); bb = np.array([0.7, -1.1])
    jy, jx = np.mgrid[0:g.ny, 0:g.nx].astype(np.float64)
    ca = np.stack([A[0, 0] * 8 * jx + A[0, 1] * 8 * jy + bb[0], A[1, 0] * 8 * jx + A[1, 1] * 8 * jy + bb[1]])
    Y, X = np.mgrid[0:34, 0:50].astype(np.float64)
    np.testing.assert_allclose(O.grid_dense(g, ca), np.stack([A[0, 0] * X + A[0, 1] * Y + bb[0],
                                                              A[1, 0] * X + A[1, 1] * Y + bb[1]]), atol=1e-12)
    y1, x1 = np.mgrid[0:17, 0:25].astype(np.float64)
    X1, Y1 = 2 * x1 + 0.5, 2 * y1 + 0.5
    lvl = O.grid_level_dense(g, ca / 2, 1, 17, 25)
    np.testing.assert_allclose(lvl, 0.5 * np.stack([A[0, 0] * X1 + A[0, 1] * Y1 + bb[0],
                                                    A[1, 0] * X1 + A[1, 1] * Y1 + bb[1]]), atol=1e-12)


def test_grid_field_equals_scipy_linear_grid_interpolation():
    # the dense field of random control values against scipy's piecewise-linear interpolation on
    # the same grid of points (0, s, 2 s, ...) along each axis, including grids whose last cell
    # extends past the frame and a spacing that is not a power of two
    interp = pytest.importorskip("scipy.interpolate")
    for W, H, sp in ((50, 34, 8), (128, 96, 16), (37, 41, 5)):
        g = O.grid_for(W, H, sp)
        c = np.random.default_rng(15).uniform(-1.0, 1.0, size=(2, g.ny, g.nx))
        u = O.grid_dense(g, c)
        Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
        pts = np.stack([Y.ravel(), X.ravel()], 1)
        for k in range(2):
            f = interp.RegularGridInterpolator((np.arange(g.ny) * g.s, np.arange(g.nx) * g.s), c[k], method="linear")
            np.testing.assert_allclose(u[k], f(pts).reshape(H, W), atol=1e-14)


def test_grid_composition_equals_scipy_interpolation_at_the_displaced_points():
    # B's initial guess (Sec. 2.3.2) on the control grid: c_j = c1_j + u2(X_j + c1_j), with u2
    # evaluated by scipy's piecewise-linear grid interpolation of c2, for random fields whose
    # displaced control points stay on the grid
    interp = pytest.importorskip("scipy.interpolate")
    g = O.grid_for(128, 96, 16)
    rng = np.random.default_rng(16)
    c1 = rng.uniform(-3.0, 3.0, size=(2, g.ny, g.nx))
    c2 = rng.uniform(-3.0, 3.0, size=(2, g.ny, g.nx))
    jy, jx = np.mgrid[0:g.ny, 0:g.nx].astype(np.float64)
    Xj, Yj = jx * g.s, jy * g.s
    c1[0] = np.clip(c1[0], -Xj, (g.nx - 1) * g.s - Xj)
    c1[1] = np.clip(c1[1], -Yj, (g.ny - 1) * g.s - Yj)
    got = O.compose_grid(g, c1, c2)
    pts = np.stack([(Yj + c1[1]).ravel(), (Xj + c1[0]).ravel()], 1)
    for k in range(2):
        f = interp.RegularGridInterpolator((np.arange(g.ny) * g.s, np.arange(g.nx) * g.s), c2[k], method="linear")
        np.testing.assert_allclose(got[k], c1[k] + f(pts).reshape(g.ny, g.nx), atol=1e-13)


# ---------------------------------------------------------------- identical frames
@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_identical_frames_give_exact_identity(mode):
    R, _ = synth.translated_pair(64, 64, (0, 0), noise_snr=10.0, seed=21)
    cfg = O.Config(levels=2, mode=mode)
    p = O.pyramid(R, 2)
    phi, st = O.register(p, p, O.identity(mode, 64, 64), cfg)
    assert not np.any(phi)
    assert st.iters == [0, 0] and st.energy == 0.0


# ---------------------------------------------------------------- known shifts
@pytest.mark.parametrize("seed", range(6))
def test_recovers_known_translation(seed):
    rng = np.random.default_rng(100 + seed)
    s = rng.uniform(-3.4, 3.4, size=2)
    R, T = synth.translated_pair(96, 96, s, seed=seed, noise_snr=None if seed % 2 else 10.0)
    th, st = O.register_rigid(O.pyramid(R, 2), O.pyramid(T, 2), np.zeros(3), O.Config(levels=2))
    assert abs(th[1] - s[0]) <= 0.05 and abs(th[2] - s[1]) <= 0.05, (th, s)
    assert abs(th[0]) <= 1e-3


@pytest.mark.parametrize("alpha", [0.01, -0.015])
def test_recovers_known_rotation(alpha):
    R, T = synth.rigid_pair(128, 128, alpha, (1.2, -0.7), noise_snr=None, seed=5)
    th, _ = O.register_rigid(O.pyramid(R, 2), O.pyramid(T, 2), np.zeros(3), O.Config(levels=2))
    assert abs(th[0] - alpha) <= 1e-4
    assert abs(th[1] - 1.2) <= 0.05 and abs(th[2] + 0.7) <= 0.05


def test_nonrigid_recovers_smooth_field():
    ser = synth.make_series(synth.SeriesSpec(2, 96, 96, step=2.0, field_amp=1.0, snr=(10, 10),
                                             field_rate=(0.8, 1.2), seed=31))
    F = ser.frames.numpy()
    cfg = O.Config(levels=2, mode="nonrigid")
    c, st = O.register_nonrigid(O.pyramid(F[0], 2), O.pyramid(F[1], 2), None, cfg)
    u = O.grid_dense(O.grid_for(96, 96), c)
    err = (u - ser.truth_field(1))[:, 12:-12, 12:-12]
    assert np.sqrt((err ** 2).sum(0).mean()) <= 0.1
    # and the field moved away from a pure translation where the truth does
    tf = ser.truth_field(1)
    assert np.abs(tf - tf.mean(axis=(1, 2), keepdims=True)).max() > 0.1


def test_nonrigid_flow_stops_on_the_metric_gradient_norm():
    # the reading of the stop rule: a level ends when |d|_M = sqrt(mean_j |Nc dE/dc_j|^2) falls
    # below tol_grad; check it on the returned control values with the energy's own gradient
    ser = synth.make_series(synth.SeriesSpec(2, 96, 96, step=1.5, field_amp=1.0, snr=(10, 10), seed=32))
    F = ser.frames.numpy()
    cfg = O.Config(levels=2, mode="nonrigid")
    c, st = O.register_nonrigid(O.pyramid(F[0], 2), O.pyramid(F[1], 2), None, cfg)
    assert st.stop == [0, 0]
    g = O.grid_for(96, 96)
    _, gr = O.grid_energy(F[0].astype(np.float64), F[1].astype(np.float64), 0, g, c, cfg.lam)
    Nc = g.nx * g.ny
    assert math.sqrt(((Nc * gr) ** 2).sum() / Nc) < cfg.tol_grad


@pytest.mark.parametrize("seed", [33, 34])
def test_nonrigid_result_is_insensitive_to_float32_sized_perturbations(seed):
    # with a continuously differentiable energy and the gradient stop, the result is the minimiser
    # to within the stop tolerance: frames perturbed at the float32 rounding level (1e-7 relative)
    # give the same deformation to a few thousandths of a pixel
    ser = synth.make_series(synth.SeriesSpec(2, 128, 128, step=1.0, field_amp=1.5, snr=(10, 10), seed=seed))
    F = ser.frames.numpy().astype(np.float64)
    cfg = O.Config(levels=2, mode="nonrigid")
    c0, _ = O.register_nonrigid(O.pyramid(F[0], 2), O.pyramid(F[1], 2), None, cfg)
    rng = np.random.default_rng(seed)
    Fp = F * (1.0 + 1e-7 * rng.standard_normal(F.shape))
    c1, _ = O.register_nonrigid(O.pyramid(Fp[0], 2), O.pyramid(Fp[1], 2), None, cfg)
    assert O.max_px_error(c0, c1, 128, 128, "nonrigid") <= 0.005


# ---------------------------------------------------------------- three levels
@pytest.mark.parametrize("seed", range(3))
def test_three_levels_recover_known_translation_on_a_coarse_lattice(seed):
    # with a 16-px lattice the coarsest of three levels still resolves the period (4 px)
    rng = np.random.default_rng(300 + seed)
    s = rng.uniform(-6.0, 6.0, size=2)
    R, T = synth.translated_pair(160, 160, s, seed=seed, noise_snr=None if seed % 2 == 0 else 20.0, period=16.0,
                                 sigma=3.0)
    th, st = O.register_rigid(O.pyramid(R, 3), O.pyramid(T, 3), np.zeros(3), O.Config(levels=3))
    assert abs(th[1] - s[0]) <= 0.05 and abs(th[2] - s[1]) <= 0.05, (th, s)
    ser = synth.make_series(synth.SeriesSpec(2, 128, 128, step=4.0, field_amp=1.0, snr=(10, 10), period=16.0,
                                             sigma=3.0, field_rate=(0.8, 1.2), seed=310 + seed))
    F = ser.frames.numpy()
    c, _ = O.register_nonrigid(O.pyramid(F[0], 3), O.pyramid(F[1], 3), None, O.Config(levels=3, mode="nonrigid"))
    err = (O.grid_dense(O.grid_for(128, 128), c) - ser.truth_field(1))[:, 16:-16, 16:-16]
    assert np.sqrt((err ** 2).sum(0).mean()) <= 0.1


def test_three_level_flow_lands_on_brute_force_minimiser():
    R, T = synth.rigid_pair(64, 64, 0.0, (2.63, -1.41), noise_snr=6.0, seed=42, period=16.0, sigma=3.0)
    cfg = O.Config(levels=3, tol_grad=1e-7)
    th, _ = O.register_rigid(O.pyramid(R, 3), O.pyramid(T, 3), np.zeros(3), cfg)
    grid = np.arange(-0.05, 0.05 + 1e-12, 0.005)
    E = np.array([[O.rigid_energy(R, T, [th[0], th[1] + a, th[2] + b], grad=False) for b in grid] for a in grid])
    ia, ib = np.unravel_index(E.argmin(), E.shape)
    assert abs(grid[ia]) <= 0.005 and abs(grid[ib]) <= 0.005
    assert abs(th[1] - 2.63) <= 0.05 and abs(th[2] + 1.41) <= 0.05


# ---------------------------------------------------------------- brute force
def test_gradient_flow_lands_on_brute_force_minimiser():
    R, T = synth.rigid_pair(32, 32, 0.0, (0.63, -0.41), noise_snr=6.0, seed=41)
    cfg = O.Config(levels=2, tol_grad=1e-7)
    th, _ = O.register_rigid(O.pyramid(R, 2), O.pyramid(T, 2), np.zeros(3), cfg)

    def best(center, half, step):
        grid = np.arange(-half, half + 1e-12, step)
        bestE, arg = np.inf, None
        for gx in center[0] + grid:
            for gy in center[1] + grid:
                E = O.rigid_energy(R, T, [th[0], gx, gy], grad=False)
                if E < bestE:
                    bestE, arg = E, (gx, gy)
        return np.array(arg), bestE

    coarse, _ = best((0.63, -0.41), 1.0, 0.05)
    fine, Ebf = best(coarse, 0.05, 0.005)
    assert np.abs(fine - th[1:]).max() <= 0.01, (fine, th)
    assert O.rigid_energy(R, T, th, grad=False) <= Ebf + 1e-9
    # alpha: 1-D search at the returned translation
    al = th[0] + np.arange(-2e-3, 2e-3 + 1e-12, 2e-5)
    Es = [O.rigid_energy(R, T, [a, th[1], th[2]], grad=False) for a in al]
    assert abs(al[int(np.argmin(Es))] - th[0]) <= 4e-5


# ---------------------------------------------------------------- composition
def _rigid_map(th, pts, W, H):
    cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
    ca, sa = math.cos(th[0]), math.sin(th[0])
    x, y = pts[:, 0] - cx, pts[:, 1] - cy
    return np.stack([ca * x - sa * y + cx + th[1], sa * x + ca * y + cy + th[2]], axis=1)


def test_rigid_composition_matches_pointwise_composition():
    rng = np.random.default_rng(51)
    a, b = np.array([0.1, 2.0, -1.0]), np.array([-0.3, 0.5, 4.0])
    pts = rng.uniform(0, 100, size=(20, 2))
    direct = _rigid_map(b, _rigid_map(a, pts, 101, 77), 101, 77)
    np.testing.assert_allclose(_rigid_map(O.compose_rigid(a, b), pts, 101, 77), direct, atol=1e-12)


def test_rigid_composition_associative_with_identity():
    rng = np.random.default_rng(52)
    a, b, c = (rng.uniform(-1, 1, 3) for _ in range(3))
    l = O.compose_rigid(O.compose_rigid(a, b), c)
    r = O.compose_rigid(a, O.compose_rigid(b, c))
    np.testing.assert_allclose(l, r, atol=1e-12)
    np.testing.assert_array_equal(O.compose_rigid(a, np.zeros(3)), a)
    np.testing.assert_allclose(O.compose_rigid(np.zeros(3), a), a, atol=0)


def test_grid_composition_of_translations_and_linear_fields():
    g = O.grid_for(40, 33, 8)
    t1 = np.broadcast_to(np.array([0.7, -1.2])[:, None, None], (2, g.ny, g.nx)).copy()
    t2 = np.broadcast_to(np.array([-0.2, 0.4])[:, None, None], (2, g.ny, g.nx)).copy()
    np.testing.assert_allclose(O.compose_grid(g, t1, t2), t1 + t2, atol=1e-14)
    # u2(X) = (0.1 X, 0): composition at control point X_j is c1_j + 0.1 (X_j + c1_jx) inside the grid
    jy, jx = np.mgrid[0:g.ny, 0:g.nx].astype(np.float64)
    u2 = np.stack([0.1 * 8 * jx, np.zeros_like(jx)])
    c = O.compose_grid(g, 0.5 * t1, u2)
    inside = (8 * jx + 0.35 <= 8 * (g.nx - 1))
    np.testing.assert_allclose(c[0][inside], (0.35 + 0.1 * (8 * jx + 0.35))[inside], atol=1e-12)


# ---------------------------------------------------------------- scan DAGs
def _concat_check(d):
    vals = [f"{i}," for i in range(d.n)]
    for (l, r) in d.ops:
        vals.append(("" if l < 0 else vals[l]) + ("" if r < 0 else vals[r]))
    return vals


@pytest.mark.parametrize("name", list(O.DAGS))
def test_dag_computes_inclusive_prefixes(name):
    for n in range(1, 70):
        d = O.DAGS[name](n)
        vals = _concat_check(d)
        for i, o in enumerate(d.out):
            assert vals[o] == "".join(f"{j}," for j in range(i + 1)), (name, n, i)


def test_blelloch_is_exclusive_and_one_shift_from_inclusive():
    # Sec. 1: an exclusive result becomes inclusive by one shift plus one operator application
    for n in range(1, 70):
        d = O.dag_blelloch(n)
        vals = _concat_check(d)
        excl = ["" if o < 0 else vals[o] for o in d.out]
        for i in range(n):
            assert excl[i] == "".join(f"{j}," for j in range(i))
            assert excl[i] + f"{i}," == "".join(f"{j}," for j in range(i + 1))
        # Table 1's work 2 (n - 1), identity applications included, also off the powers of two
        assert d.work() == 2 * max(0, n - 1), n


def test_dag_work_and_depth_match_table1_and_fig2():
    g = json.load(open(GOLDEN))
    for N in (2, 4, 8, 16, 64, 256, 4096):
        lg = int(math.log2(N))
        assert O.dag_sequential(N).work() == N - 1 and O.dag_sequential(N).depth() == N - 1
        assert O.dag_blelloch(N).work() == 2 * (N - 1)
        assert O.dag_dissemination(N).work() == N * lg - N + 1
        assert O.dag_dissemination(N).depth() == lg
        assert O.dag_ladner_fischer(N).work() < 4 * N - 5
        assert O.dag_ladner_fischer(N).depth() == lg
        assert O.dag_brent_kung(N).work() == 2 * N - 2 - lg
    f2 = g["fig2_dissemination_n8"]
    d = O.dag_dissemination(f2["N"])
    assert d.work() == f2["work"] and d.depth() == f2["rounds"]


def test_table5_work_counts():
    # full registration on P ranks: N preprocessing A's, N-P local reduction steps,
    # the global scan over P elements, N steps in the last local phase (Sec. 4.1, Table 5)
    g = json.load(open(GOLDEN))["table5_work"]
    N = g["N"]
    assert g["serial"] == N + (N - 1) == O.dag_sequential(N).work() + N
    for P, wd, wl in zip(g["P"], g["dissemination"], g["ladner_fischer"]):
        assert N + (N - P) + O.dag_dissemination(P).work() + N == wd
        assert N + (N - P) + O.dag_ladner_fischer(P).work() + N == wl


# ---------------------------------------------------------------- operator / scan
@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_operator_associativity_on_tiny_series(mode):
    spec = synth.SeriesSpec(4, 64, 64, step=1.5, field_amp=0.5, snr=(10, 10), seed=61)
    F = synth.make_series(spec).frames.numpy()
    cfg = O.Config(levels=2, mode=mode)
    pyrs = [O.pyramid(f, 2) for f in F]
    a, b, c = (O.op_A(pyrs, i, i + 1, cfg) for i in range(3))
    left = O.op_B(O.op_B(a, b, pyrs, cfg), c, pyrs, cfg)
    right = O.op_B(a, O.op_B(b, c, pyrs, cfg), pyrs, cfg)
    assert (left.i, left.k) == (right.i, right.k) == (0, 3)
    assert O.max_px_error(left.phi, right.phi, 64, 64, mode) <= 0.02


def test_operator_B_rejects_non_adjacent_elements():
    e1 = O.Elem(0, 1, np.zeros(3))
    e2 = O.Elem(2, 3, np.zeros(3))
    with pytest.raises(ValueError):
        O.op_B(e1, e2, None, O.Config())


@pytest.mark.parametrize("dag", ["brent_kung", "dissemination", "ladner_fischer", "lookback2", "lookback4"])
def test_parallel_scan_equals_sequential_recursion(dag):
    spec = synth.spec_c1()
    spec.n_frames = 9
    F = synth.make_series(spec).frames.numpy()
    cfg = O.Config(levels=2)
    pyrs = [O.pyramid(f, 2) for f in F]
    leaves = [O.op_A(pyrs, i, i + 1, cfg) for i in range(len(F) - 1)]
    seq = O.scan(F, cfg, O.dag_sequential(len(F) - 1), leaves=leaves, pyrs=pyrs)
    par = O.scan(F, cfg, O.DAGS[dag](len(F) - 1), leaves=leaves, pyrs=pyrs)
    for i, (s, p) in enumerate(zip(seq, par)):
        assert (s.i, s.k) == (p.i, p.k) == (0, i + 1)
        assert O.max_px_error(s.phi, p.phi, 128, 128, "rigid") <= 0.02


# ------------------------------------------------------------------ the line search's step rule
@pytest.mark.parametrize("E0,s,c", [(0.3, -2.0, 5.0), (1.0, -0.01, 0.4), (0.05, -1e-6, 3e-5)])
def test_step_rule_lands_on_the_minimiser_of_a_parabola(E0, s, c):
    # E(t) = E0 + s t + c t^2 has its minimum at t* = -s / (2 c); a trial at tau gives the
    # parabola exactly, so the rule returns t* clamped to its safeguard interval
    tstar = -s / (2 * c)
    for tau in (0.3 * tstar, 0.9 * tstar, 1.7 * tstar, 3.0 * tstar, 12.0 * tstar):
        Et = E0 + s * tau + c * tau * tau
        accepted = Et <= E0 + 0.25 * tau * s
        got = O.step_size(E0, s, tau, Et, accepted)
        lo, hi = (0.5 * tau, 4.0 * tau) if accepted else (0.1 * tau, 0.5 * tau)
        # Et - E0 - s tau recovers c tau^2 up to the rounding of the energies (a few ulp of E0)
        rel = max(1e-12, 8e-16 * E0 / (c * tau * tau))
        assert got == pytest.approx(min(max(tstar, lo), hi), rel=rel)


def test_step_rule_without_curvature_doubles_or_halves():
    # a trial at or below the tangent line (no positive curvature): plain doubling / halving
    assert O.step_size(1.0, -1.0, 0.5, 0.4, True) == 1.0
    assert O.step_size(1.0, -1.0, 0.5, 0.5, False) == 0.25


# ------------------------------------------------------------------ the first trial step
def test_bb_first_step_is_the_exact_step_on_a_round_quadratic():
    # E = a/2 |x|^2 in the plain metric: d = -a x; after a step of tau_acc along d_prev the
    # Barzilai-Borwein step is 1/a, the exact minimiser along any direction
    a = 3.7
    x0 = np.array([0.4, -1.2, 0.9, 2.0])
    tau_acc = 0.11
    dp = -a * x0
    x1 = x0 + tau_acc * dp
    assert O.bb_first_step(0.5, tau_acc, dp, -a * x1) == pytest.approx(1.0 / a, rel=1e-14)


def test_bb_first_step_in_the_rigid_metric():
    # E = 1/2 sum h_k t_k^2 with h = c (m0, 1, 1): in the metric diag(m0, 1, 1) the direction is
    # d = -c t and the exact step 1/c
    c, m0 = 0.8, 40.0
    h = c * np.array([m0, 1.0, 1.0])
    t0 = np.array([0.01, 1.5, -0.7])
    dp = -(h * t0) / np.array([m0, 1.0, 1.0])
    t1 = t0 + 0.3 * dp
    d = -(h * t1) / np.array([m0, 1.0, 1.0])
    assert O.bb_first_step(0.5, 0.3, dp, d, m0) == pytest.approx(1.0 / c, rel=1e-13)


def test_bb_first_step_falls_back_without_curvature():
    dp = np.array([1.0, -2.0])
    assert O.bb_first_step(0.25, 0.1, dp, dp) == 0.25           # no change of direction
    assert O.bb_first_step(0.25, 0.1, dp, 2.0 * dp) == 0.25     # negative curvature along the step


# ------------------------------------------------------------------ the nonrigid flow's scalar product
def test_metric_on_an_affine_image_is_the_closed_form():
    # T = 0.2 + b x + c y: the model's derivative is (b, c) wherever its window stays inside the frame,
    # so for a control point whose support does too, sum_x w_j(x)^2 dT^2 = b^2 S^2 (resp. c^2 S^2),
    # S = sum over one axis of the tent weight squared = 1 + 2 sum_{t=1}^{s-1} (1 - t/s)^2
    H, W, sp_ = 49, 65, 8
    b, c = 0.03, -0.05
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    T = 0.2 + b * x + c * y
    g = O.grid_for(W, H, sp_)
    lam = 1.5
    m = O.grid_metric(T, 0, g, np.zeros((2, g.ny, g.nx)), lam)
    P = W * H
    var = smooth_1_8_3_4_1_8(T).var()    # variance of the model's samples at the zero field
    S = 1.0 + 2.0 * sum((1.0 - t / sp_) ** 2 for t in range(1, sp_))
    # unnormalised values of the whole grid, then the normalisation by the mean of all 2 Nc values
    nb = np.zeros((g.ny, g.nx))
    nb[:, 1:] += 1; nb[:, :-1] += 1; nb[1:, :] += 1; nb[:-1, :] += 1
    interior = (slice(2, g.ny - 2), slice(2, g.nx - 2))       # supports [8 (j-1), 8 (j+1)] 2 px or more inside
    raw_x = b * b * S * S / (P * var) + lam * 4 / P
    raw_y = c * c * S * S / (P * var) + lam * 4 / P
    ratio = (m[0][interior] / raw_x).ravel().tolist() + (m[1][interior] / raw_y).ravel().tolist()
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-10)   # one normalisation constant for all
    assert m[0][interior] == pytest.approx(raw_x * ratio[0], rel=1e-12)


def test_metric_of_a_constant_image_is_the_regulariser_alone():
    g = O.grid_for(40, 30, 8)
    m = O.grid_metric(np.full((30, 40), 0.4), 0, g, np.zeros((2, g.ny, g.nx)), 2.0)
    nb = np.zeros((g.ny, g.nx))
    nb[:, 1:] += 1; nb[:, :-1] += 1; nb[1:, :] += 1; nb[:-1, :] += 1
    np.testing.assert_allclose(m[0], nb / nb.mean(), rtol=1e-13)
    np.testing.assert_allclose(m[1], nb / nb.mean(), rtol=1e-13)


def test_the_metric_changes_the_path_not_the_minimiser():
    # the stationary point of the energy does not depend on the scalar product of the flow
    ser = synth.make_series(synth.SeriesSpec(2, 96, 96, step=1.5, field_amp=1.0, snr=(10, 10), seed=35))
    F = ser.frames.numpy()
    out = []
    for metric in (0, 1):
        cfg = O.Config(levels=2, mode="nonrigid", metric=metric, tol_grad=1e-7, max_iter=4000)
        c, st = O.register_nonrigid(O.pyramid(F[0], 2), O.pyramid(F[1], 2), None, cfg)
        assert st.stop == [0, 0]
        out.append(c)
    assert O.max_px_error(out[0], out[1], 96, 96, "nonrigid") <= 1e-4


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_lookback_dag_prefixes_work_and_chain_depth(k):
    # every output is the inclusive prefix; the chain of prefixes advances k leaves per operator, so
    # the depth is about n/k + 2 log2 k; work: n - 1 prefixes plus sum_m (n - 2^m + 1) windows
    n = 37
    d = O.dag_lookback(n, k)
    sym = [frozenset([j]) for j in range(n)]
    span = [(j, j) for j in range(n)]
    for (l, r) in d.ops:
        assert span[l][1] + 1 == span[r][0]            # B needs adjacent elements
        span.append((span[l][0], span[r][1]))
    for i, o in enumerate(d.out):
        assert span[o] == (0, i)
    m = k.bit_length() - 1
    assert d.work() == (n - 1) + sum(n - (1 << lev) + 1 for lev in range(1, m + 1))
    if k == 1:
        assert d.ops == O.dag_sequential(n).ops
    assert d.depth() <= (n - 1) // k + 2 * m + k


# ------------------------------------------------------------------ the H1 scalar product (metric 2)
def _graph_h1(ny, nx, sigma):
    # M = I + sigma^2 L built from networkx's own grid graph and Laplacian (independent of the oracle)
    nxlib = pytest.importorskip("networkx")
    Gr = nxlib.grid_2d_graph(ny, nx)
    nodes = [(r, c) for r in range(ny) for c in range(nx)]
    L = nxlib.laplacian_matrix(Gr, nodelist=nodes).toarray().astype(np.float64)
    return np.eye(ny * nx) + sigma * sigma * L


@pytest.mark.parametrize("ny,nx,sigma", [(5, 7, 1.0), (9, 4, 2.5), (1, 6, 0.7)])
def test_h1_apply_and_inverse_against_the_graph_laplacian(ny, nx, sigma):
    g = O.Grid(nx, ny, 16, 16 * (nx - 1) + 1, 16 * (ny - 1) + 1)
    rng = np.random.default_rng(ny * 100 + nx)
    v = rng.standard_normal((ny, nx))
    M = _graph_h1(ny, nx, sigma)
    assert np.allclose(O.h1_apply(g, sigma, v).ravel(), M @ v.ravel(), rtol=0, atol=1e-12)
    x = O.h1_inverse(g, sigma, v)
    assert np.allclose(M @ x.ravel(), v.ravel(), rtol=0, atol=1e-11)
    assert np.allclose(x.ravel(), np.linalg.solve(M, v.ravel()), rtol=0, atol=1e-11)


def test_h1_inverse_on_the_cosine_modes_and_the_constant_field():
    # the grid graph's Laplacian (free ends) has the eigenvectors cos(pi k (j + 1/2) / n) per axis,
    # eigenvalues 2 - 2 cos(pi k / n): M^-1 divides such a mode by 1 + sigma^2 (lam_x + lam_y) and
    # leaves a constant field as it is
    ny, nx, sigma = 6, 9, 1.7
    g = O.Grid(nx, ny, 8, 8 * (nx - 1) + 1, 8 * (ny - 1) + 1)
    jy, jx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    for k, m in [(1, 0), (2, 3), (8, 5)]:
        v = np.cos(np.pi * k * (jx + 0.5) / nx) * np.cos(np.pi * m * (jy + 0.5) / ny)
        lam = (2 - 2 * math.cos(math.pi * k / nx)) + (2 - 2 * math.cos(math.pi * m / ny))
        assert np.allclose(O.h1_inverse(g, sigma, v), v / (1 + sigma * sigma * lam), rtol=0, atol=1e-12)
    assert np.allclose(O.h1_inverse(g, sigma, np.full((ny, nx), 0.37)), 0.37, rtol=0, atol=1e-13)
    # sigma = 0: the identity
    v = np.random.default_rng(5).standard_normal((ny, nx))
    assert np.array_equal(O.h1_inverse(g, 0.0, v), v)


def test_h1_flow_reaches_the_minimiser_of_the_other_scalar_products():
    # the scalar product changes the path of the flow, not its stationary point: stopped on a tight
    # gradient tolerance, the H1 flow, the mean flow and the Gauss-Newton flow land together; with
    # sigma = 0 the H1 flow is the mean flow step for step (its step-size sums run in another order,
    # hence rounding-level differences)
    ser = synth.make_series(synth.SeriesSpec(2, 96, 96, step=1.0, field_amp=1.2, snr=(12, 12), seed=41))
    F = ser.frames.numpy().astype(np.float64)
    P0, P1 = O.pyramid(F[0], 2), O.pyramid(F[1], 2)
    res = {}
    for name, metric, sigma in [("mean", 0, 1.0), ("gn", 1, 1.0), ("h1", 2, 1.5), ("h1s0", 2, 0.0)]:
        cfg = O.Config(levels=2, mode="nonrigid", metric=metric, sigma=sigma, tol_grad=1e-6)
        res[name] = O.register_nonrigid(P0, P1, None, cfg)
    g = O.grid_for(96, 96)
    for name in ("gn", "h1"):
        assert O.max_px_error(res[name][0], res["mean"][0], 96, 96, "nonrigid") < 2e-3, name
    assert O.max_px_error(res["h1s0"][0], res["mean"][0], 96, 96, "nonrigid") < 1e-7
    assert res["h1s0"][1].iters == res["mean"][1].iters


# ------------------------------------------------------------------ the coarse levels' stop rule
def test_coarse_level_tolerance_changes_the_path_not_the_result():
    # a coarse level only supplies the next level's initial guess: stopped at 10x the tolerance it
    # takes fewer evaluations, and the finest level (same tolerance) ends at the same minimiser
    ser = synth.make_series(synth.SeriesSpec(3, 128, 128, step=1.0, field_amp=1.2, snr=(12, 12), seed=51))
    F = ser.frames.numpy().astype(np.float64)
    P0, P1 = O.pyramid(F[0], 2), O.pyramid(F[1], 2)
    for mode in ("nonrigid", "rigid"):
        res = {}
        for tc in (1.0, 10.0):
            cfg = O.Config(levels=2, mode=mode, tol_coarse=tc, tol_grad=1e-6)
            res[tc] = O.register(P0, P1, O.identity(mode, 128, 128, cfg.grid), cfg)
        assert res[10.0][1].evals[1] < res[1.0][1].evals[1], mode
        assert O.max_px_error(res[10.0][0], res[1.0][0], 128, 128, mode) < 2e-3, mode
    # one level: the factor never applies
    for mode in ("nonrigid", "rigid"):
        out = [O.register([P0[0]], [P1[0]], O.identity(mode, 128, 128, 0), O.Config(levels=1, mode=mode, tol_coarse=tc))
               for tc in (1.0, 10.0)]
        assert np.array_equal(np.asarray(out[0][0]), np.asarray(out[1][0])), mode
        assert out[0][1].evals == out[1][1].evals, mode
