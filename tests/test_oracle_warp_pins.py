"""Pins of the oracle's registered-series functions (Sec. 2: the frames of the series are
registered to the first frame and averaged), against facts that do not come from the oracle:
exact index shifts, an exact quarter-turn, affine reproduction by bilinear interpolation, and
the plain mean."""
import math

import numpy as np
import pytest

import oracle as O


def _frame(H=24, W=20, seed=0):
    return np.random.default_rng(seed).random((H, W))


def _shift_by_index(T, dx, dy):
    # out[r, c] = T[clip(r + dy), clip(c + dx)]: integer translation with clamp-to-edge
    H, W = T.shape
    r = np.clip(np.arange(H) + dy, 0, H - 1)
    c = np.clip(np.arange(W) + dx, 0, W - 1)
    return T[np.ix_(r, c)]


def test_identity_reproduces_the_frame_exactly():
    T = _frame()
    assert np.array_equal(O.warp(T, "rigid", [0.0, 0.0, 0.0]), T)
    g = O.grid_for(20, 24, 8)
    assert np.array_equal(O.warp(T, "nonrigid", np.zeros((2, g.ny, g.nx)), grid=8), T)


@pytest.mark.parametrize("dx,dy", [(3, -2), (-5, 4), (0, 7), (25, -30)])
def test_integer_translation_is_an_index_shift_with_edge_clamp(dx, dy):
    T = _frame()
    assert np.array_equal(O.warp(T, "rigid", [0.0, float(dx), float(dy)]), _shift_by_index(T, dx, dy))
    g = O.grid_for(20, 24, 8)
    c = np.zeros((2, g.ny, g.nx))
    c[0] += dx
    c[1] += dy
    assert np.array_equal(O.warp(T, "nonrigid", c, grid=8), _shift_by_index(T, dx, dy))


def test_quarter_turn_about_the_centre_is_an_index_rotation():
    # R(pi/2) maps centred (xc, yc) to (-yc, xc): out[y, x] = T[x, n-1-y] on a square frame
    n = 13
    T = _frame(n, n, 3)
    want = np.array([[T[x, n - 1 - y] for x in range(n)] for y in range(n)])
    assert np.abs(O.warp(T, "rigid", [math.pi / 2, 0.0, 0.0]) - want).max() < 1e-12


def test_affine_image_is_reproduced_at_subpixel_positions():
    # bilinear interpolation is exact on a + b x + c y, so T o phi is the ramp at phi(x)
    H, W = 30, 40
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    T = 0.3 + 0.02 * x - 0.015 * y
    th = [0.01, 1.37, -0.62]
    out = O.warp(T, "rigid", th)
    ca, sa = math.cos(th[0]), math.sin(th[0])
    cx, cy = (W - 1) / 2, (H - 1) / 2
    px = ca * (x - cx) - sa * (y - cy) + cx + th[1]
    py = sa * (x - cx) + ca * (y - cy) + cy + th[2]
    inside = (px >= 0) & (px <= W - 1) & (py >= 0) & (py <= H - 1)
    assert inside.sum() > 0.8 * H * W
    assert np.abs(out - (0.3 + 0.02 * px - 0.015 * py))[inside].max() < 1e-12


def test_smooth_field_on_an_affine_image():
    # a control grid whose values are an affine function of the point gives an affine u
    # (bilinear interpolation of affine values is exact), and T o phi is the ramp at x + u(x)
    H, W = 33, 33
    g = O.grid_for(W, H, 8)
    jy, jx = np.mgrid[0:g.ny, 0:g.nx].astype(np.float64) * g.s
    c = np.stack([0.4 + 0.01 * jx - 0.02 * jy, -0.3 + 0.015 * jx + 0.005 * jy])
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    T = 1.0 + 0.05 * x + 0.03 * y
    out = O.warp(T, "nonrigid", c, grid=8)
    px = x + 0.4 + 0.01 * x - 0.02 * y
    py = y - 0.3 + 0.015 * x + 0.005 * y
    inside = (px >= 0) & (px <= W - 1) & (py >= 0) & (py <= H - 1)
    assert np.abs(out - (1.0 + 0.05 * px + 0.03 * py))[inside].max() < 1e-12


def test_registered_series_and_mean():
    # frames that are exact integer shifts of f0 (interior), registered with those shifts,
    # are f0 again away from the clamped border; the mean is the plain average
    f0 = _frame(32, 32, 7)
    shifts = [(1, 2), (-3, 1), (2, -2)]
    frames = [f0] + [_shift_by_index(f0, -dx, -dy) for dx, dy in shifts]
    phis = [[0.0, float(dx), float(dy)] for dx, dy in shifts]
    out, mean = O.register_series(np.stack(frames), "rigid", phis)
    assert np.array_equal(out[0], f0)
    for k in range(1, 4):
        assert np.array_equal(out[k][4:-4, 4:-4], f0[4:-4, 4:-4])
    assert np.abs(mean - np.stack(out).mean(axis=0)).max() < 1e-15
    assert np.abs(mean[4:-4, 4:-4] - f0[4:-4, 4:-4]).max() < 1e-15
