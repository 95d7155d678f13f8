"""Parity of reg_warp (registered series and its mean, Sec. 2) with the FP64 oracle.

Both sides resample the same frames by the same deformations (the FP32 elements or control
values the CUDA path holds, widened to FP64 for the oracle).  The bar is FP32 arithmetic on
values of order 1: a sample position carries a relative error of a few 1e-7 of the
displacement (|v| <= a few tens of px here, so <= 1e-5 px) and the interpolation a few ulps,
so |out_gpu - out_oracle| <= 1e-5 everywhere.  The mean sums FP32 runs of 16 frames
(error <= 16 ulp of the run sum, ~2e-6 relative) folded into float-float, and the chunks in
FP64, so its error stays far below the same bound.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_12478_gb300 import binding as B
from paper_2010_12478_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_12478_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def frames_of(n, H, W, seed=1410):
    spec = synth.SeriesSpec(n, H, W, step=2.0, field_amp=1.0, snr=(10.0, 10.0), seed=seed)
    return synth.make_series(spec).frames


def rigid_elems(n, rng, amax=0.02, gmax=6.0):
    return [(0, k + 1, float(rng.uniform(-amax, amax)), float(rng.uniform(-gmax, gmax)),
             float(rng.uniform(-gmax, gmax))) for k in range(n)]


def oracle_rigid(F, elems):
    phis = [np.array(e[2:], dtype=np.float32).astype(np.float64) for e in elems]
    return O.register_series(F.astype(np.float64), "rigid", phis)


def run_warp(ctx, F, elems=None, grids=None, want_out=True, want_mean=True):
    N, H, W = F.shape
    dF = torch.from_numpy(F).cuda()
    out = torch.full((N, H, W), float("nan"), device="cuda") if want_out else None
    mean = torch.full((H, W), float("nan"), device="cuda") if want_mean else None
    ctx.warp(dF, elems=elems, grids=grids, out=out, mean=mean)
    torch.cuda.synchronize()
    return (out.cpu().numpy() if want_out else None), (mean.cpu().numpy() if want_mean else None)


@pytest.mark.parametrize("shape", [(128, 128), (96, 200), (45, 67), (40, 81)])
def test_rigid_registered_series_matches_oracle(shape):
    H, W = shape
    F = frames_of(9, H, W).numpy()
    els = rigid_elems(8, np.random.default_rng(H * 1000 + W))
    ctx = B.Context(B.Config())
    ctx.set_timing(True)
    out, mean = run_warp(ctx, F, elems=els)
    # TMA staging whenever the 80 x 40 box fits the frame and rows are 16-byte multiples
    assert ctx.last_timing()["tma_staged"] == int(W >= 80 and H >= 40 and W % 4 == 0)
    want, wmean = oracle_rigid(F, els)
    assert np.array_equal(out[0], F[0])
    assert np.abs(out - want).max() <= TOL
    assert np.abs(mean - wmean).max() <= TOL


def test_rigid_large_rotation_and_far_shifts_fall_back_and_clamp():
    # a 0.6 rad turn does not fit the staged box (global-memory samples); a 1000 px shift
    # samples only the clamped edge
    F = frames_of(4, 128, 160).numpy()
    els = [(0, 1, 0.6, 3.0, -2.0), (0, 2, -0.3, 1000.0, 5.0), (0, 3, 0.0, -7.25, 3.5)]
    ctx = B.Context(B.Config())
    out, mean = run_warp(ctx, F, elems=els)
    want, wmean = oracle_rigid(F, els)
    assert np.abs(out - want).max() <= TOL
    assert np.abs(mean - wmean).max() <= TOL


@pytest.mark.parametrize("grid", [0, 16, 4])
def test_nonrigid_registered_series_matches_oracle(grid):
    H, W = 128, 144
    N = 6
    F = frames_of(N, H, W).numpy()
    nx, ny, s = B.grid_dims(W, H, grid, 2)
    rng = np.random.default_rng(grid + 7)
    # smooth-ish control values: a common shift plus per-point wiggle
    g = (rng.uniform(-3, 3, (N - 1, 1, 1, 2)) + rng.uniform(-1.5, 1.5, (N - 1, ny, nx, 2))).astype(np.float32)
    ctx = B.Context(B.Config(mode="nonrigid", grid=grid))
    out, mean = run_warp(ctx, F, grids=torch.from_numpy(g).cuda())
    phis = [np.transpose(g[k].astype(np.float64), (2, 0, 1)) for k in range(N - 1)]
    want, wmean = O.register_series(F.astype(np.float64), "nonrigid", phis, grid=grid)
    assert np.abs(out - want).max() <= TOL
    assert np.abs(mean - wmean).max() <= TOL


def test_single_frame_and_mean_only_and_determinism():
    F = frames_of(1, 64, 96).numpy()
    ctx = B.Context(B.Config())
    out, mean = run_warp(ctx, F)
    assert np.array_equal(out[0], F[0]) and np.array_equal(mean, F[0])
    F = frames_of(70, 96, 128).numpy()   # two chunks of frames in the mean
    els = rigid_elems(69, np.random.default_rng(3))
    _, m1 = run_warp(ctx, F, elems=els, want_out=False)
    _, m2 = run_warp(ctx, F, elems=els, want_out=False)
    assert np.array_equal(m1, m2)
    _, wmean = oracle_rigid(F, els)
    assert np.abs(m1 - wmean).max() <= TOL


def test_invalid_arguments_are_rejected():
    ctx = B.Context(B.Config())
    F = torch.zeros((3, 64, 64), device="cuda")
    with pytest.raises(B.RegError) as e:
        ctx.warp(F, elems=[(0, 1, 0, 0, 0), (0, 2, 0, 0, 0)])   # no output
    assert e.value.code == B.REG_EINVAL
    with pytest.raises(B.RegError) as e:
        ctx.warp(F, out=torch.zeros_like(F))   # rigid needs the elements
    assert e.value.code == B.REG_EINVAL
    nctx = B.Context(B.Config(mode="nonrigid"))
    with pytest.raises(B.RegError) as e:
        nctx.scan_grids(torch.zeros(1, device="cuda"))   # no scan yet
    assert e.value.code == B.REG_ESTATE


def test_scan_then_warp_registers_the_series():
    # the nonrigid scan's control values, read back with reg_scan_grids, register the series:
    # the result equals the oracle's resampling by those values, and the registered mean
    # correlates better with f_0 than the plain mean of the drifting frames
    spec = synth.spec_c1()
    ser = synth.make_series(spec, device="cuda")
    F = ser.frames
    N, H, W = F.shape
    ctx = B.Context(B.Config(mode="nonrigid"))
    ctx.scan(F, schedule="brent_kung", exec="persistent")
    nx, ny, s = B.grid_dims(W, H, 0, 2)
    g = torch.zeros((N - 1, ny, nx, 2), device="cuda")
    assert ctx.scan_grids(g) == N - 1
    out = torch.zeros_like(F)
    mean = torch.zeros((H, W), device="cuda")
    ctx.warp(F, grids=g, out=out, mean=mean)
    Fh = F.cpu().numpy().astype(np.float64)
    phis = [np.transpose(g[k].cpu().numpy().astype(np.float64), (2, 0, 1)) for k in range(N - 1)]
    want, wmean = O.register_series(Fh, "nonrigid", phis)
    assert np.abs(out.cpu().numpy() - want).max() <= TOL
    assert np.abs(mean.cpu().numpy() - wmean).max() <= TOL

    def ncc(a, b):
        a = a[8:-8, 8:-8] - a[8:-8, 8:-8].mean()
        b = b[8:-8, 8:-8] - b[8:-8, 8:-8].mean()
        return float((a * b).sum() / np.sqrt((a * a).sum() * (b * b).sum()))

    assert ncc(wmean, Fh[0]) > ncc(Fh.mean(axis=0), Fh[0]) + 0.2


def test_c2_full_size_sampled_registered_frames_match_oracle():
    # 256 frames of 512 x 512, rigid scan then warp, in the launch shape of the full workload;
    # sampled frames element by element and the mean at sampled rows
    spec = synth.spec_c2()
    ser = synth.make_series(spec, device="cuda")
    F = ser.frames
    N, H, W = F.shape
    ctx = B.Context(B.Config())
    els, _ = ctx.scan(F, schedule="brent_kung", exec="persistent")
    out = torch.zeros_like(F)
    mean = torch.zeros((H, W), device="cuda")
    ctx.warp(F, elems=els, out=out, mean=mean)
    Fh = F.cpu().numpy()
    rng = np.random.default_rng(1410)
    for k in rng.choice(np.arange(1, N), 3, replace=False):
        want = O.warp(Fh[k].astype(np.float64), "rigid", np.array(els[k - 1][2:], dtype=np.float32).astype(np.float64))
        assert np.abs(out[k].cpu().numpy() - want).max() <= TOL
    _, wmean = oracle_rigid(Fh, els)
    assert np.abs(mean.cpu().numpy() - wmean).max() <= TOL


def test_device_elements_equal_host_elements():
    import ctypes
    F = frames_of(12, 96, 128).numpy()
    els = rigid_elems(11, np.random.default_rng(11))
    arr = B.elem_array(els)
    raw = torch.empty(ctypes.sizeof(arr), dtype=torch.uint8)
    ctypes.memmove(raw.data_ptr(), ctypes.addressof(arr), ctypes.sizeof(arr))
    ctx = B.Context(B.Config())
    o1, m1 = run_warp(ctx, F, elems=els)
    o2, m2 = run_warp(ctx, F, elems=raw.cuda())
    assert np.array_equal(o1, o2) and np.array_equal(m1, m2)
