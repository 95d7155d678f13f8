"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: |phi_gpu(x) - phi_oracle(x)| <= 0.02 px at every finest-level pixel and
relative energy error <= 1e-5 for FP32 storage; <= 0.1 px for BF16/FP16
storage.  Kernel-level steps (pyramid, energy/gradient, composition) are
compared element by element with tolerances derived from FP32 arithmetic.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_12478_gb300 import binding as B
from paper_2010_12478_gb300 import synth

pytestmark = pytest.mark.gpu

PX_TOL = 0.02
E_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_12478_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def ctx_of(**kw):
    return B.Context(B.Config(**kw))


def ocfg(cfg: B.Config) -> O.Config:
    return O.Config(levels=cfg.levels, max_iter=cfg.max_iter, max_rejects=cfg.max_rejects, tol_grad=cfg.tol_grad,
                    tol_rel_e=cfg.tol_rel_e, armijo_c=cfg.armijo_c, tau0=cfg.tau0, step_cap=cfg.step_cap,
                    lam=cfg.lam, mode=cfg.mode, grid=cfg.grid, metric=cfg.metric,
                    sigma=cfg.sigma,
                    tol_coarse=cfg.tol_coarse)


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-12)


# ------------------------------------------------------------------ kernel-level steps
@pytest.mark.parametrize("shape", [(64, 64), (45, 67), (3, 5)])
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_pyramid_matches_oracle(shape, storage):
    H, W = shape
    levels = 2 if min(H, W) < 8 else 3
    img = np.random.default_rng(1).uniform(0, 1, size=(H, W)).astype(np.float32)
    ctx = ctx_of()
    sizes = []
    h, w = H, W
    for _ in range(levels):
        sizes.append((h, w))
        h, w = (h + 1) // 2, (w + 1) // 2
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[storage]
    out = torch.zeros(sum(a * b for a, b in sizes), dtype=dt, device="cuda")
    ctx.pyramid(torch.from_numpy(img).cuda(), levels, storage, out)
    got = out.float().cpu().numpy()
    levels_got, off = [], 0
    for (h, w) in sizes:
        levels_got.append(got[off:off + h * w].reshape(h, w).astype(np.float64))
        off += h * w
    tol = {"f32": 3e-7, "bf16": 8e-3, "f16": 1e-3}[storage]
    np.testing.assert_allclose(levels_got[0], img.astype(np.float64), rtol=tol, atol=tol)
    for l in range(1, levels):
        # the oracle's box average of the GPU's previous level as stored (storage rounding is part of the path)
        np.testing.assert_allclose(levels_got[l], O.downsample(levels_got[l - 1]), rtol=tol, atol=tol)


def test_rigid_energy_and_gradient_match_oracle():
    R, T = synth.rigid_pair(97, 131, 0.01, (1.3, -0.8), noise_snr=8.0, seed=3)
    ctx = ctx_of()
    for th in ([0.0, 0.0, 0.0], [0.012, 1.1, -0.7], [-0.02, 2.5, 3.1], [0.0, 0.25, 0.5]):
        Eg, gg = ctx.energy_rigid(torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda(), th)
        Eo, go = O.rigid_energy(R, T, th)
        assert rel(Eg, Eo) <= 1e-6
        assert np.abs(gg - go).max() <= 1e-4 * max(1.0, np.abs(go).max()), (gg, go)


@pytest.mark.parametrize("grid", [8, 12, 16, 24])
def test_grid_energy_and_gradient_match_oracle(grid):
    H, W = 53, 71
    R, T = synth.translated_pair(H, W, (0.7, -0.4), noise_snr=8.0, seed=4)
    g = O.grid_for(W, H, grid)
    assert B.grid_dims(W, H, grid, 1) == (g.nx, g.ny, g.s)
    c = np.random.default_rng(5).uniform(-0.5, 0.5, size=(2, g.ny, g.nx)) + 0.3
    ctx = ctx_of(mode="nonrigid", lam=3.0, grid=grid)
    cd = torch.from_numpy(np.ascontiguousarray(c.transpose(1, 2, 0)).astype(np.float32)).cuda()
    gd = torch.zeros((g.ny, g.nx, 2), device="cuda")
    Eg = ctx.energy_grid(torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda(), cd, gd)
    Eo, go = O.grid_energy(R, T, 0, g, cd.cpu().numpy().transpose(2, 0, 1).astype(np.float64), 3.0)
    assert rel(Eg, Eo) <= 1e-6
    np.testing.assert_allclose(gd.cpu().numpy().transpose(2, 0, 1), go, atol=2e-4 * np.abs(go).max())


def test_compose_grid_matches_oracle():
    H, W = 40, 33
    g = O.grid_for(W, H, 8)
    rng = np.random.default_rng(6)
    c1 = rng.uniform(-3, 3, size=(g.ny, g.nx, 2)).astype(np.float32)
    c2 = rng.uniform(-3, 3, size=(g.ny, g.nx, 2)).astype(np.float32)
    ctx = ctx_of(mode="nonrigid", grid=8)
    out = torch.zeros((g.ny, g.nx, 2), device="cuda")
    ctx.compose_grid(torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda(), W, H, out)
    ref = O.compose_grid(g, c1.transpose(2, 0, 1), c2.transpose(2, 0, 1))
    np.testing.assert_allclose(out.cpu().numpy().transpose(2, 0, 1), ref, atol=2e-5)


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_identical_frames_give_exact_identity(mode):
    R, _ = synth.translated_pair(96, 80, (0, 0), noise_snr=10.0, seed=7)
    cfg = B.Config(mode=mode)
    ctx = B.Context(cfg)
    Rt = torch.from_numpy(R).cuda()
    fo = torch.full((2, 96, 80), 7.0, device="cuda")
    (i, k, a, gx, gy), st = ctx.pairwise(Rt, Rt.clone(), field_out=fo)
    assert (a, gx, gy) == (0.0, 0.0, 0.0)
    assert st["iters"] == [0, 0] and st["energy"] == 0.0
    if mode == "nonrigid":
        assert not fo.any()


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("case", range(4))
def test_pairwise_rigid_matches_oracle(cluster, case):
    rng = np.random.default_rng(20 + case)
    H, W = [(128, 128), (97, 131), (64, 200), (33, 47)][case]
    s = rng.uniform(-3, 3, 2)
    R, T = synth.rigid_pair(H, W, rng.uniform(-0.01, 0.01), s, noise_snr=[None, 10.0, 5.0, 10.0][case], seed=case)
    cfg = B.Config(cluster=cluster)
    ctx = B.Context(cfg)
    (i, k, a, gx, gy), st = ctx.pairwise(torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda())
    th_o, st_o = O.register_rigid(O.pyramid(R, 2), O.pyramid(T, 2), np.zeros(3), ocfg(cfg))
    err = O.max_px_error(np.array(st["theta"]), th_o, H, W, "rigid")
    assert err <= PX_TOL, (st, st_o, th_o)
    assert rel(st["energy"], st_o.energy) <= E_TOL


def test_pairwise_rigid_with_initial_guess_matches_oracle():
    R, T = synth.rigid_pair(128, 96, 0.004, (9.7, -6.2), noise_snr=10.0, seed=9)
    cfg = B.Config()
    ctx = B.Context(cfg)
    init = [0.002, 8.9, -5.5]
    _, st = ctx.pairwise(torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda(), init=init)
    th_o, st_o = O.register_rigid(O.pyramid(R, 2), O.pyramid(T, 2), np.array(init, np.float32).astype(np.float64),
                                  ocfg(cfg))
    assert O.max_px_error(np.array(st["theta"]), th_o, 128, 96, "rigid") <= PX_TOL


@pytest.mark.parametrize("cluster,grid", [(1, 0), (4, 0), (4, 12)])
def test_pairwise_nonrigid_matches_oracle(cluster, grid):
    ser = synth.make_series(synth.SeriesSpec(2, 96, 112, step=2.0, field_amp=1.0, snr=(10, 10),
                                             field_rate=(0.8, 1.2), seed=11))
    F = ser.frames.numpy()
    cfg = B.Config(mode="nonrigid", cluster=cluster, grid=grid)
    ctx = B.Context(cfg)
    fo = torch.zeros((2, 96, 112), device="cuda")
    _, st = ctx.pairwise(torch.from_numpy(F[0]).cuda(), torch.from_numpy(F[1]).cuda(), field_out=fo)
    c_o, st_o = O.register_nonrigid(O.pyramid(F[0], 2), O.pyramid(F[1], 2), None, ocfg(cfg))
    err = O.max_px_error(fo.cpu().numpy(), c_o, 96, 112, "nonrigid", grid)
    assert err <= PX_TOL, (err, st, st_o)
    assert rel(st["energy"], st_o.energy) <= E_TOL


# ------------------------------------------------------------------ scans
def c1_frames(n=16, seed=1410):
    spec = synth.spec_c1(seed)
    spec.n_frames = n
    return synth.make_series(spec).frames.numpy()


def oracle_scan(F, cfg, schedule):
    oc = ocfg(cfg)
    return O.scan(F, oc, O.DAGS[schedule](len(F) - 1))


@pytest.mark.parametrize("schedule", ["sequential", "brent_kung", "dissemination", "ladner_fischer"])
@pytest.mark.parametrize("exec_", ["plain", "level", "persistent", "graph"])
def test_scan_rigid_c1_matches_oracle(schedule, exec_):
    F = c1_frames()
    cfg = B.Config()
    ctx = B.Context(cfg)
    els, st = ctx.scan(torch.from_numpy(F).cuda(), schedule=schedule, exec=exec_)
    ref = oracle_scan(F, cfg, schedule)
    for i, (e, o) in enumerate(zip(els, ref)):
        assert (e[0], e[1]) == (o.i, o.k) == (0, i + 1)
        err = O.max_px_error(np.array(e[2:]), o.phi, 128, 128, "rigid")
        assert err <= PX_TOL, (i, e, o.phi)
    # every operator's energy (leaves first, then B in DAG order)
    n = len(F) - 1
    leaves = [O.op_A([O.pyramid(f, 2) for f in F], j, j + 1, ocfg(cfg)) for j in range(2)]
    for j in range(2):
        assert rel(st[j]["energy"], leaves[j].stats.energy) <= E_TOL
    assert len(st) == n + B.scan_work(schedule, n)


def test_scan_host_frames_equal_device_frames():
    F = c1_frames(9)
    ctx = B.Context(B.Config())
    a, _ = ctx.scan(torch.from_numpy(F).cuda())
    b, _ = ctx.scan(np.ascontiguousarray(F))
    assert a == b


@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_scan_staging_paths_agree(mode):
    # device frames (no staging), page-locked frames (the SMs read them over the link: also a view
    # that starts inside its allocation), pageable frames, and page-locked frames whose size or
    # start is not a multiple of 16 bytes (both cudaMemcpyAsync) give bit-identical scans
    ctx = B.Context(B.Config(mode=mode, cluster=2))
    ctx.set_timing(True)
    cases = []
    spec = synth.spec_c1()
    spec.n_frames, spec.H, spec.W = 7, 67, 93        # 7 * 67 * 93 * 4 bytes: not a multiple of 16
    odd = synth.make_series(spec).frames
    F = torch.from_numpy(c1_frames(9))
    pinned = torch.empty((11,) + F.shape[1:], pin_memory=True)
    pinned[2:] = F
    flat = torch.empty(F.numel() + 1, pin_memory=True)
    flat[1:] = F.reshape(-1)
    for frames, path in ((F.cuda(), 0), (F.clone().pin_memory(), 2), (pinned[2:], 2), (F.numpy(), 1),
                         (flat[1:].view(F.shape), 1)):
        el, st = ctx.scan(frames, exec="persistent")
        t = ctx.last_timing()
        assert t["h2d_path"] == path
        assert (t["h2d_ms"] > 0) == (path > 0)
        cases.append((el, [x["evals"] for x in st]))
    assert all(c == cases[0] for c in cases[1:])
    a, _ = ctx.scan(odd.cuda(), exec="persistent")
    b, _ = ctx.scan(odd.pin_memory(), exec="persistent")
    assert ctx.last_timing()["h2d_path"] == 1
    assert a == b


def test_scan_is_deterministic_and_independent_of_executor():
    F = c1_frames(12)
    ctx = B.Context(B.Config(cluster=2))
    runs = [ctx.scan(torch.from_numpy(F).cuda(), exec=e)[0] for e in ("level", "level", "plain", "persistent", "graph")]
    assert runs[0] == runs[1] == runs[2] == runs[3] == runs[4]


def test_graph_executor_replays_the_captured_plan():
    # the first call captures, repeats with the same plan replay; a new N or new frames in the
    # same buffers give the same results as the one-launch-per-operator path
    ctx = B.Context(B.Config(cluster=2))
    ctx.set_timing(True)
    F = torch.from_numpy(c1_frames(10)).cuda()
    a, sa = ctx.scan(F, exec="graph")
    assert ctx.last_timing()["graph_captures"] == 1
    assert ctx.last_timing()["op_launches"] == len(sa)
    b, sb = ctx.scan(F, exec="graph")
    assert ctx.last_timing()["graph_captures"] == 0
    assert a == b and [s["evals"] for s in sa] == [s["evals"] for s in sb]
    F2 = torch.flip(F, dims=[0]).contiguous()
    c, _ = ctx.scan(F2, exec="graph")
    assert ctx.last_timing()["graph_captures"] == 0   # same plan and workspaces, new frame data
    assert c == ctx.scan(F2, exec="plain")[0]
    d, _ = ctx.scan(F[:7].contiguous(), exec="graph")
    assert ctx.last_timing()["graph_captures"] == 1   # another N: another plan
    assert d == ctx.scan(F[:7].contiguous(), exec="plain")[0]


@pytest.mark.parametrize("exec_", ["level", "persistent", "graph"])
def test_scan_nonrigid_c1_matches_oracle(exec_):
    F = c1_frames(6)
    cfg = B.Config(mode="nonrigid")
    ctx = B.Context(cfg)
    n = len(F) - 1
    fo = torch.zeros((n, 2, 128, 128), device="cuda")
    els, st = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec=exec_, fields_out=fo)
    ref = oracle_scan(F, cfg, "brent_kung")
    got = fo.cpu().numpy()
    for i, o in enumerate(ref):
        err = O.max_px_error(got[i], o.phi, 128, 128, "nonrigid")
        assert err <= PX_TOL, (i, err)


@pytest.mark.parametrize("unroll,ctas_per_sm", [(2, 3), (4, 4), (2, 4)])
def test_scan_nonrigid_c1_tile_shapes_match_oracle(unroll, ctas_per_sm):
    """Every register form and energy-pass unroll the autotuner may choose, against the oracle."""
    F = c1_frames(6)
    cfg = B.Config(mode="nonrigid", cluster=4, unroll=unroll, ctas_per_sm=ctas_per_sm)
    ctx = B.Context(cfg)
    ctx.set_timing(True)
    n = len(F) - 1
    fo = torch.zeros((n, 2, 128, 128), device="cuda")
    ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec="persistent", fields_out=fo)
    t = ctx.last_timing()
    assert (t["cluster"], t["unroll"], t["ctas_per_sm"]) == (4, unroll, ctas_per_sm)
    ref = oracle_scan(F, cfg, "brent_kung")
    got = fo.cpu().numpy()
    for i, o in enumerate(ref):
        err = O.max_px_error(got[i], o.phi, 128, 128, "nonrigid")
        assert err <= PX_TOL, (i, err)


@pytest.mark.parametrize("sigma", [1.0, 2.5])
@pytest.mark.parametrize("exec_", ["persistent", "plain"])
def test_scan_nonrigid_h1_matches_oracle(sigma, exec_):
    """The H1 scalar product (the gradient smoothed over sigma grid spacings): the cosine-transform
    solve of the kernels against the oracle's banded Cholesky, through a whole nonrigid scan."""
    F = c1_frames(6)
    cfg = B.Config(mode="nonrigid", metric=B.METRIC_H1, sigma=sigma, cluster=4)
    ctx = B.Context(cfg)
    n = len(F) - 1
    fo = torch.zeros((n, 2, 128, 128), device="cuda")
    _, st = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec=exec_, fields_out=fo)
    ref = oracle_scan(F, cfg, "brent_kung")
    got = fo.cpu().numpy()
    for i, o in enumerate(ref):
        err = O.max_px_error(got[i], o.phi, 128, 128, "nonrigid")
        assert err <= PX_TOL, (i, err)
    # no level ran out of steps (the gradient norm, or a line search at the FP32 floor, ends each)
    assert all(v != B.REG_STOP_MAXIT for s in st for v in s["stop"])


def test_h1_pairwise_at_512_matches_oracle():
    """A neighbour operator on a 512^2 lattice pair (33 x 33 control points) with the H1 product."""
    spec = synth.spec_c2()
    spec.n_frames = 2
    F = synth.make_series(spec).frames.numpy()
    cfg = B.Config(mode="nonrigid", metric=B.METRIC_H1, sigma=1.0)
    ctx = B.Context(cfg)
    fo = torch.zeros((2, 512, 512), device="cuda")
    ctx.pairwise(torch.from_numpy(F[0]).cuda(), torch.from_numpy(F[1]).cuda(), field_out=fo)
    oc = ocfg(cfg)
    o = O.op_A({0: O.pyramid(F[0], oc.levels), 1: O.pyramid(F[1], oc.levels)}, 0, 1, oc)
    assert O.max_px_error(fo.cpu().numpy(), o.phi, 512, 512, "nonrigid") <= PX_TOL


@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_scan_c1_with_the_coarse_stop_factor_one_matches_oracle(mode):
    """tol_coarse reaches both controllers: with factor 1 (every level to tol_grad) the scan still
    matches the oracle run with the same factor."""
    F = c1_frames(6)
    cfg = B.Config(mode=mode, tol_coarse=1.0, cluster=4)
    ctx = B.Context(cfg)
    n = len(F) - 1
    if mode == "rigid":
        els, _ = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec="persistent")
    else:
        fo = torch.zeros((n, 2, 128, 128), device="cuda")
        els, _ = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec="persistent", fields_out=fo)
    ref = oracle_scan(F, cfg, "brent_kung")
    for i, o in enumerate(ref):
        got = np.array(els[i][2:]) if mode == "rigid" else fo[i].cpu().numpy()
        assert O.max_px_error(got, o.phi, 128, 128, mode) <= PX_TOL, (i, mode)


def test_scan_two_frames():
    F = c1_frames(2)
    ctx = B.Context(B.Config())
    els, st = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung")
    o = oracle_scan(F, B.Config(), "brent_kung")[0]
    assert len(els) == 1 and O.max_px_error(np.array(els[0][2:]), o.phi, 128, 128, "rigid") <= PX_TOL


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_precision_storage_within_tenth_pixel(storage):
    F = c1_frames(8)
    cfg = B.Config(storage=storage)
    ctx = B.Context(cfg)
    els, _ = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung")
    ref = oracle_scan(F, B.Config(), "brent_kung")
    for e, o in zip(els, ref):
        assert O.max_px_error(np.array(e[2:]), o.phi, 128, 128, "rigid") <= 0.1


def test_invalid_arguments_are_rejected():
    ctx = B.Context(B.Config(levels=3))
    F = torch.zeros((3, 6, 6), device="cuda")
    els, st = ctx.scan(F)   # 6x6 at 3 levels has a 2x2 coarsest level: allowed (constant frames: E = 1)
    assert all(s["energy"] == 1.0 for s in st)
    F = torch.zeros((3, 5, 5), device="cuda")   # 5 -> 3 -> 2 is fine, 3 levels of 3x3 are not
    F = torch.zeros((3, 3, 3), device="cuda")
    with pytest.raises(B.RegError) as e:
        ctx.scan(F)
    assert e.value.code == B.REG_EINVAL
    # a series of one frame has nothing to register
    with pytest.raises(B.RegError) as e:
        ctx.scan(torch.zeros((1, 32, 32), device="cuda"))
    assert e.value.code == B.REG_EINVAL
    with pytest.raises(B.RegError) as e:
        ctx.scan_batch(torch.zeros((2, 1, 32, 32), device="cuda"))
    assert e.value.code == B.REG_EINVAL


@pytest.mark.parametrize("H,W", [(2048, 2048), (1024, 4096)])
def test_large_frames_energy_and_gradient_match_oracle(H, W):
    # the largest control grids (65 points per axis; spacing 32 and 64, the latter with cells
    # wider than a warp) at one evaluation: energy and control-point gradient
    R, T = synth.translated_pair(H, W, (1.3, -0.6), noise_snr=10.0, seed=9)
    g = O.grid_for(W, H)
    assert (g.nx <= 65 and g.ny <= 65) and B.grid_dims(W, H, 0, 1) == (g.nx, g.ny, g.s)
    c = np.random.default_rng(6).uniform(-0.5, 0.5, size=(2, g.ny, g.nx)) + np.array([1.2, -0.5])[:, None, None]
    ctx = ctx_of(mode="nonrigid", lam=2.0)
    cd = torch.from_numpy(np.ascontiguousarray(c.transpose(1, 2, 0)).astype(np.float32)).cuda()
    gd = torch.zeros((g.ny, g.nx, 2), device="cuda")
    Eg = ctx.energy_grid(torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda(), cd, gd)
    Eo, go = O.grid_energy(R, T, 0, g, cd.cpu().numpy().transpose(2, 0, 1).astype(np.float64), 2.0)
    assert rel(Eg, Eo) <= 1e-6
    np.testing.assert_allclose(gd.cpu().numpy().transpose(2, 0, 1), go, atol=2e-4 * np.abs(go).max())


# ------------------------------------------------------------------ full size (256 x 512^2), sampled
def test_c2_full_size_sampled_operators_match_oracle():
    # the benchmark's launch configuration: one operator per launch, 16 CTAs per operator
    sampled_rigid_scan_parity(synth.spec_c2(), "plain", 16)


def test_c3_full_size_sampled_operators_match_oracle():
    # 4,096 frames with uneven iteration counts (SNR 3-20, 5 % jumps) through the persistent
    # device queue, in the launch shape the batched form uses
    sampled_rigid_scan_parity(synth.spec_c3(), "persistent", 16)


def sampled_rigid_scan_parity(spec, exec_, cluster):
    ser = synth.make_series(spec, device="cuda")
    frames = ser.frames
    cfg = B.Config(cluster=cluster)
    ctx = B.Context(cfg)
    n = spec.n_frames - 1
    els, st = ctx.scan(frames, schedule="brent_kung", exec=exec_)
    ops, out = B.scan_dag("brent_kung", n)
    Fh = frames.cpu().numpy()
    oc = ocfg(cfg)
    pyr = {}

    def P(i):
        if i not in pyr:
            pyr[i] = O.pyramid(Fh[i], cfg.levels)
        return pyr[i]

    node = [None] * (n + len(ops))
    for j in range(n):
        node[j] = O.Elem(st[j]["i"], st[j]["k"], np.array(st[j]["theta"]))
    for j, (l, r) in enumerate(ops):
        node[n + j] = O.Elem(st[n + j]["i"], st[n + j]["k"], np.array(st[n + j]["theta"]))
    rng = np.random.default_rng(1410)
    # leaves: A from the frames; B: from the GPU's exact input elements
    for j in rng.choice(n, 2, replace=False):
        th, so = O.register_rigid(P(j), P(j + 1), np.zeros(3), oc)
        assert O.max_px_error(node[j].phi, th, 512, 512, "rigid") <= PX_TOL
        assert rel(st[j]["energy"], so.energy) <= E_TOL
    for j in rng.choice(len(ops), 3, replace=False):
        l, r = ops[j]
        e = O.op_B(node[l], node[r], {node[l].i: P(node[l].i), node[r].k: P(node[r].k)}, oc)
        assert O.max_px_error(node[n + j].phi, e.phi, 512, 512, "rigid") <= PX_TOL
        assert rel(st[n + j]["energy"], e.stats.energy) <= E_TOL
    # the prefixes are the sequential recursion at sampled points (Sec. 3)
    for i in rng.choice(n - 1, 2, replace=False):
        a = O.op_A({i + 1: P(i + 1), i + 2: P(i + 2)}, i + 1, i + 2, oc)
        prev = O.Elem(0, i + 1, np.array(els[i][2:], dtype=np.float64))
        e = O.op_B(prev, a, {0: P(0), i + 2: P(i + 2)}, oc)
        assert O.max_px_error(np.array(els[i + 1][2:], dtype=np.float64), e.phi, 512, 512, "rigid") <= PX_TOL


def grid_init_as_sampled(g, c, H, W):
    """Control values the library derives from a dense initial field (reg_pairwise's field_in):
    the float32 field of c at the control points, clamped into the frame."""
    dense = O.grid_dense(g, c).astype(np.float32)
    ys = np.minimum(np.arange(g.ny) * g.s, H - 1)
    xs = np.minimum(np.arange(g.nx) * g.s, W - 1)
    return dense, dense[:, ys][:, :, xs].astype(np.float64)


def c2_nonrigid_operator_cases(frames, Fh, cfg, n_sets, seed):
    """A(f_i, f_i+1) and B over (f_i, f_i+2) from the composition of the oracle's A's, at 512^2:
    (reference, template, dense initial field or None, oracle result)."""
    oc = ocfg(cfg)
    g = O.grid_for(512, 512)
    rng = np.random.default_rng(seed)
    out = []
    for i in rng.choice(frames.shape[0] - 2, n_sets, replace=False):
        P = {j: O.pyramid(Fh[j], cfg.levels) for j in (i, i + 1, i + 2)}
        a1, a2 = O.op_A(P, i, i + 1, oc), O.op_A(P, i + 1, i + 2, oc)
        out.append((i, i + 1, None, a1))
        dense, init = grid_init_as_sampled(g, O.compose_grid(g, a1.phi, a2.phi), 512, 512)
        phi, so = O.register_nonrigid(P[i], P[i + 2], init, oc)
        out.append((i, i + 2, dense, O.Elem(i, i + 2, phi, so)))
    return out


def test_c2_full_size_nonrigid_operators_match_oracle():
    # A and B at 512 x 512 through reg_pairwise in the scan's launch shape (16 CTAs), against the
    # oracle from the same initial control values
    spec = synth.spec_c2()
    frames = synth.make_series(spec, device="cuda").frames
    Fh = frames.cpu().numpy()
    cfg = B.Config(mode="nonrigid", cluster=16)
    ctx = B.Context(cfg)
    for i, k, dense, ref in c2_nonrigid_operator_cases(frames, Fh, cfg, 4, 2010):
        u = torch.empty((2, 512, 512), device="cuda")
        fin = torch.from_numpy(dense).cuda() if dense is not None else None
        _, st = ctx.pairwise(frames[i].contiguous(), frames[k].contiguous(), field_in=fin, field_out=u)
        err = O.max_px_error(u.cpu().numpy(), ref.phi, 512, 512, "nonrigid")
        assert err <= PX_TOL, (i, k, err, st["stop"], list(ref.stats.stop))
        assert rel(st["energy"], ref.stats.energy) <= E_TOL, (i, k)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_c2_full_size_nonrigid_reduced_precision_within_tenth_pixel(storage):
    # pyramids stored in 2-byte floats: A and B at 512 x 512 against the FP64 oracle of the fp32 frames
    spec = synth.spec_c2()
    frames = synth.make_series(spec, device="cuda").frames
    Fh = frames.cpu().numpy()
    cfg = B.Config(mode="nonrigid", cluster=16, storage=storage)
    ctx = B.Context(cfg)
    for i, k, dense, ref in c2_nonrigid_operator_cases(frames, Fh, B.Config(mode="nonrigid"), 3, 2011):
        u = torch.empty((2, 512, 512), device="cuda")
        fin = torch.from_numpy(dense).cuda() if dense is not None else None
        ctx.pairwise(frames[i].contiguous(), frames[k].contiguous(), field_in=fin, field_out=u)
        assert O.max_px_error(u.cpu().numpy(), ref.phi, 512, 512, "nonrigid") <= 0.1, (storage, i, k)


def test_nonrigid_plain_scan_at_512_matches_oracle_brent_kung():
    # the benchmark's launch shape end to end: one operator per launch on the stream pool, 16 CTAs
    # per operator, 512 x 512 frames, every prefix of the Brent-Kung scan against the oracle's
    spec = synth.spec_c2(n_frames=16)
    frames = synth.make_series(spec, device="cuda").frames
    F = frames.cpu().numpy()
    cfg = B.Config(mode="nonrigid", cluster=16)
    ctx = B.Context(cfg)
    n = F.shape[0] - 1
    nx, ny, _ = B.grid_dims(512, 512)
    els, st = ctx.scan(frames, schedule="brent_kung", exec="plain", want_stats=True)
    grids = torch.zeros((n, ny, nx, 2), device="cuda")
    assert ctx.scan_grids(grids) == n
    ref = oracle_scan(F, cfg, "brent_kung")
    got = grids.cpu().numpy().astype(np.float64)
    _, out_node = B.scan_dag("brent_kung", n)   # per-operator stats are indexed by the node they produce
    for i, o in enumerate(ref):
        assert (els[i][0], els[i][1]) == (o.i, o.k) == (0, i + 1)
        err = O.max_px_error(np.transpose(got[i], (2, 0, 1)), o.phi, 512, 512, "nonrigid")
        assert err <= PX_TOL, (i, err)
        assert rel(st[out_node[i]]["energy"], o.stats.energy) <= E_TOL, i


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_nonrigid_reduced_precision_scan_within_tenth_pixel(storage):
    F = c1_frames(8)
    cfg = B.Config(mode="nonrigid", storage=storage)
    ctx = B.Context(cfg)
    n = len(F) - 1
    fo = torch.zeros((n, 2, 128, 128), device="cuda")
    ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec="persistent", fields_out=fo)
    ref = oracle_scan(F, B.Config(mode="nonrigid"), "brent_kung")
    got = fo.cpu().numpy()
    for i, o in enumerate(ref):
        assert O.max_px_error(got[i], o.phi, 128, 128, "nonrigid") <= 0.1, (storage, i)


@pytest.mark.parametrize("exec_", ["persistent", "level", "plain"])
def test_scan_batch_equals_per_series_scans(exec_):
    # independent series registered together give each series' own scan, bit for bit
    series = [c1_frames(7, seed) for seed in (1410, 1411, 1412)]
    for mode in ("rigid", "nonrigid"):
        ctx = B.Context(B.Config(mode=mode, cluster=4))
        Fb = torch.from_numpy(np.stack(series)).cuda()
        els_b, st_b = ctx.scan_batch(Fb, schedule="brent_kung", exec=exec_)
        if mode == "nonrigid":
            nx, ny, _ = B.grid_dims(128, 128)
            gb = torch.zeros((3, 6, ny, nx, 2), device="cuda")
            assert ctx.scan_grids(gb) == 18
        for q, F in enumerate(series):
            els, st = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec=exec_)
            assert els_b[q] == els
            assert [s["energy"] for s in st_b[q]] == [s["energy"] for s in st]
            assert [(s["i"], s["k"]) for s in st_b[q]] == [(s["i"], s["k"]) for s in st]
            if mode == "nonrigid":
                g1 = torch.zeros((6, ny, nx, 2), device="cuda")
                ctx.scan_grids(g1)
                assert torch.equal(g1, gb[q])
        # the same batch from page-locked host memory (staged by the SMs)
        ctx.set_timing(True)
        els_h, st_h = ctx.scan_batch(Fb.cpu().pin_memory(), schedule="brent_kung", exec=exec_)
        assert ctx.last_timing()["h2d_path"] == 2
        ctx.set_timing(False)
        assert els_h == els_b
        assert [[s["energy"] for s in x] for x in st_h] == [[s["energy"] for s in x] for x in st_b]


def test_pitched_frames_and_odd_grid_spacing_through_the_c_abi():
    # frames with a row pitch larger than W (and not a multiple of 4: no TMA staging in the
    # warp), and a control-grid spacing that is not a power of two
    import ctypes
    F = c1_frames(5)                       # [5, 128, 128]
    N, H, W = F.shape
    pitch = W + 3
    Fp = np.zeros((N, H, pitch), np.float32)
    Fp[:, :, :W] = F
    dF = torch.from_numpy(Fp).cuda()
    for mode, grid in (("rigid", 0), ("nonrigid", 12)):
        ctx = B.Context(B.Config(mode=mode, grid=grid))
        out = (B.reg_elem_t * (N - 1))()
        nx, ny, _ = B.grid_dims(W, H, grid)
        fo = torch.zeros((N - 1, 2, H, W), device="cuda") if mode == "nonrigid" else None
        rc = B.lib().reg_scan(ctx.h, ctypes.cast(ctypes.c_void_p(dF.data_ptr()), ctypes.POINTER(ctypes.c_float)),
                              N, W, H, pitch, B.SCHEDULES["brent_kung"], B.EXECS["persistent"],
                              ctypes.addressof(out), B._ptr(fo), None, None)
        assert rc == B.REG_OK
        ref_els, _ = ctx.scan(torch.from_numpy(F).cuda(), schedule="brent_kung", exec="persistent",
                              fields_out=torch.zeros_like(fo) if fo is not None else None)
        assert [(e.i, e.k, e.alpha, e.gx, e.gy) for e in out] == ref_els
        ref = oracle_scan(F, B.Config(mode=mode, grid=grid), "brent_kung")
        for i, o in enumerate(ref):
            phi = np.array([out[i].alpha, out[i].gx, out[i].gy]) if mode == "rigid" else fo[i].cpu().numpy()
            assert O.max_px_error(phi, o.phi, H, W, mode, grid) <= PX_TOL
        # the registered series from pitched frames (global-memory sampling path)
        if mode == "rigid":
            o1 = torch.zeros((N, H, W), device="cuda")
            arr = B.elem_array(ref_els)
            rc = B.lib().reg_warp(ctx.h, ctypes.cast(ctypes.c_void_p(dF.data_ptr()), ctypes.POINTER(ctypes.c_float)),
                                  N, W, H, pitch, arr, None, B._ptr(o1), None, None)
            assert rc == B.REG_OK
            o2 = torch.zeros((N, H, W), device="cuda")
            ctx.warp(torch.from_numpy(F).cuda(), elems=ref_els, out=o2)
            # the TMA-staged and the global-memory samplers round differently in the last bit
            assert (o1 - o2).abs().max().item() <= 1e-5


def test_c2_full_size_nonrigid_scan_sampled_nodes_match_oracle():
    # the whole c2 nonrigid scan (256 x 512^2) in the benchmark's launch shape; sampled leaves
    # against the oracle's A, sampled B operators against the oracle's B fed the GPU's exact inputs
    spec = synth.spec_c2()
    frames = synth.make_series(spec, device="cuda").frames
    Fh = frames.cpu().numpy()
    cfg = B.Config(mode="nonrigid", cluster=16)
    oc = ocfg(cfg)
    ctx = B.Context(cfg)
    n = spec.n_frames - 1
    els, st = ctx.scan(frames, schedule="brent_kung", exec="plain")
    ops, out_node = B.scan_dag("brent_kung", n)
    nx, ny, _ = B.grid_dims(512, 512)
    rng = np.random.default_rng(1411)
    leaves = [int(j) for j in rng.choice(n, 2, replace=False)]
    bops = [int(j) for j in rng.choice(len(ops), 3, replace=False)]
    want = leaves + [n + j for j in bops] + [v for j in bops for v in ops[j]]
    gd = torch.zeros((len(want), ny, nx, 2), device="cuda")
    ctx.scan_node_grids(want, gd)
    grid_of = {w: np.transpose(gd[q].cpu().numpy().astype(np.float64), (2, 0, 1)) for q, w in enumerate(want)}
    pyr = {}

    def P(i):
        if i not in pyr:
            pyr[i] = O.pyramid(Fh[i], cfg.levels)
        return pyr[i]

    for j in leaves:
        e = O.op_A({j: P(j), j + 1: P(j + 1)}, j, j + 1, oc)
        assert O.max_px_error(grid_of[j], e.phi, 512, 512, "nonrigid") <= PX_TOL, j
        assert rel(st[j]["energy"], e.stats.energy) <= E_TOL, j
    for j in bops:
        l, r = ops[j]
        el = O.Elem(st[l]["i"], st[l]["k"], grid_of[l])
        er = O.Elem(st[r]["i"], st[r]["k"], grid_of[r])
        e = O.op_B(el, er, {el.i: P(el.i), er.k: P(er.k)}, oc)
        assert O.max_px_error(grid_of[n + j], e.phi, 512, 512, "nonrigid") <= PX_TOL, (j, l, r)
        assert rel(st[n + j]["energy"], e.stats.energy) <= E_TOL, j
    # the prefixes are these nodes: scan_grids equals the node grids of the output nodes
    pg = torch.zeros((n, ny, nx, 2), device="cuda")
    ctx.scan_grids(pg)
    sel = [3, n // 2, n - 1]
    g2 = torch.zeros((len(sel), ny, nx, 2), device="cuda")
    ctx.scan_node_grids([out_node[i] for i in sel], g2)
    assert torch.equal(g2, pg[sel])


@pytest.mark.parametrize("exec_", ["plain", "level", "persistent"])
def test_split_phases_give_the_same_scan_and_time_both_phases(exec_):
    F = torch.from_numpy(c1_frames(12)).cuda()
    for mode in ("rigid", "nonrigid"):
        ctx = B.Context(B.Config(mode=mode, cluster=4))
        ctx.set_timing(True)
        a, sa = ctx.scan(F, exec=exec_)
        b, sb = ctx.scan(F, exec=exec_, split=True)
        t = ctx.last_timing()
        assert a == b and [s["energy"] for s in sa] == [s["energy"] for s in sb]
        assert t["leaf_ops"] == 11 and t["dag_ops"] == B.scan_work("brent_kung", 11)
        assert t["leaf_ms"] > 0 and t["dag_ms"] > 0
    with pytest.raises(B.RegError) as e:
        ctx.scan(F, exec="graph", split=True)
    assert e.value.code == B.REG_EINVAL


def test_node_grids_end_with_a_pairwise_call():
    F = torch.from_numpy(c1_frames(5)).cuda()
    ctx = B.Context(B.Config(mode="nonrigid"))
    ctx.scan(F, exec="level")
    nx, ny, _ = B.grid_dims(128, 128)
    g = torch.zeros((1, ny, nx, 2), device="cuda")
    ctx.scan_node_grids([0], g)
    with pytest.raises(B.RegError) as e:
        ctx.scan_node_grids([99], g)
    assert e.value.code == B.REG_EINVAL
    ctx.pairwise(F[0].contiguous(), F[1].contiguous(), field_out=torch.zeros((2, 128, 128), device="cuda"))
    with pytest.raises(B.RegError) as e:
        ctx.scan_node_grids([0], g)
    assert e.value.code == B.REG_ESTATE


@pytest.mark.parametrize("cluster,ctas_per_sm", [(4, 3), (8, 4)])
def test_c3_full_size_nonrigid_sampled_operators_match_oracle(cluster, ctas_per_sm):
    # the 4,096-frame nonrigid scan through the persistent device queue, in both launch shapes the
    # autotuner chooses between on this workload (4 CTAs per operator with the 80-register form, 8
    # with the 64-register form); the B operators with the largest drift between their frames
    # (prefixes f_0 -> f_k far down the series, where part of f_0 has no counterpart in f_k) and
    # random ones, against the oracle fed the GPU's exact inputs
    spec = synth.spec_c3()
    ser = synth.make_series(spec, device="cuda")
    frames = ser.frames
    cfg = B.Config(mode="nonrigid", cluster=cluster, ctas_per_sm=ctas_per_sm, unroll=4)
    oc = ocfg(cfg)
    ctx = B.Context(cfg)
    n = spec.n_frames - 1
    els, st = ctx.scan(frames, schedule="brent_kung", exec="persistent")
    ops, _ = B.scan_dag("brent_kung", n)
    ik = np.array([(s["i"], s["k"]) for s in st])
    drift = np.sqrt(((ser.shifts[ik[:, 1]] - ser.shifts[ik[:, 0]]) ** 2).sum(1))
    rng = np.random.default_rng(3)
    bops = [int(np.argmax(np.where(np.arange(len(st)) >= n, drift, -1.0)))]
    bops += [int(v) for v in rng.choice(np.arange(n, len(st)), 2, replace=False)]
    leaves = [int(v) for v in rng.choice(n, 2, replace=False)]
    want = leaves + bops + [v for j in bops for v in ops[j - n]]
    nx, ny, _ = B.grid_dims(512, 512)
    gd = torch.zeros((len(want), ny, nx, 2), device="cuda")
    ctx.scan_node_grids(want, gd)
    grid_of = {w: np.transpose(gd[q].cpu().numpy().astype(np.float64), (2, 0, 1)) for q, w in enumerate(want)}

    def P(i):
        return O.pyramid(frames[i].cpu().numpy(), cfg.levels)

    for j in leaves:
        e = O.op_A({j: P(j), j + 1: P(j + 1)}, j, j + 1, oc)
        assert O.max_px_error(grid_of[j], e.phi, 512, 512, "nonrigid") <= PX_TOL, j
        assert rel(st[j]["energy"], e.stats.energy) <= E_TOL, j
    for j in bops:
        l, r = ops[j - n]
        el = O.Elem(int(ik[l][0]), int(ik[l][1]), grid_of[l])
        er = O.Elem(int(ik[r][0]), int(ik[r][1]), grid_of[r])
        e = O.op_B(el, er, {el.i: P(el.i), er.k: P(er.k)}, oc)
        assert O.max_px_error(grid_of[j], e.phi, 512, 512, "nonrigid") <= PX_TOL, (j, tuple(ik[j]), drift[j])
        assert rel(st[j]["energy"], e.stats.energy) <= E_TOL, j
