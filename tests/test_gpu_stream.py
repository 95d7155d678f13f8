"""Streaming service (reg_stream_*): online registration with continuous batching.

An acquisition stream registers each new frame f_i to f_0 by the sequential
recursion phi_{0,i} = B(phi_{0,i-1}, A(f_{i-1}, f_i)) (Sec. 3).  Its results
must equal the sequential scan's, must be the same alone and in a mix with
other streams of other sizes, and must meet the oracle bar.
"""
import threading
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_2010_12478_gb300 import binding as B
from paper_2010_12478_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_12478_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def series(n, H, W, seed):
    spec = synth.SeriesSpec(n, H, W, step=1.5, field_amp=0.8, snr=(10, 10), seed=seed)
    return synth.make_series(spec).frames.numpy()


def run_stream(st, frames, ids, poll_every=1):
    """Submit frames in order (retrying on REG_EBUDGET after polling), collect all results."""
    out = []
    for t, f in enumerate(frames):
        while True:
            rc = st.submit(np.ascontiguousarray(f), ids[t])
            if rc == B.REG_OK:
                break
            assert rc == B.REG_EBUDGET, B.lib().reg_last_error_message()
            out += st.poll(64, 20000)
        if t % poll_every == 0:
            out += st.poll(64, 0)
    while len(out) < len(frames):
        out += st.poll(64, 2_000_000)
    return out


@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_stream_equals_sequential_scan_and_oracle(mode):
    F = series(12, 128, 128, 81)
    cfg = B.Config(mode=mode, cluster=4)
    ctx = B.Context(cfg)
    st = B.Stream(ctx, 128, 128)
    ring = None
    if mode == "nonrigid":
        nx, ny, _ = B.grid_dims(128, 128)
        ring = torch.full((16, ny, nx, 2), 9.0, device="cuda")
        st.set_grids(ring)
    res = run_stream(st, F, list(range(100, 112)))
    st.close()
    assert [r["frame_id"] for r in res] == list(range(100, 112))
    assert res[0]["elem"][2:] == (0.0, 0.0, 0.0)
    els, _ = ctx.scan(torch.from_numpy(F).cuda(), schedule="sequential", exec="plain")
    for i in range(1, 12):
        assert res[i]["elem"] == els[i - 1], (i, res[i], els[i - 1])
        assert res[i]["status"] == 0 and res[i]["done_us"] >= res[i]["submit_us"]
    oc = O.Config(levels=cfg.levels, max_iter=cfg.max_iter, max_rejects=cfg.max_rejects, tol_grad=cfg.tol_grad,
                  tol_rel_e=cfg.tol_rel_e, armijo_c=cfg.armijo_c, tau0=cfg.tau0, step_cap=cfg.step_cap,
                  lam=cfg.lam, mode=cfg.mode, metric=cfg.metric, sigma=cfg.sigma,
                  tol_coarse=cfg.tol_coarse)
    ref = O.scan(F, oc, O.dag_sequential(11))
    if mode == "rigid":
        for i, o in enumerate(ref):
            assert O.max_px_error(np.array(res[i + 1]["elem"][2:], np.float64), o.phi, 128, 128, "rigid") <= 0.02
    else:
        # every frame's control values: the sequential scan's bit for bit, the oracle's within the bar
        sg = torch.zeros((11, ny, nx, 2), device="cuda")
        ctx.scan_grids(sg)
        assert not ring[0].any()                          # f_0: the identity
        assert torch.equal(ring[1:12], sg)
        got = ring[1:12].cpu().numpy().astype(np.float64)
        for i, o in enumerate(ref):
            assert O.max_px_error(np.transpose(got[i], (2, 0, 1)), o.phi, 128, 128, "nonrigid") <= 0.02, i


@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_stream_results_are_the_same_alone_and_in_the_mix(mode):
    F = series(10, 160, 144, 82)
    cfg = B.Config(mode=mode, cluster=4)
    ctx = B.Context(cfg)
    st = B.Stream(ctx, 144, 160)
    alone = run_stream(st, F, list(range(10)))
    st.close()
    # the same stream while three other streams of other sizes share the device
    others = [(series(14, 96, 96, 90 + k), (96, 96)) if k % 2 else (series(14, 256, 192, 90 + k), (192, 256))
              for k in range(3)]
    mixed = {}

    def feed(idx, frames, W, H):
        s2 = B.Stream(ctx, W, H)
        mixed[idx] = run_stream(s2, frames, list(range(len(frames))))
        s2.close()

    ths = [threading.Thread(target=feed, args=(k, fr, W, H)) for k, (fr, (W, H)) in enumerate(others)]
    for t in ths:
        t.start()
    st = B.Stream(ctx, 144, 160)
    mix = run_stream(st, F, list(range(10)))
    st.close()
    for t in ths:
        t.join()
    assert [r["elem"] for r in mix] == [r["elem"] for r in alone]
    assert all(len(mixed[k]) == 14 for k in range(3))


def test_stream_grids_rejections():
    ctx = B.Context(B.Config())
    st = B.Stream(ctx, 64, 64)
    with pytest.raises(B.RegError) as e:
        st.set_grids(torch.zeros((4, 5, 5, 2), device="cuda"))   # rigid stream: no control grids
    assert e.value.code == B.REG_EINVAL
    st.close()
    ctx = B.Context(B.Config(mode="nonrigid"))
    st = B.Stream(ctx, 64, 64)
    nx, ny, _ = B.grid_dims(64, 64)
    with pytest.raises(B.RegError) as e:
        st.set_grids(torch.zeros((4, ny, nx, 2)))               # host memory
    assert e.value.code == B.REG_EINVAL
    run_stream(st, series(2, 64, 64, 84), [0, 1])
    with pytest.raises(B.RegError) as e:
        st.set_grids(torch.zeros((4, ny, nx, 2), device="cuda"))   # after the first submit
    assert e.value.code == B.REG_ESTATE
    st.close()


def test_stream_admission_by_memory_budget_and_poll_timeout():
    ctx = B.Context(B.Config(mem_budget=64 << 20))
    st = B.Stream(ctx, 128, 128)            # fits
    with pytest.raises(B.RegError) as e:
        B.Stream(ctx, 1024, 1024)           # 25 slots of a 1024^2 pyramid do not fit in 64 MB
    assert e.value.code == B.REG_EBUDGET
    t0 = time.time()
    assert st.poll(8, 2000) == []            # nothing submitted: times out, returns nothing
    assert time.time() - t0 < 1.0
    st.close()


def test_stream_submit_refuses_while_every_slot_is_in_flight():
    # 2048^2 frames submitted from device memory, and operators that run until their line search
    # gives up (no gradient stop): a submit takes about a millisecond while one operator of the
    # chain takes far longer, so the slots fill up
    spec = synth.SeriesSpec(60, 2048, 2048, step=1.5, field_amp=0.8, snr=(10, 10), seed=83)
    F = synth.make_series(spec, device="cuda").frames
    ctx = B.Context(B.Config(mode="nonrigid", tol_grad=0.0))
    st = B.Stream(ctx, 2048, 2048)
    codes = [st.submit(F[t], t) for t in range(F.shape[0])]
    # 24 frame slots; 60 frames arrive far faster than the chain of B operators completes
    assert B.REG_EBUDGET in codes
    assert codes[:25] == [B.REG_OK] * 25
    st.close()


@pytest.mark.parametrize("k", [2, 4])
@pytest.mark.parametrize("mode", ["rigid", "nonrigid"])
def test_stream_lookback_equals_the_lookback_scan_and_oracle(k, mode):
    F = series(13, 96, 112, 85)
    cfg = B.Config(mode=mode, cluster=4)
    ctx = B.Context(cfg)
    st = B.Stream(ctx, 112, 96)
    st.set_lookback(k)
    ring = None
    if mode == "nonrigid":
        nx, ny, _ = B.grid_dims(112, 96)
        ring = torch.zeros((16, ny, nx, 2), device="cuda")
        st.set_grids(ring)
    res = run_stream(st, F, list(range(13)))
    st.close()
    assert [r["frame_id"] for r in res] == list(range(13))
    els, _ = ctx.scan(torch.from_numpy(F).cuda(), schedule=f"lookback{k}", exec="plain")
    assert [r["elem"] for r in res[1:]] == els
    oc = O.Config(levels=cfg.levels, mode=mode, metric=cfg.metric)
    ref = O.scan(F, oc, O.dag_lookback(12, k))
    if mode == "nonrigid":
        sg = torch.zeros((12, ny, nx, 2), device="cuda")
        ctx.scan_grids(sg)
        assert torch.equal(ring[1:13], sg)
        got = ring[1:13].cpu().numpy().astype(np.float64)
    for i, o in enumerate(ref):
        phi = np.transpose(got[i], (2, 0, 1)) if mode == "nonrigid" else np.array(res[i + 1]["elem"][2:], np.float64)
        assert O.max_px_error(phi, o.phi, 96, 112, mode) <= 0.02, (k, i)


def test_stream_lookback_rejections():
    ctx = B.Context(B.Config())
    st = B.Stream(ctx, 64, 64)
    with pytest.raises(B.RegError) as e:
        st.set_lookback(3)
    assert e.value.code == B.REG_EINVAL
    run_stream(st, series(2, 64, 64, 86), [0, 1])
    with pytest.raises(B.RegError) as e:
        st.set_lookback(2)
    assert e.value.code == B.REG_ESTATE
    st.close()


def test_stream_refuses_the_h1_product():
    ctx = B.Context(B.Config(mode="nonrigid", metric=B.METRIC_H1))
    with pytest.raises(B.RegError) as e:
        B.Stream(ctx, 128, 128)
    assert e.value.code == B.REG_EINVAL
