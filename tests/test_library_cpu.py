"""Host-side checks of libreg that need no GPU: the library loads, exports every
symbol include/reg.h declares, and its scan DAGs (host C++) equal the oracle's
independently written generators and the paper's work counts."""
import ctypes
import json
import os
import re

import pytest

import oracle as O
from paper_2010_12478_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_12478_gb300 import build
    build.build()
    return B.lib()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "reg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(reg_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(B.EXPORTS) == syms


def test_struct_layouts_match_header(lib):
    assert ctypes.sizeof(B.reg_elem_t) == 20          # 20-byte scan element (Sec. 5)
    assert ctypes.sizeof(B.reg_stats_t) == 144
    assert ctypes.sizeof(B.reg_timing_t) == 80
    cfg = B.reg_config_t()
    lib.reg_config_default(ctypes.byref(cfg))
    assert cfg.levels == 2 and cfg.mode == B.RIGID and cfg.storage == B.F32
    # the stop rule and scalar product of the oracle's configuration: metric gradient norm 3e-5, no
    # relative-decrease test, the Gauss-Newton scalar product for the nonrigid flow
    assert cfg.tol_grad == O.Config().tol_grad == B.Config().tol_grad == 3e-5
    assert cfg.tol_rel_e == O.Config().tol_rel_e == B.Config().tol_rel_e == 0.0
    assert cfg.metric == O.Config().metric == B.Config().metric == 1
    # the launch shape is left to the autotuner unless set
    assert cfg.unroll == 0 and cfg.ctas_per_sm == 0 and B.Config().c().unroll == 0
    # the H1 product's smoothing length
    assert cfg.sigma == O.Config().sigma == B.Config().sigma == 1.0
    # the coarse levels' stop factor
    assert cfg.tol_coarse == O.Config().tol_coarse == B.Config().tol_coarse == 10.0


def test_errors_without_gpu_are_reported_not_crashing(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    h = ctypes.c_void_p()
    rc = lib.reg_ctx_create(None, 0, ctypes.byref(h))
    assert rc == B.REG_ECUDA and not h.value
    assert lib.reg_strerror(rc) == b"CUDA error"
    bad = B.reg_config_t()
    lib.reg_config_default(ctypes.byref(bad))
    bad.levels = 9
    assert lib.reg_ctx_create(ctypes.byref(bad), 0, ctypes.byref(h)) == B.REG_EINVAL
    assert b"levels" in lib.reg_last_error_message()
    for field, value in (("unroll", 3), ("ctas_per_sm", 2), ("metric", 3), ("sigma", -1.0), ("tol_coarse", 0.5)):
        bad = B.reg_config_t()
        lib.reg_config_default(ctypes.byref(bad))
        setattr(bad, field, value)
        assert lib.reg_ctx_create(ctypes.byref(bad), 0, ctypes.byref(h)) == B.REG_EINVAL
        assert field.encode() in lib.reg_last_error_message()


@pytest.mark.parametrize("name", ["sequential", "brent_kung", "dissemination", "ladner_fischer", "lookback2",
                                  "lookback4", "lookback8", "blelloch"])
def test_library_dag_equals_oracle_dag(lib, name):
    for n in list(range(1, 40)) + [255, 256, 1000, 4095]:
        ops, out = B.scan_dag(name, n)
        ref = O.dag_blelloch(n) if name == "blelloch" else O.DAGS[name](n)
        assert ops == [tuple(o) for o in ref.ops], (name, n)
        assert out == ref.out, (name, n)


def test_library_work_counts_match_paper(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "scan_work.json")))
    assert B.scan_work("dissemination", 8) == g["fig2_dissemination_n8"]["work"]
    t5 = g["table5_work"]
    N = t5["N"]
    for P, wd, wl in zip(t5["P"], t5["dissemination"], t5["ladner_fischer"]):
        assert N + (N - P) + B.scan_work("dissemination", P) + N == wd
        assert N + (N - P) + B.scan_work("ladner_fischer", P) + N == wl
    assert B.scan_work("sequential", N) + N == t5["serial"]
    for n in (2, 16, 256, 4096):
        assert B.scan_work("brent_kung", n) == 2 * n - 2 - n.bit_length() + 1
    assert lib.reg_scan_work(99, 10) == -1


@pytest.mark.parametrize("W,H,grid", [(512, 512, 0), (1024, 1024, 0), (2048, 1536, 0), (4096, 4096, 0),
                                      (500, 333, 0), (144, 128, 0), (45, 67, 0), (128, 144, 4),
                                      (512, 512, 12), (512, 512, 24)])
def test_control_grid_matches_oracle_geometry(lib, W, H, grid):
    # the library's control grid (host C++) equals the oracle's independently written rule:
    # spacing 16 doubled until <= 65 points per axis, points cover the frame
    g = O.grid_for(W, H, grid)
    assert B.grid_dims(W, H, grid, 2) == (g.nx, g.ny, g.s)
    assert (g.nx - 1) * g.s >= W - 1 and (g.ny - 1) * g.s >= H - 1
    if grid == 0:
        assert max(g.nx, g.ny) <= 65


def test_control_grid_rejections(lib):
    with pytest.raises(B.RegError) as e:   # spacing must halve exactly at every level
        B.grid_dims(512, 512, 10, 3)
    assert e.value.code == B.REG_EINVAL
    with pytest.raises(B.RegError) as e:
        B.grid_dims(512, 512, -1, 2)
    assert e.value.code == B.REG_EINVAL
    # shared-memory fit of a one-CTA operator: c, d, ct and the band (4 float2 per point) plus
    # one 16-byte control row per warp; 1,000 x 2 points fit, 1,300 x 2 do not
    assert B.grid_dims(1999, 3, 2, 2)[:2] == (1000, 2)
    with pytest.raises(B.RegError) as e:
        B.grid_dims(2599, 3, 2, 2)
    assert e.value.code == B.REG_EINVAL and "shared memory" in str(e.value)
