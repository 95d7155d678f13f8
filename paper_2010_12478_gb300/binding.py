"""Thin ctypes binding of libreg (the C ABI of include/reg.h).

Argument marshalling only: every step of the registration runs in the
library's CUDA kernels.  Arrays are torch tensors (device or host) or numpy
arrays (host); the binding passes their data pointers.  If libreg.so has not
been built, importing the symbols raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libreg.so")

REG_OK, REG_EINVAL, REG_ENOMEM, REG_EBUDGET, REG_ETIMEOUT, REG_ECUDA, REG_ESTATE = 0, -1, -2, -3, -4, -5, -6
RIGID, NONRIGID = 0, 1
F32, BF16, F16 = 0, 1, 2
SCHEDULES = {"sequential": 0, "brent_kung": 1, "dissemination": 2, "ladner_fischer": 3, "blelloch": 4,
             "lookback2": 17, "lookback4": 18, "lookback8": 19}
EXECS = {"plain": 0, "level": 1, "persistent": 2, "graph": 3}
SPLIT_PHASES = 0x100   # OR into an executor: A leaves before the first B, phases timed apart
STORAGES = {"f32": F32, "bf16": BF16, "f16": F16}
MAX_LEVELS = 8

# every symbol include/reg.h declares
EXPORTS = ["reg_config_default", "reg_ctx_create", "reg_ctx_destroy", "reg_pairwise", "reg_scan",
           "reg_scan_work", "reg_scan_dag", "reg_pyramid", "reg_energy", "reg_compose_grid", "reg_grid_dims",
           "reg_stream_open", "reg_stream_submit", "reg_stream_poll", "reg_stream_close",
           "reg_ctx_set_timing", "reg_ctx_last_timing", "reg_strerror", "reg_last_error_message",
           "reg_pairwise_noalloc", "reg_autotune", "reg_autotune_save", "reg_autotune_load",
           "reg_scan_grids", "reg_warp", "reg_scan_batch", "reg_scan_node_grids", "reg_stream_grids",
           "reg_stream_set_lookback", "reg_mock_scan", "reg_autotune_get"]
METRIC_MEAN, METRIC_GAUSS_NEWTON, METRIC_H1 = 0, 1, 2
REG_STOP_GRAD, REG_STOP_REL, REG_STOP_LS, REG_STOP_MAXIT = 0, 1, 2, 3


class RegError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class reg_elem_t(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("k", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("gx", ctypes.c_float), ("gy", ctypes.c_float)]


class reg_config_t(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("levels", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_rejects", ctypes.c_int), ("tol_grad", ctypes.c_double), ("tol_rel_e", ctypes.c_double),
                ("armijo_c", ctypes.c_double), ("tau0", ctypes.c_double), ("step_cap", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("storage", ctypes.c_int), ("cluster", ctypes.c_int),
                ("workers", ctypes.c_int), ("mem_budget", ctypes.c_size_t), ("grid", ctypes.c_int),
                ("metric", ctypes.c_int), ("unroll", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("sigma", ctypes.c_double), ("tol_coarse", ctypes.c_double)]


class reg_stats_t(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int32), ("k", ctypes.c_int32), ("iters", ctypes.c_int32 * MAX_LEVELS),
                ("evals", ctypes.c_int32 * MAX_LEVELS), ("stop", ctypes.c_int32 * MAX_LEVELS),
                ("rejects", ctypes.c_int32), ("status", ctypes.c_int32), ("energy", ctypes.c_double),
                ("theta", ctypes.c_double * 3)]


class reg_timing_t(ctypes.Structure):
    _fields_ = [("op_launches", ctypes.c_int32), ("pyramid_launches", ctypes.c_int32),
                ("op_kernel_ms", ctypes.c_double), ("pyramid_ms", ctypes.c_double),
                ("graph_captures", ctypes.c_int32), ("tma_staged", ctypes.c_int32),
                ("leaf_ops", ctypes.c_int32), ("dag_ops", ctypes.c_int32),
                ("leaf_ms", ctypes.c_double), ("dag_ms", ctypes.c_double), ("cluster", ctypes.c_int32),
                ("unroll", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("h2d_path", ctypes.c_int32),
                ("h2d_ms", ctypes.c_double)]


class reg_result_t(ctypes.Structure):
    _fields_ = [("frame_id", ctypes.c_uint64), ("elem", reg_elem_t), ("submit_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("status", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libreg.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libreg.so is not built ({LIB_PATH}); run paper_2010_12478_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp, fp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        L.reg_config_default.argtypes = [ctypes.POINTER(reg_config_t)]
        L.reg_ctx_create.argtypes = [ctypes.POINTER(reg_config_t), ip, ctypes.POINTER(vp)]
        L.reg_ctx_destroy.argtypes = [vp]
        L.reg_pairwise.argtypes = [vp, fp, fp, ip, ip, ip, ctypes.POINTER(reg_elem_t), fp,
                                   ctypes.POINTER(reg_elem_t), fp, ctypes.POINTER(reg_stats_t), vp]
        L.reg_scan.argtypes = [vp, fp, ip, ip, ip, ip, ip, ip, vp, fp, ctypes.POINTER(reg_stats_t), vp]
        L.reg_scan_work.argtypes = [ip, ip]
        L.reg_scan_dag.argtypes = [ip, ip, vp, vp, vp]
        L.reg_pyramid.argtypes = [vp, fp, ip, ip, ip, ip, ip, vp, vp]
        L.reg_energy.argtypes = [vp, fp, fp, ip, ip, dp, fp, dp, dp, fp, vp]
        L.reg_compose_grid.argtypes = [vp, fp, fp, ip, ip, fp, vp]
        L.reg_grid_dims.argtypes = [ip, ip, ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip)]
        L.reg_stream_open.argtypes = [vp, ip, ip, ctypes.POINTER(vp)]
        L.reg_stream_submit.argtypes = [vp, fp, ctypes.c_uint64]
        L.reg_stream_poll.argtypes = [vp, ctypes.POINTER(reg_result_t), ip, ctypes.POINTER(ctypes.c_int), ip]
        L.reg_stream_close.argtypes = [vp]
        L.reg_stream_grids.argtypes = [vp, fp, ip]
        L.reg_stream_set_lookback.argtypes = [vp, ip]
        L.reg_mock_scan.argtypes = [vp, ip, ip, ip, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
        L.reg_pairwise_noalloc.argtypes = [ctypes.POINTER(reg_config_t), ip, fp, fp, ip, ip, ip,
                                           ctypes.POINTER(reg_elem_t), ctypes.POINTER(reg_elem_t),
                                           ctypes.POINTER(reg_stats_t), vp]
        L.reg_autotune.argtypes = [vp, fp, ip, ip, ip, ip, ip, ip, ctypes.POINTER(ip)]
        L.reg_autotune_get.argtypes = [vp, ip, ip, ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip)]
        L.reg_scan_grids.argtypes = [vp, fp, ctypes.POINTER(ip), vp]
        L.reg_scan_node_grids.argtypes = [vp, vp, ip, fp, vp]
        L.reg_scan_batch.argtypes = [vp, fp, ip, ip, ip, ip, ip, ip, ip, vp, fp, ctypes.POINTER(reg_stats_t), vp]
        L.reg_warp.argtypes = [vp, fp, ip, ip, ip, ip, ctypes.POINTER(reg_elem_t), fp, fp, fp, vp]
        L.reg_autotune_save.argtypes = [vp, ctypes.c_char_p]
        L.reg_autotune_load.argtypes = [vp, ctypes.c_char_p]
        L.reg_ctx_set_timing.argtypes = [vp, ip]
        L.reg_ctx_last_timing.argtypes = [vp, ctypes.POINTER(reg_timing_t)]
        L.reg_strerror.argtypes = [ip]
        L.reg_strerror.restype = ctypes.c_char_p
        L.reg_last_error_message.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(code: int, where: str):
    if code != REG_OK:
        msg = lib().reg_last_error_message().decode(errors="replace")
        raise RegError(code, where, f"{lib().reg_strerror(code).decode()}: {msg}")


def _ptr(a) -> Optional[int]:
    """Data pointer of a torch tensor or numpy array (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


@dataclasses.dataclass
class Config:
    mode: str = "rigid"
    levels: int = 2
    max_iter: int = 500
    max_rejects: int = 30
    tol_grad: float = 3e-5
    tol_rel_e: float = 0.0
    armijo_c: float = 0.25
    tau0: float = 1.0
    step_cap: float = 0.5
    lam: float = 2.0
    storage: str = "f32"
    cluster: int = 0
    workers: int = 0
    mem_budget: int = 0
    grid: int = 0
    metric: int = 1               # nonrigid scalar product: 1 Gauss-Newton diagonal, 0 mean over control
                                  # points, 2 H1 (identity + sigma^2 grid Laplacian)
    unroll: int = 0               # nonrigid energy passes: pixels per lane (2, 4); 0 = tuned or 4
    ctas_per_sm: int = 0          # nonrigid register form (3, 4); 0 = tuned or by CTAs per operator
    sigma: float = 1.0            # metric 2 (H1): smoothing length in control-grid spacings
    tol_coarse: float = 10.0      # stop factor at every level above the finest

    def c(self) -> reg_config_t:
        return reg_config_t(RIGID if self.mode == "rigid" else NONRIGID, self.levels, self.max_iter,
                            self.max_rejects, self.tol_grad, self.tol_rel_e, self.armijo_c, self.tau0,
                            self.step_cap, self.lam, STORAGES[self.storage], self.cluster, self.workers,
                            self.mem_budget, self.grid, self.metric, self.unroll, self.ctas_per_sm, self.sigma,
                            self.tol_coarse)


def stats_dict(s: reg_stats_t, levels: int) -> dict:
    return dict(i=s.i, k=s.k, iters=list(s.iters[:levels]), evals=list(s.evals[:levels]),
                stop=list(s.stop[:levels]), rejects=s.rejects, status=s.status, energy=s.energy,
                theta=list(s.theta))


def elems_list(elems):
    """reg_elem_t records as (i, k, alpha, gx, gy) tuples (None passes through)."""
    return [(e.i, e.k, e.alpha, e.gx, e.gy) for e in elems] if elems is not None else None


def stats_list(stats, levels: int):
    """reg_stats_t records as dicts (None passes through)."""
    return [stats_dict(s, levels) for s in stats] if stats is not None else None


def scan_work(schedule: str, n: int) -> int:
    return lib().reg_scan_work(SCHEDULES[schedule], n)


def scan_dag(schedule: str, n: int):
    m = scan_work(schedule, n)
    left = np.zeros(max(m, 1), np.int32)
    right = np.zeros(max(m, 1), np.int32)
    out = np.zeros(max(n, 1), np.int32)
    lib().reg_scan_dag(SCHEDULES[schedule], n, left.ctypes.data, right.ctypes.data, out.ctypes.data)
    return list(zip(left[:m].tolist(), right[:m].tolist())), out[:n].tolist()


class Context:
    """A libreg context on one GPU (owns pyramids, queues and workspaces)."""

    def __init__(self, cfg: Optional[Config] = None, device: int = 0):
        self.cfg = cfg or Config()
        self._c = self.cfg.c()
        h = ctypes.c_void_p()
        check(lib().reg_ctx_create(ctypes.byref(self._c), device, ctypes.byref(h)), "reg_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().reg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, frames, schedule: str = "brent_kung", exec: str = "persistent") -> int:
        N, H, W = frames.shape
        best = ctypes.c_int()
        check(lib().reg_autotune(self.h, _ptr(frames), N, W, H, W, SCHEDULES[schedule], EXECS[exec],
                                 ctypes.byref(best)), "reg_autotune")
        return best.value

    def tuned_shape(self, frames_shape, exec: str = "persistent") -> Optional[dict]:
        """The autotuned launch shape for frames of shape (N, H, W) and an executor, or None."""
        N, H, W = frames_shape
        c, u, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        if lib().reg_autotune_get(self.h, N, W, H, EXECS[exec], ctypes.byref(c), ctypes.byref(u),
                                  ctypes.byref(m)) != 0:
            return None
        return dict(cluster=c.value, unroll=u.value, ctas_per_sm=m.value)

    def autotune_save(self, path: str):
        check(lib().reg_autotune_save(self.h, path.encode()), "reg_autotune_save")

    def autotune_load(self, path: str):
        check(lib().reg_autotune_load(self.h, path.encode()), "reg_autotune_load")

    def set_timing(self, enable: bool = True):
        check(lib().reg_ctx_set_timing(self.h, int(enable)), "reg_ctx_set_timing")

    def last_timing(self) -> dict:
        t = reg_timing_t()
        check(lib().reg_ctx_last_timing(self.h, ctypes.byref(t)), "reg_ctx_last_timing")
        return dict(op_launches=t.op_launches, pyramid_launches=t.pyramid_launches,
                    op_kernel_ms=t.op_kernel_ms, pyramid_ms=t.pyramid_ms, graph_captures=t.graph_captures,
                    tma_staged=t.tma_staged, leaf_ops=t.leaf_ops, dag_ops=t.dag_ops, leaf_ms=t.leaf_ms,
                    dag_ms=t.dag_ms, cluster=t.cluster, unroll=t.unroll, ctas_per_sm=t.ctas_per_sm,
                    h2d_path=t.h2d_path, h2d_ms=t.h2d_ms)

    # ---- operators
    def pairwise(self, R, T, init: Optional[Sequence[float]] = None, field_in=None, field_out=None,
                 stream=None, W: Optional[int] = None, pitch: Optional[int] = None):
        """A (init None) or B's minimisation from init.  R, T: [H, W] arrays, or [H, pitch] rows
        of which the first W columns are the frame (pass W and pitch)."""
        H = R.shape[-2]
        W = R.shape[-1] if W is None else W
        pitch = R.shape[-1] if pitch is None else pitch
        out = reg_elem_t()
        st = reg_stats_t()
        ini = None
        if init is not None:
            ini = reg_elem_t(0, 1, float(init[0]), float(init[1]), float(init[2]))
        check(lib().reg_pairwise(self.h, _ptr(R), _ptr(T), W, H, pitch, ctypes.byref(ini) if ini else None,
                                 _ptr(field_in), ctypes.byref(out), _ptr(field_out), ctypes.byref(st),
                                 _stream(stream)), "reg_pairwise")
        return (out.i, out.k, out.alpha, out.gx, out.gy), stats_dict(st, self.cfg.levels)

    def scan(self, frames, schedule: str = "brent_kung", exec: str = "level", fields_out=None,
             out_elems=None, want_stats: bool = True, stream=None, split: bool = False, raw: bool = False):
        """reg_scan; split=True runs every A leaf before the first B and times the phases apart.
        raw=True returns the host arrays as reg_scan filled them (reg_elem_t and reg_stats_t
        records); elems_list() and stats_list() convert them later."""
        N, H, W = frames.shape
        n = N - 1
        m = scan_work(schedule, n)
        elems = (reg_elem_t * n)() if out_elems is None else None
        stats = (reg_stats_t * (n + m))() if want_stats else None
        out_ptr = ctypes.addressof(elems) if elems is not None else _ptr(out_elems)
        ex = EXECS[exec] | (SPLIT_PHASES if split else 0)
        check(lib().reg_scan(self.h, _ptr(frames), N, W, H, W, SCHEDULES[schedule], ex, out_ptr,
                             _ptr(fields_out), stats, _stream(stream)), "reg_scan")
        if raw:
            return elems, stats
        return elems_list(elems), stats_list(stats, self.cfg.levels)

    def scan_batch(self, frames, schedule: str = "brent_kung", exec: str = "persistent", fields_out=None,
                   want_stats: bool = True, stream=None, raw: bool = False):
        """S series [S, N, H, W] in one call; returns per-series element lists and stats
        (raw=True: the host arrays reg_scan_batch filled, series after series)."""
        S, N, H, W = frames.shape
        n = N - 1
        m = scan_work(schedule, n)
        elems = (reg_elem_t * (S * n))()
        stats = (reg_stats_t * (S * (n + m)))() if want_stats else None
        check(lib().reg_scan_batch(self.h, _ptr(frames), S, N, W, H, W, SCHEDULES[schedule], EXECS[exec],
                                   ctypes.addressof(elems), _ptr(fields_out), stats, _stream(stream)),
              "reg_scan_batch")
        if raw:
            return elems, stats
        el = [[(e.i, e.k, e.alpha, e.gx, e.gy) for e in elems[q * n:(q + 1) * n]] for q in range(S)]
        st = None
        if stats is not None:
            st = [[stats_dict(x, self.cfg.levels) for x in stats[q * (n + m):(q + 1) * (n + m)]] for q in range(S)]
        return el, st

    def scan_grids(self, out):
        """Control values [N-1, ny, nx, 2] (device) of the last nonrigid scan's prefixes."""
        n = ctypes.c_int()
        check(lib().reg_scan_grids(self.h, _ptr(out), ctypes.byref(n), None), "reg_scan_grids")
        return n.value

    def mock_scan(self, values, op_us, schedule: str = "brent_kung", exec: str = "persistent"):
        """reg_mock_scan: the schedule's DAG of the mock operator (sum after a spin of op_us[j]
        microseconds); returns (prefix sums, device milliseconds)."""
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
        us = np.ascontiguousarray(np.asarray(op_us, dtype=np.float32))
        out = np.zeros(len(v), dtype=np.float64)
        ms = ctypes.c_double()
        check(lib().reg_mock_scan(self.h, len(v), SCHEDULES[schedule], EXECS[exec], v.ctypes.data, us.ctypes.data,
                                  out.ctypes.data, ctypes.byref(ms)), "reg_mock_scan")
        return out, ms.value

    def scan_node_grids(self, ops: Sequence[int], out):
        """Control values [len(ops), ny, nx, 2] (device) of the given operators' results of the last
        nonrigid scan (per_op order: leaves first, then B operators in DAG order)."""
        idx = np.ascontiguousarray(np.asarray(ops, dtype=np.int32))
        check(lib().reg_scan_node_grids(self.h, idx.ctypes.data, len(idx), _ptr(out), None), "reg_scan_node_grids")

    def warp(self, frames, elems=None, grids=None, out=None, mean=None, stream=None):
        """Registered series out[k] = f_k o phi_{0,k} and/or its mean (device tensors).
        elems: rigid prefixes, as returned by scan() (a list of tuples), as an elem_array(),
        or as a device tensor holding reg_elem_t records; grids: nonrigid control values."""
        N, H, W = frames.shape
        if elems is None or isinstance(elems, ctypes.Array):
            eptr = elems
        elif hasattr(elems, "data_ptr"):
            eptr = ctypes.cast(ctypes.c_void_p(elems.data_ptr()), ctypes.POINTER(reg_elem_t))
        else:
            eptr = elem_array(elems)
        check(lib().reg_warp(self.h, _ptr(frames), N, W, H, W, eptr, _ptr(grids), _ptr(out), _ptr(mean),
                             _stream(stream)), "reg_warp")

    # ---- kernel-level steps
    def pyramid(self, frame, levels: int, storage: str, out):
        H, W = frame.shape
        check(lib().reg_pyramid(self.h, _ptr(frame), W, H, W, levels, STORAGES[storage], _ptr(out), None),
              "reg_pyramid")

    def energy_rigid(self, R, T, theta):
        H, W = R.shape
        th = (ctypes.c_double * 3)(*[float(v) for v in theta])
        E = ctypes.c_double()
        g = (ctypes.c_double * 3)()
        check(lib().reg_energy(self.h, _ptr(R), _ptr(T), W, H, th, None, ctypes.byref(E), g, None, None),
              "reg_energy")
        return E.value, np.array(list(g))

    def energy_grid(self, R, T, values, grad_values=None):
        """E (and dE/dc into grad_values) at control values [ny, nx, 2] (device)."""
        H, W = R.shape
        E = ctypes.c_double()
        check(lib().reg_energy(self.h, _ptr(R), _ptr(T), W, H, None, _ptr(values), ctypes.byref(E), None,
                               _ptr(grad_values), None), "reg_energy")
        return E.value

    def compose_grid(self, q1, q2, W: int, H: int, out):
        check(lib().reg_compose_grid(self.h, _ptr(q1), _ptr(q2), W, H, _ptr(out), None), "reg_compose_grid")


def elem_array(elems):
    """ctypes array of reg_elem_t from (i, k, alpha, gx, gy) tuples (host memory)."""
    arr = (reg_elem_t * max(1, len(elems)))()
    for j, e in enumerate(elems):
        arr[j] = reg_elem_t(int(e[0]), int(e[1]), float(e[2]), float(e[3]), float(e[4]))
    return arr


def grid_dims(W: int, H: int, grid: int = 0, levels: int = 2):
    nx, ny, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().reg_grid_dims(W, H, grid, levels, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(sp)),
          "reg_grid_dims")
    return nx.value, ny.value, sp.value


def pairwise_noalloc(cfg: Config, R, T, init: Optional[Sequence[float]] = None, device: int = 0, stream=None,
                     W: Optional[int] = None, pitch: Optional[int] = None):
    """reg_pairwise_noalloc: rigid pairwise registration that allocates nothing (device R, T;
    [H, pitch] rows of which the first W columns are the frame when W and pitch are given)."""
    H = R.shape[-2]
    W = R.shape[-1] if W is None else W
    pitch = R.shape[-1] if pitch is None else pitch
    c = cfg.c()
    out = reg_elem_t()
    st = reg_stats_t()
    ini = reg_elem_t(0, 1, float(init[0]), float(init[1]), float(init[2])) if init is not None else None
    check(lib().reg_pairwise_noalloc(ctypes.byref(c), device, _ptr(R), _ptr(T), W, H, pitch,
                                     ctypes.byref(ini) if ini else None, ctypes.byref(out), ctypes.byref(st),
                                     _stream(stream)), "reg_pairwise_noalloc")
    return (out.i, out.k, out.alpha, out.gx, out.gy), stats_dict(st, cfg.levels)


class Stream:
    """An acquisition stream of the serving API (reg_stream_*)."""

    def __init__(self, ctx: Context, W: int, H: int):
        self.ctx = ctx
        h = ctypes.c_void_p()
        check(lib().reg_stream_open(ctx.h, W, H, ctypes.byref(h)), "reg_stream_open")
        self.h = h

    def set_lookback(self, k: int):
        """Online scan with a look-back of k leaves (1, 2, 4 or 8); call before the first submit."""
        check(lib().reg_stream_set_lookback(self.h, k), "reg_stream_set_lookback")

    def set_grids(self, ring):
        """Nonrigid streams: write each result's control values into ring[i % len(ring)] (device
        tensor [capacity, ny, nx, 2]); call before the first submit."""
        check(lib().reg_stream_grids(self.h, _ptr(ring), ring.shape[0]), "reg_stream_grids")

    def submit(self, frame, frame_id: int) -> int:
        return lib().reg_stream_submit(self.h, _ptr(frame), frame_id)

    def poll(self, max_results: int = 64, timeout_us: int = 0) -> List[dict]:
        buf = (reg_result_t * max_results)()
        n = ctypes.c_int()
        rc = lib().reg_stream_poll(self.h, buf, max_results, ctypes.byref(n), timeout_us)
        if rc not in (REG_OK, REG_ETIMEOUT):
            check(rc, "reg_stream_poll")
        return [dict(frame_id=r.frame_id, elem=(r.elem.i, r.elem.k, r.elem.alpha, r.elem.gx, r.elem.gy),
                     submit_us=r.submit_us, done_us=r.done_us, status=r.status) for r in buf[:n.value]]

    def close(self):
        if self.h:
            check(lib().reg_stream_close(self.h), "reg_stream_close")
            self.h = None
