"""FP64 CPU oracle of the registration scan operator (arXiv 2010.12478).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path (``paper_2010_12478_gb300``) and never imports it; the product
never imports this.

Layers:
  * ``oracle.c`` (compiled to ``_build/liboracle.so`` with gcc, FP64, no fast
    math): pyramid, bilinear sampling, NCC energy and gradient, the gradient
    flow with Armijo backtracking (rigid and nonrigid), composition.
  * this module: ctypes marshalling, the operators A and B (Sec. 2.3.1-2.3.2),
    the scan DAG generators (Sec. 3, Table 1) and the scan driver that applies
    B along a DAG, one call at a time.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 8
STOP_NAMES = {0: "grad", 1: "rel", 2: "linesearch", 3: "maxiter"}


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (strict IEEE double: no fast math, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("max_iter", ctypes.c_int), ("max_rejects", ctypes.c_int),
                ("tol_grad", ctypes.c_double), ("tol_rel_e", ctypes.c_double),
                ("armijo_c", ctypes.c_double), ("tau0", ctypes.c_double),
                ("step_cap", ctypes.c_double), ("lambda_", ctypes.c_double), ("metric", ctypes.c_int),
                ("sigma", ctypes.c_double), ("tol_coarse", ctypes.c_double)]


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("s", ctypes.c_int), ("W0", ctypes.c_int),
                ("H0", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int * MAX_LEVELS), ("evals", ctypes.c_int * MAX_LEVELS),
                ("stop", ctypes.c_int * MAX_LEVELS), ("rejects", ctypes.c_int),
                ("energy", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ipp = ctypes.POINTER(ctypes.c_int)
            dpp = ctypes.POINTER(dp)
            L.or_downsample.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
            L.or_sample.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            L.or_sample_q.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, dp]
            L.or_rigid_energy.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.or_rigid_energy.restype = ctypes.c_int
            L.or_rigid_compose.argtypes = [dp, dp, dp]
            L.or_rigid_register.argtypes = [dpp, dpp, ipp, ipp, ctypes.POINTER(_Cfg), dp, dp,
                                            ctypes.POINTER(_Stats)]
            gp = ctypes.POINTER(_Grid)
            L.or_grid_regulariser.argtypes = [gp, dp, dp, ctypes.c_double, ctypes.c_double]
            L.or_grid_regulariser.restype = ctypes.c_double
            L.or_grid_energy.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, gp, dp, dp,
                                         ctypes.c_double, dp, dp, dp]
            L.or_grid_energy.restype = ctypes.c_int
            L.or_grid_register.argtypes = [dpp, dpp, ipp, ipp, ctypes.POINTER(_Cfg), gp, dp, dp, dp, dp,
                                           ctypes.POINTER(_Stats)]
            L.or_grid_compose.argtypes = [gp, dp, dp, dp, dp, dp, dp]
            L.or_grid_metric.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, gp, dp, dp, ctypes.c_double,
                                         dp, dp]
            L.or_grid_dense.argtypes = [gp, dp, dp, dp, dp]
            L.or_grid_level_dense.argtypes = [gp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            L.or_warp_rigid.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, dp]
            L.or_step_size.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int]
            L.or_step_size.restype = ctypes.c_double
            L.or_bb_first_step.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_int, ctypes.c_double]
            L.or_bb_first_step.restype = ctypes.c_double
            L.or_warp_grid.argtypes = [gp, dp, dp, dp, dp]
            L.or_h1_apply.argtypes = [gp, ctypes.c_double, dp, dp]
            L.or_h1_inverse.argtypes = [gp, ctypes.c_double, dp, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# configuration (readings of the paper's unstated constants)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Config:
    levels: int = 2
    max_iter: int = 500
    max_rejects: int = 30
    tol_grad: float = 3e-5
    tol_rel_e: float = 0.0
    armijo_c: float = 0.25
    tau0: float = 1.0
    step_cap: float = 0.5
    lam: float = 2.0
    grid: int = 0                 # control-grid spacing of the nonrigid field (finest px), 0 = auto
    mode: str = "rigid"           # "rigid" (the paper's map, Sec. 2.3.1) or "nonrigid" (extension)
    metric: int = 1               # nonrigid scalar product: 1 Gauss-Newton diagonal, 0 mean over control
                                  # points, 2 H1 (identity + sigma^2 grid Laplacian)
    sigma: float = 1.0            # metric 2: smoothing length in control-grid spacings
    tol_coarse: float = 10.0      # factor on tol_grad at every level above the finest

    def c(self) -> _Cfg:
        return _Cfg(self.levels, self.max_iter, self.max_rejects, self.tol_grad, self.tol_rel_e,
                    self.armijo_c, self.tau0, self.step_cap, self.lam, self.metric, self.sigma, self.tol_coarse)


@dataclasses.dataclass
class Stats:
    iters: List[int]
    evals: List[int]
    stop: List[int]
    rejects: int
    energy: float

    @staticmethod
    def of(s: _Stats, L: int) -> "Stats":
        return Stats(list(s.iters[:L]), list(s.evals[:L]), list(s.stop[:L]), s.rejects, s.energy)


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------
def downsample(img) -> np.ndarray:
    img = _f64(img)
    H, W = img.shape
    out = np.empty(((H + 1) // 2, (W + 1) // 2), dtype=np.float64)
    lib().or_downsample(_dp(img), W, H, _dp(out))
    return out


def pyramid(img, levels: int) -> List[np.ndarray]:
    """Level 0 = the frame itself (as float64); level l+1 = 2x2 box average of level l."""
    p = [_f64(img)]
    for _ in range(levels - 1):
        p.append(downsample(p[-1]))
    return p


def sample(T, px: float, py: float):
    T = _f64(T)
    H, W = T.shape
    out = np.empty(3, dtype=np.float64)
    lib().or_sample(_dp(T), W, H, px, py, _dp(out))
    return out


def sample_q(T, px: float, py: float, outside: Optional[float] = None):
    """Quadratic B-spline model of T's samples at (px, py), samples beyond the frame equal to
    ``outside`` (default: T's mean, as in the nonrigid energy): (value, d/dpx, d/dpy)."""
    T = _f64(T)
    H, W = T.shape
    out = np.empty(3, dtype=np.float64)
    lib().or_sample_q(_dp(T), W, H, float(T.mean()) if outside is None else float(outside), px, py, _dp(out))
    return out


def rigid_energy(R, T, theta, grad: bool = True):
    R, T, th = _f64(R), _f64(T), _f64(theta)
    H, W = R.shape
    E = np.zeros(1)
    g = np.zeros(3)
    lib().or_rigid_energy(_dp(R), _dp(T), W, H, _dp(th), _dp(E), _dp(g) if grad else None)
    return (float(E[0]), g) if grad else float(E[0])


@dataclasses.dataclass
class Grid:
    """Control grid of the nonrigid field: points (jx*s, jy*s), jx < nx, jy < ny (finest px)."""
    nx: int
    ny: int
    s: int
    W0: int
    H0: int

    def c(self) -> _Grid:
        return _Grid(self.nx, self.ny, self.s, self.W0, self.H0)


def grid_for(W0: int, H0: int, spacing: int = 0) -> Grid:
    """Spacing 16 px, doubled until the grid has at most 65 points per axis (spacing 0),
    or the given spacing."""
    s = spacing if spacing > 0 else 16
    if spacing <= 0:
        while (W0 - 1 + s - 1) // s + 1 > 65 or (H0 - 1 + s - 1) // s + 1 > 65:
            s *= 2
    return Grid((W0 - 1 + s - 1) // s + 1, (H0 - 1 + s - 1) // s + 1, s, W0, H0)


def grid_energy(R, T, level: int, g: Grid, c, lam: float, grad: bool = True):
    """Energy of the level-``level`` images for control values c [2, ny, nx] in pixels of that level."""
    R, T = _f64(R), _f64(T)
    cx, cy = _f64(c[0]), _f64(c[1])
    H, W = R.shape
    E = np.zeros(1)
    gc = g.c()
    if grad:
        gx = np.zeros((g.ny, g.nx)); gy = np.zeros((g.ny, g.nx))
        lib().or_grid_energy(_dp(R), _dp(T), W, H, level, ctypes.byref(gc), _dp(cx), _dp(cy), lam, _dp(E),
                             _dp(gx), _dp(gy))
        return float(E[0]), np.stack([gx, gy])
    lib().or_grid_energy(_dp(R), _dp(T), W, H, level, ctypes.byref(gc), _dp(cx), _dp(cy), lam, _dp(E), None, None)
    return float(E[0])


def grid_metric(T, level: int, g: Grid, c, lam: float) -> np.ndarray:
    """The nonrigid flow's scalar product [2, ny, nx] (Gauss-Newton diagonal, normalised) for the
    level-``level`` template T at control values c (pixels of that level)."""
    T = _f64(T)
    H, W = T.shape
    cx, cy = _f64(c[0]), _f64(c[1])
    mx = np.zeros((g.ny, g.nx)); my = np.zeros((g.ny, g.nx))
    gc = g.c()
    lib().or_grid_metric(_dp(T), W, H, level, ctypes.byref(gc), _dp(cx), _dp(cy), lam, _dp(mx), _dp(my))
    return np.stack([mx, my])


def h1_apply(g: Grid, sigma: float, v) -> np.ndarray:
    """(I + sigma^2 Lg) v for a control-point field v [ny, nx], Lg the control grid's graph Laplacian."""
    v = _f64(v)
    out = np.zeros_like(v)
    gc = g.c()
    lib().or_h1_apply(ctypes.byref(gc), sigma, _dp(v), _dp(out))
    return out


def h1_inverse(g: Grid, sigma: float, rhs) -> np.ndarray:
    """(I + sigma^2 Lg)^-1 rhs by banded Cholesky (the H1 flow's solve)."""
    rhs = _f64(rhs)
    out = np.zeros_like(rhs)
    gc = g.c()
    lib().or_h1_inverse(ctypes.byref(gc), sigma, _dp(rhs), _dp(out))
    return out


def grid_regulariser(g: Grid, c, lam: float, P: float) -> float:
    cx, cy = _f64(c[0]), _f64(c[1])
    gc = g.c()
    return float(lib().or_grid_regulariser(ctypes.byref(gc), _dp(cx), _dp(cy), lam, P))


def grid_dense(g: Grid, c) -> np.ndarray:
    """Dense finest-level field [2, H0, W0] of control values c (finest px)."""
    cx, cy = _f64(c[0]), _f64(c[1])
    ux = np.zeros((g.H0, g.W0)); uy = np.zeros((g.H0, g.W0))
    gc = g.c()
    lib().or_grid_dense(ctypes.byref(gc), _dp(cx), _dp(cy), _dp(ux), _dp(uy))
    return np.stack([ux, uy])


def grid_level_dense(g: Grid, c, level: int, H: int, W: int) -> np.ndarray:
    """Field [2, H, W] on the pixels of pyramid level ``level`` for control values in that level's px."""
    cx, cy = _f64(c[0]), _f64(c[1])
    ux = np.zeros((H, W)); uy = np.zeros((H, W))
    gc = g.c()
    lib().or_grid_level_dense(ctypes.byref(gc), _dp(cx), _dp(cy), level, W, H, _dp(ux), _dp(uy))
    return np.stack([ux, uy])


def compose_grid(g: Grid, c1, c2) -> np.ndarray:
    """Control values of phi_2 o phi_1 at the control points (B's initial guess, Sec. 2.3.2)."""
    a0, a1, b0, b1 = (_f64(v) for v in (c1[0], c1[1], c2[0], c2[1]))
    ox = np.zeros((g.ny, g.nx)); oy = np.zeros((g.ny, g.nx))
    gc = g.c()
    lib().or_grid_compose(ctypes.byref(gc), _dp(a0), _dp(a1), _dp(b0), _dp(b1), _dp(ox), _dp(oy))
    return np.stack([ox, oy])


def compose_rigid(a, b) -> np.ndarray:
    """phi_b o phi_a (apply a first): B's initial guess phi_jk o phi_ij (Sec. 2.3.2)."""
    a, b = _f64(a), _f64(b)
    out = np.zeros(3)
    lib().or_rigid_compose(_dp(a), _dp(b), _dp(out))
    return out


def _pyr_args(pyr: Sequence[np.ndarray]):
    L = len(pyr)
    arr = (ctypes.POINTER(ctypes.c_double) * L)(*[_dp(p) for p in pyr])
    Ws = (ctypes.c_int * L)(*[p.shape[1] for p in pyr])
    Hs = (ctypes.c_int * L)(*[p.shape[0] for p in pyr])
    return arr, Ws, Hs


def register_rigid(Rpyr, Tpyr, init, cfg: Config):
    """Multilevel gradient-flow registration of T onto R, rigid map of Sec. 2.3.1."""
    assert len(Rpyr) == cfg.levels == len(Tpyr)
    ra, Ws, Hs = _pyr_args(Rpyr)
    ta, _, _ = _pyr_args(Tpyr)
    init = _f64(init)
    out = np.zeros(3)
    st = _Stats()
    c = cfg.c()
    lib().or_rigid_register(ra, ta, Ws, Hs, ctypes.byref(c), _dp(init), _dp(out), ctypes.byref(st))
    return out, Stats.of(st, cfg.levels)


def register_nonrigid(Rpyr, Tpyr, init_c, cfg: Config):
    """Multilevel registration of the control-grid field; init_c and the result in finest px."""
    assert len(Rpyr) == cfg.levels == len(Tpyr)
    ra, Ws, Hs = _pyr_args(Rpyr)
    ta, _, _ = _pyr_args(Tpyr)
    H, W = Rpyr[0].shape
    g = grid_for(W, H, cfg.grid)
    gc = g.c()
    ox = np.zeros((g.ny, g.nx)); oy = np.zeros((g.ny, g.nx))
    st = _Stats()
    c = cfg.c()
    if init_c is None:
        lib().or_grid_register(ra, ta, Ws, Hs, ctypes.byref(c), ctypes.byref(gc), None, None, _dp(ox), _dp(oy),
                               ctypes.byref(st))
    else:
        ix, iy = _f64(init_c[0]), _f64(init_c[1])
        lib().or_grid_register(ra, ta, Ws, Hs, ctypes.byref(c), ctypes.byref(gc), _dp(ix), _dp(iy), _dp(ox),
                               _dp(oy), ctypes.byref(st))
    return np.stack([ox, oy]), Stats.of(st, cfg.levels)


# --------------------------------------------------------------------------
# scan elements and the operators A and B (Sec. 2.3.1-2.3.2)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Elem:
    i: int                        # reference frame index
    k: int                        # template frame index
    phi: np.ndarray               # rigid: (alpha, Gx, Gy); nonrigid: control values [2, ny, nx] (finest px)
    stats: Optional[Stats] = None


def identity(mode: str, H: int, W: int, grid: int = 0) -> np.ndarray:
    if mode == "rigid":
        return np.zeros(3)
    g = grid_for(W, H, grid)
    return np.zeros((2, g.ny, g.nx))


def register(Rpyr, Tpyr, init, cfg: Config):
    if cfg.mode == "rigid":
        return register_rigid(Rpyr, Tpyr, init, cfg)
    return register_nonrigid(Rpyr, Tpyr, init, cfg)


def op_A(pyrs, i: int, k: int, cfg: Config) -> Elem:
    """A(f_i, f_k): register from the identity (neighbouring frames)."""
    H, W = pyrs[i][0].shape
    phi, st = register(pyrs[i], pyrs[k], identity(cfg.mode, H, W, cfg.grid), cfg)
    return Elem(i, k, phi, st)


def op_B(e1: Elem, e2: Elem, pyrs, cfg: Config) -> Elem:
    """B(phi_ij, phi_jk) = register f_k onto f_i from phi_jk o phi_ij (Sec. 2.3.2)."""
    if e1.k != e2.i:
        raise ValueError(f"B needs adjacent elements, got ({e1.i},{e1.k}) and ({e2.i},{e2.k})")
    if cfg.mode == "rigid":
        init = compose_rigid(e1.phi, e2.phi)
    else:
        H, W = pyrs[e1.i][0].shape
        init = compose_grid(grid_for(W, H, cfg.grid), e1.phi, e2.phi)
    phi, st = register(pyrs[e1.i], pyrs[e2.k], init, cfg)
    return Elem(e1.i, e2.k, phi, st)


# --------------------------------------------------------------------------
# scan DAGs (Sec. 3, Table 1).  SSA form: leaves 0..n-1 are the inputs x_0..x_{n-1};
# op j creates node n+j = node[l] (.) node[r]; out[i] holds x_0 (.) ... (.) x_i.
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Dag:
    name: str
    n: int
    ops: List[tuple]
    out: List[int]
    exclusive: bool = False

    def work(self) -> int:
        return len(self.ops)

    def depth(self) -> int:
        d = [0] * (self.n + len(self.ops))
        for j, (l, r) in enumerate(self.ops):
            d[self.n + j] = 1 + max(d[l] if l >= 0 else 0, d[r] if r >= 0 else 0)
        return max(d) if d else 0


class _Builder:
    def __init__(self, n):
        self.n = n
        self.ops = []

    def op(self, l, r):
        self.ops.append((l, r))
        return self.n + len(self.ops) - 1


def dag_sequential(n: int) -> Dag:
    """Left fold y_i = y_{i-1} (.) x_i: depth and work n-1 (Table 1)."""
    b = _Builder(n)
    cur = list(range(n))
    for i in range(1, n):
        cur[i] = b.op(cur[i - 1], cur[i])
    return Dag("sequential", n, b.ops, cur)


def dag_brent_kung(n: int) -> Dag:
    """Tree scan: up-sweep over strides 1,2,4,..., then the down-sweep fills the gaps."""
    b = _Builder(n)
    cur = list(range(n))
    d = 1
    while d < n:
        for i in range(2 * d - 1, n, 2 * d):
            cur[i] = b.op(cur[i - d], cur[i])
        d *= 2
    d = 1 << max(0, (n.bit_length() - 2)) if n > 1 else 1
    while d >= 1:
        for i in range(3 * d - 1, n, 2 * d):
            cur[i] = b.op(cur[i - d], cur[i])
        d //= 2
    return Dag("brent_kung", n, b.ops, cur)


def dag_dissemination(n: int) -> Dag:
    """Recursive doubling: round r combines elements 2^r apart (Fig. 2)."""
    b = _Builder(n)
    cur = list(range(n))
    d = 1
    while d < n:
        prev = list(cur)
        for i in range(d, n):
            cur[i] = b.op(prev[i - d], prev[i])
        d *= 2
    return Dag("dissemination", n, b.ops, cur)


def dag_ladner_fischer(n: int, k: int = 0) -> Dag:
    """Ladner-Fischer family P_k.  P_0(n): P_1 on the left half, P_0 on the right half,
    then the left total is combined into every right output (n/2 ops).  P_k(n), k >= 1:
    pairwise combine, P_{k-1} on the n/2 pair sums, then fill the even positions."""
    b = _Builder(n)

    def rec(xs, k):
        m = len(xs)
        if m == 1:
            return list(xs)
        if m == 2:
            return [xs[0], b.op(xs[0], xs[1])]
        if k == 0:
            h = (m + 1) // 2
            left = rec(xs[:h], 1)
            right = rec(xs[h:], 0)
            return left + [b.op(left[-1], r) for r in right]
        pairs = [b.op(xs[2 * i], xs[2 * i + 1]) for i in range(m // 2)]
        sub = rec(pairs, k - 1)
        out = [xs[0]]
        for i in range(1, m):
            if i % 2 == 1:
                out.append(sub[i // 2])
            else:
                out.append(b.op(sub[i // 2 - 1], xs[i]))
        return out

    out = rec(list(range(n)), k)
    return Dag(f"ladner_fischer{k}", n, b.ops, out)


def dag_blelloch(n: int) -> Dag:
    """Exclusive tree scan (up-sweep, then down-sweep from the identity, node -1), on the series
    padded with identity elements to a power of two P: an application with a padded operand is
    x (.) e = x and is not made, nor one whose result only feeds padded positions.  Counted with
    its identity applications: work 2(n-1), depth 2 log2 P (Table 1)."""
    b = _Builder(n)
    P = 1
    while P < n:
        P *= 2
    cur = list(range(n)) + [-1] * (P - n)
    d = 1
    while d < P:
        for i in range(2 * d - 1, P, 2 * d):
            # padding is a suffix: a padded left operand has a padded right one
            cur[i] = cur[i - d] if cur[i] == -1 else b.op(cur[i - d], cur[i])
        d *= 2
    if n > 0:
        cur[P - 1] = -1
    d = P // 2
    while d >= 1:
        for i in range(2 * d - 1, P, 2 * d):
            left, parent = cur[i - d], cur[i]
            cur[i - d] = parent
            # positions i-d+1 .. i take this value: all padding when i-d+1 >= n
            cur[i] = b.op(parent, left) if left != -1 and i - d + 1 < n else parent
        d //= 2
    return Dag("blelloch", n, b.ops, cur[:n], exclusive=True)


def dag_lookback(n: int, k: int) -> Dag:
    """The online scan of an acquisition stream with a look-back of k leaves (k a power of two).
    As leaf j arrives, window nodes w_m(j) = x_{j-2^m+1} (.) ... (.) x_j are formed by doubling,
    w_m(j) = w_{m-1}(j - 2^(m-1)) (.) w_{m-1}(j) for j >= 2^m - 1, m = 1..log2 k, and the prefix
    p_j = p_{j-1} (.) x_j for 0 < j < k, p_j = p_{j-k} (.) w_{log2 k}(j) for j >= k.  The chain of
    prefixes then advances k leaves per operator (k chains side by side); k = 1 is the
    sequential recursion (Sec. 3)."""
    if k < 1 or k & (k - 1):
        raise ValueError("k must be a power of two")
    b = _Builder(n)
    m = k.bit_length() - 1
    w = [list(range(n))] + [[None] * n for _ in range(m)]
    p = [None] * n
    for j in range(n):
        for lev in range(1, m + 1):
            if j >= (1 << lev) - 1:
                w[lev][j] = b.op(w[lev - 1][j - (1 << (lev - 1))], w[lev - 1][j])
        if j == 0:
            p[0] = 0
        elif j < k:
            p[j] = b.op(p[j - 1], j)
        else:
            p[j] = b.op(p[j - k], w[m][j])
    return Dag(f"lookback{k}", n, b.ops, p)


DAGS = {"sequential": dag_sequential, "brent_kung": dag_brent_kung,
        "dissemination": dag_dissemination, "ladner_fischer": dag_ladner_fischer,
        "lookback2": lambda n: dag_lookback(n, 2), "lookback4": lambda n: dag_lookback(n, 4),
        "lookback8": lambda n: dag_lookback(n, 8)}


def scan(frames, cfg: Config, dag: Optional[Dag] = None, leaves: Optional[List[Elem]] = None,
         pyrs=None) -> List[Elem]:
    """Register every frame to frame 0: leaves A(f_{i-1}, f_i), then B along ``dag``.
    Returns [phi_{0,1}, ..., phi_{0,N-1}] (inclusive scan of Sec. 3)."""
    N = len(frames)
    n = N - 1
    if pyrs is None:
        pyrs = [pyramid(np.asarray(f), cfg.levels) for f in frames]
    if dag is None:
        dag = dag_sequential(n)
    assert dag.n == n and not dag.exclusive
    nodes: List[Elem] = list(leaves) if leaves is not None else [op_A(pyrs, i, i + 1, cfg) for i in range(n)]
    for (l, r) in dag.ops:
        nodes.append(op_B(nodes[l], nodes[r], pyrs, cfg))
    return [nodes[o] for o in dag.out]


def step_size(E: float, slope: float, tau: float, Et: float, accepted: bool) -> float:
    """The line search's next step after a trial at tau with energy Et (see oracle.c)."""
    return float(lib().or_step_size(E, slope, tau, Et, 1 if accepted else 0))


def bb_first_step(tau_q: float, tau_acc: float, d_prev, d, m0: float = 1.0) -> float:
    """First trial of a line search after an accepted step of length tau_acc along d_prev, with the
    new direction d: the Barzilai-Borwein step in the metric diag(m0, 1, ...), else tau_q."""
    a, b = _f64(np.ravel(d_prev)), _f64(np.ravel(d))
    return float(lib().or_bb_first_step(tau_q, tau_acc, _dp(a), _dp(b), a.size, m0))


# --------------------------------------------------------------------------
# registered series (Sec. 2: frames registered to the first one, then averaged)
# --------------------------------------------------------------------------
def warp(T, mode: str, phi, grid: int = 0) -> np.ndarray:
    """T resampled onto the reference grid: out(x) = T(phi(x)).  Rigid phi = (alpha, gx, gy);
    nonrigid phi = control values [2, ny, nx] (finest px) of the grid ``grid_for(W, H, grid)``."""
    T = _f64(T)
    H, W = T.shape
    out = np.zeros((H, W))
    if mode == "rigid":
        lib().or_warp_rigid(_dp(T), W, H, _dp(_f64(phi)), _dp(out))
    else:
        g = grid_for(W, H, grid)
        c = _f64(phi)
        gc = g.c()
        lib().or_warp_grid(ctypes.byref(gc), _dp(T), _dp(_f64(c[0])), _dp(_f64(c[1])), _dp(out))
    return out


def register_series(frames, mode: str, phis, grid: int = 0):
    """Registered series and its mean: out[0] = f_0, out[k] = f_k o phi_{0,k} for the N-1
    prefixes ``phis`` of the scan; mean = (1/N) sum_k out[k]."""
    frames = np.asarray(frames)
    N = len(frames)
    assert len(phis) == N - 1
    out = np.zeros(frames.shape, dtype=np.float64)
    out[0] = frames[0]
    for k in range(1, N):
        out[k] = warp(frames[k], mode, phis[k - 1], grid)
    return out, out.sum(axis=0) / N


# --------------------------------------------------------------------------
# comparisons
# --------------------------------------------------------------------------
def rigid_displacement(theta, H: int, W: int) -> np.ndarray:
    """phi(x) - x on the pixel grid, [2, H, W] (for pixel-error comparisons)."""
    th = _f64(theta)
    cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    xc, yc = x - cx, y - cy
    ca, sa = math.cos(th[0]), math.sin(th[0])
    px = ca * xc - sa * yc + cx + th[1]
    py = sa * xc + ca * yc + cy + th[2]
    return np.stack([px - x, py - y])


def max_px_error(phi_a, phi_b, H: int, W: int, mode: str, grid: int = 0) -> float:
    """max over finest-level pixels of |phi_a(x) - phi_b(x)|_2 (nonrigid: control values,
    or dense [2, H, W] fields)."""
    if mode == "rigid":
        d = rigid_displacement(phi_a, H, W) - rigid_displacement(phi_b, H, W)
    else:
        g = grid_for(W, H, grid)
        a = _f64(phi_a) if np.shape(phi_a)[1:] == (H, W) else grid_dense(g, phi_a)
        b = _f64(phi_b) if np.shape(phi_b)[1:] == (H, W) else grid_dense(g, phi_b)
        d = a - b
    return float(np.sqrt((d ** 2).sum(axis=0)).max())
