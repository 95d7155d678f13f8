"""Seeded synthetic electron-microscopy series: crystal-lattice frames with drift.

This module only generates inputs.  It holds none of the registration
arithmetic, and both the CUDA path and the FP64 oracle consume the frames it
produces.

A frame is an analytic render of a square lattice of Gaussian atom columns:

    f_t(y) = b + a * sum_atoms exp(-|y - s_t - w_t(y) - atom|^2 / (2 sigma^2)) + noise

where ``s_t`` is the drift of frame ``t`` (translation, pixels) and ``w_t`` a
smooth displacement field built from four low-frequency sinusoids.  The
Gaussian sum is separable, so each pixel costs eight exponentials (atoms
farther than 8 px contribute below 1e-6 of the peak and are dropped).  Noise
is Gaussian with standard deviation std(clean frame) / SNR.

Frame ``t`` aligned to frame 0 satisfies ``f_t(phi(x)) ~= f_0(x)`` for
``phi(x) ~= x + (s_t - s_0) + (w_t(x) - w_0(x))``: that is the ground truth
returned beside the frames.  The electron-microscopy data of the paper
(Sec. 5, 1920x1856 TEM frames) is not available; these series stand in for it
with the paper's structure: a (nearly) periodic image whose neighbouring
frames differ by less than half a period (Sec. 2.3.2).

Seeds: numpy's PCG64 seeded with ``(seed, series)`` draws the per-series and
per-frame parameters; the per-pixel noise comes from a ``torch.Generator``
seeded with ``seed * 1_000_003 + frame`` on the device the frames are built on.
The default seed 1410 is the one the paper uses for its mock operator (Sec. 5.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

DEFAULT_SEED = 1410


@dataclasses.dataclass
class SeriesSpec:
    n_frames: int
    H: int
    W: int
    sigma: float = 1.5            # atom-column width, px
    period: float = 8.0           # lattice spacing, px
    background: float = 0.1
    amplitude: float = 1.0        # atom peak above background
    drift: str = "increment"      # "increment": s_t = s_{t-1} + U(-step, step) per axis
    step: float = 3.0             # per-frame drift bound, px per axis
    field_amp: float = 1.0        # bound on |w_t(x)|, px (0 = no field)
    field_rate: Tuple[float, float] = (0.05, 0.2)  # temporal frequency of the field modes, rad/frame
    snr: Optional[Tuple[float, float]] = (10.0, 10.0)  # per-frame SNR drawn uniformly; None = no noise
    jump_frac: float = 0.0        # fraction of frames whose drift increment gets an extra jump
    jump_max: float = 0.0         # jump length U(0, jump_max] px in a random direction
    seed: int = DEFAULT_SEED
    series: int = 0               # index of this series under the seed


@dataclasses.dataclass
class Series:
    frames: torch.Tensor          # [N, H, W] float32
    shifts: np.ndarray            # [N, 2] drift s_t (x, y), px
    truth_shift: np.ndarray       # [N, 2] s_t - s_0
    field_modes: dict             # parameters of w_t, for truth_field()
    spec: SeriesSpec

    def truth_field(self, t: int) -> np.ndarray:
        """First-order ground-truth displacement of frame t against frame 0, [2, H, W]."""
        w_t = _field(self.field_modes, t, self.spec.H, self.spec.W, torch.device("cpu"))
        w_0 = _field(self.field_modes, 0, self.spec.H, self.spec.W, torch.device("cpu"))
        d = (w_t - w_0).numpy()
        d[0] += self.truth_shift[t, 0]
        d[1] += self.truth_shift[t, 1]
        return d


# Named workloads (sizes and structure of the series the registration is run on).
def spec_c1(seed: int = DEFAULT_SEED) -> SeriesSpec:
    """16 frames of 128x128: per-frame drift U(+-3) px per axis, field <= 1 px, SNR 10."""
    return SeriesSpec(16, 128, 128, step=3.0, field_amp=1.0, snr=(10.0, 10.0), seed=seed)


def spec_c2(seed: int = DEFAULT_SEED, n_frames: int = 256) -> SeriesSpec:
    """256 frames of 512x512: random walk U(+-1) px per axis, field <= 1.5 px, SNR 10."""
    return SeriesSpec(n_frames, 512, 512, step=1.0, field_amp=1.5, snr=(10.0, 10.0), seed=seed)


def spec_c3(seed: int = DEFAULT_SEED, n_frames: int = 4096) -> SeriesSpec:
    """4096 frames of 512x512: as spec_c2 with SNR U(3, 20) and 5% jumps of up to 8 px."""
    return SeriesSpec(n_frames, 512, 512, step=1.0, field_amp=1.5, snr=(3.0, 20.0),
                      jump_frac=0.05, jump_max=8.0, seed=seed)


def _rng(spec: SeriesSpec) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([spec.seed, spec.series, 0x5EED]))


def _draw_parameters(spec: SeriesSpec):
    rng = _rng(spec)
    phase = rng.uniform(0.0, spec.period, size=2)
    inc = rng.uniform(-spec.step, spec.step, size=(spec.n_frames, 2))
    inc[0] = 0.0
    if spec.jump_frac > 0.0:
        jump = rng.uniform(size=spec.n_frames) < spec.jump_frac
        jump[0] = False
        length = spec.jump_max * (1.0 - rng.uniform(size=spec.n_frames))  # (0, jump_max]
        ang = rng.uniform(0.0, 2.0 * math.pi, size=spec.n_frames)
        inc[:, 0] += np.where(jump, length * np.cos(ang), 0.0)
        inc[:, 1] += np.where(jump, length * np.sin(ang), 0.0)
    shifts = np.cumsum(inc, axis=0)
    # four field modes: integer wave numbers in -2..2 (not both 0)
    modes = []
    for _ in range(4):
        while True:
            k, l = rng.integers(-2, 3, size=2)
            if k != 0 or l != 0:
                break
        ang = rng.uniform(0.0, 2.0 * math.pi)
        modes.append(dict(k=int(k), l=int(l), phi=float(rng.uniform(0.0, 2.0 * math.pi)),
                          dx=math.cos(ang), dy=math.sin(ang),
                          a=float(rng.uniform(0.5, 1.0)),
                          omega=float(rng.uniform(*spec.field_rate)),
                          beta=float(rng.uniform(0.0, 2.0 * math.pi))))
    total = sum(m["a"] for m in modes)
    for m in modes:  # sum of |a_m| = field_amp bounds |w| by field_amp
        m["a"] *= spec.field_amp / total if total > 0 else 0.0
    if spec.snr is None:
        snr = np.full(spec.n_frames, np.inf)
    else:
        snr = rng.uniform(spec.snr[0], spec.snr[1], size=spec.n_frames)
    return phase, shifts, modes, snr


def _field(modes, t: int, H: int, W: int, device) -> torch.Tensor:
    y = torch.arange(H, dtype=torch.float64, device=device).view(H, 1)
    x = torch.arange(W, dtype=torch.float64, device=device).view(1, W)
    wx = torch.zeros(H, W, dtype=torch.float64, device=device)
    wy = torch.zeros(H, W, dtype=torch.float64, device=device)
    for m in modes:
        c = m["a"] * math.sin(m["omega"] * t + m["beta"])
        s = torch.sin(2.0 * math.pi * (m["k"] * x / W + m["l"] * y / H) + m["phi"])
        wx = wx + c * m["dx"] * s
        wy = wy + c * m["dy"] * s
    return torch.stack([wx, wy])


def _lattice_axis(q: torch.Tensor, period: float, sigma: float) -> torch.Tensor:
    """Sum over the four nearest atoms along one axis of exp(-(q - atom)^2 / (2 sigma^2))."""
    f = q - period * torch.floor(q / period)          # [0, period)
    acc = torch.zeros_like(q)
    inv = 1.0 / (2.0 * sigma * sigma)
    for j in (-1, 0, 1, 2):
        d = f - period * j
        acc = acc + torch.exp(-d * d * inv)
    return acc


def render_frame(spec: SeriesSpec, phase, shift, modes, t: int, snr: float,
                 device="cpu") -> torch.Tensor:
    device = torch.device(device)
    H, W = spec.H, spec.W
    y = torch.arange(H, dtype=torch.float64, device=device).view(H, 1).expand(H, W)
    x = torch.arange(W, dtype=torch.float64, device=device).view(1, W).expand(H, W)
    if spec.field_amp > 0.0:
        w = _field(modes, t, H, W, device)
        qx = x - shift[0] - w[0] - phase[0]
        qy = y - shift[1] - w[1] - phase[1]
    else:
        qx = x - shift[0] - phase[0]
        qy = y - shift[1] - phase[1]
    clean = spec.background + spec.amplitude * (
        _lattice_axis(qx, spec.period, spec.sigma) * _lattice_axis(qy, spec.period, spec.sigma))
    if math.isfinite(snr):
        g = torch.Generator(device=device)
        g.manual_seed(int(spec.seed) * 1_000_003 + int(spec.series) * 7919 + t)
        noise = torch.randn((H, W), generator=g, dtype=torch.float64, device=device)
        clean = clean + (clean.std() / snr) * noise
    return clean.to(torch.float32)


def make_series(spec: SeriesSpec, device="cpu", frames_out: Optional[torch.Tensor] = None) -> Series:
    """Render the whole series on ``device`` (float64 math, float32 frames)."""
    phase, shifts, modes, snr = _draw_parameters(spec)
    if frames_out is None:
        frames_out = torch.empty((spec.n_frames, spec.H, spec.W), dtype=torch.float32, device=device)
    for t in range(spec.n_frames):
        frames_out[t] = render_frame(spec, phase, shifts[t], modes, t, float(snr[t]), device)
    return Series(frames=frames_out, shifts=shifts, truth_shift=shifts - shifts[0],
                  field_modes=modes, spec=spec)


def translated_pair(H: int, W: int, shift_xy: Sequence[float], seed: int = DEFAULT_SEED,
                    noise_snr: Optional[float] = None, period: float = 8.0,
                    sigma: float = 1.5) -> Tuple[np.ndarray, np.ndarray]:
    """Two noiseless (unless ``noise_snr``) lattice frames whose content differs by a pure
    translation: ``T(x + shift) = R(x)``, so the registration should return G = shift."""
    spec = SeriesSpec(2, H, W, field_amp=0.0, snr=None, seed=seed, period=period, sigma=sigma)
    rng = _rng(spec)
    phase = rng.uniform(0.0, period, size=2)
    snr = float("inf") if noise_snr is None else float(noise_snr)
    R = render_frame(spec, phase, np.zeros(2), [], 0, snr)
    T = render_frame(spec, phase, np.asarray(shift_xy, dtype=np.float64), [], 1, snr)
    return R.numpy(), T.numpy()


def rigid_pair(H: int, W: int, alpha: float, shift_xy: Sequence[float], seed: int = DEFAULT_SEED,
               noise_snr: Optional[float] = None, period: float = 8.0,
               sigma: float = 1.5) -> Tuple[np.ndarray, np.ndarray]:
    """Lattice frames R, T with T(phi(x)) = R(x) for the rigid map
    phi(x) = Rot(alpha) (x - c) + c + G, c the image centre: T is rendered at
    phi^{-1}(y) = Rot(-alpha) (y - c - G) + c."""
    spec = SeriesSpec(2, H, W, field_amp=0.0, snr=None, seed=seed, period=period, sigma=sigma)
    rng = _rng(spec)
    phase = rng.uniform(0.0, period, size=2)
    cx, cy = 0.5 * (W - 1), 0.5 * (H - 1)
    y = torch.arange(H, dtype=torch.float64).view(H, 1).expand(H, W)
    x = torch.arange(W, dtype=torch.float64).view(1, W).expand(H, W)

    def lattice(qx, qy):
        return spec.background + spec.amplitude * (
            _lattice_axis(qx - phase[0], period, sigma) * _lattice_axis(qy - phase[1], period, sigma))

    R = lattice(x, y)
    ca, sa = math.cos(alpha), math.sin(alpha)
    dx, dy = x - cx - shift_xy[0], y - cy - shift_xy[1]
    T = lattice(ca * dx + sa * dy + cx, -sa * dx + ca * dy + cy)
    out = []
    for t, img in enumerate((R, T)):
        if noise_snr is not None:
            g = torch.Generator()
            g.manual_seed(int(seed) * 1_000_003 + 17 + t)
            img = img + (img.std() / noise_snr) * torch.randn((H, W), generator=g, dtype=torch.float64)
        out.append(img.to(torch.float32).numpy())
    return out[0], out[1]
