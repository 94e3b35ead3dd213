"""Seeded synthetic inputs: stroke programs, palettes, cotangents, pixel samples.

This module holds none of the rendering arithmetic: it only draws parameters.
Both the CUDA path and the FP64 oracle receive the arrays it returns (the oracle
widens the same float32 values to float64), so the two sides never share code.

Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) in counter form:
``z = seed + (i+1) * 0x9E3779B97F4A7C15`` mixed by the published finaliser,
and a uniform double is ``(z >> 11) * 2**-53``.

Stroke distribution (the paper's synthetic-program recipe, Sec. 6 "Synthetic
ground truth" plays the same "render of a known program" role):
  centre uniform in [0,1]^2; direction angle uniform in [0, 2 pi);
  length 0 (a drop) with probability 0.5, else uniform in [0, len_max];
  half-width log-uniform in [r_lo, r_hi]; palette of K colours uniform in
  [0,1]^3; palette assignment k uniform in {0..K-1} with logits 6 * onehot(k)
  and softmax temperature 1; white background.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive splitmix64 outputs of stream ``seed`` starting at ``offset``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from stream ``seed``."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class Program:
    """A stroke program in program order (index 0 is executed first).

    cx, cy      segment centre (canvas units, canvas [0,1]^2)
    theta       direction angle (radians)
    length      full segment length L >= 0 (0 = drop)
    half_width  r > 0
    logits      [n, k] palette-assignment logits
    palette     [k, 3] sRGB colours
    background  [3] background colour c_0
    color_temp  softmax temperature tau_c
    """
    cx: np.ndarray
    cy: np.ndarray
    theta: np.ndarray
    length: np.ndarray
    half_width: np.ndarray
    logits: np.ndarray
    palette: np.ndarray
    background: np.ndarray
    color_temp: float = 1.0
    coupling: np.ndarray | None = None  # [n, 3] c_1..c_3 of the coupling profile, or None

    @property
    def n(self) -> int:
        return int(self.cx.shape[0])

    @property
    def k(self) -> int:
        return int(self.palette.shape[0])

    def copy(self) -> "Program":
        return dataclasses.replace(self, **{f.name: (np.array(getattr(self, f.name))
                                                     if isinstance(getattr(self, f.name), np.ndarray)
                                                     else getattr(self, f.name))
                                            for f in dataclasses.fields(self)})

    def prefix(self, m: int) -> "Program":
        p = self.copy()
        for name in ("cx", "cy", "theta", "length", "half_width", "logits"):
            setattr(p, name, np.ascontiguousarray(getattr(p, name)[:m]))
        if p.coupling is not None:
            p.coupling = np.ascontiguousarray(p.coupling[:m])
        return p


def make_palette(seed: int, k: int) -> np.ndarray:
    return uniform(seed, 3 * k).reshape(k, 3).astype(np.float32)


def make_program(n: int, seed: int, palette_seed: int, k: int, r_lo: float, r_hi: float,
                 len_max: float = 0.2, p_drop: float = 0.5, logit_scale: float = 6.0,
                 palette: np.ndarray | None = None) -> Program:
    """Draw a seeded program from the stroke distribution above (float32)."""
    u = uniform(seed, 8 * n).reshape(n, 8)
    cx = u[:, 0]
    cy = u[:, 1]
    theta = 2.0 * math.pi * u[:, 2]
    length = np.where(u[:, 3] < p_drop, 0.0, len_max * u[:, 4])
    r = np.exp(math.log(r_lo) + u[:, 5] * (math.log(r_hi) - math.log(r_lo)))
    kidx = np.minimum((u[:, 6] * k).astype(np.int64), k - 1)
    logits = np.zeros((n, k), dtype=np.float64)
    logits[np.arange(n), kidx] = logit_scale
    pal = make_palette(palette_seed, k) if palette is None else np.asarray(palette, np.float32)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return Program(cx=f32(cx), cy=f32(cy), theta=f32(theta), length=f32(length),
                   half_width=f32(r), logits=f32(logits), palette=f32(pal),
                   background=np.ones(3, dtype=np.float32), color_temp=1.0)


def make_coupling(seed: int, n: int, c1_max: float = 0.4, c2_max: float = 0.15,
                  c3_max: float = 0.1) -> np.ndarray:
    """Seeded profiles (c_1, c_2, c_3) of the coupling variant, [n, 3] float32:
    c_1 ~ U[0, c1_max] (a positive first mode widens the flank and shortens the
    tips), c_2 ~ U[-c2_max, c2_max], c_3 ~ U[-c3_max, c3_max].  With the defaults
    |c_1| + |c_2| + |c_3| <= 0.65, so g >= 0.35 on every leaf."""
    u = uniform(seed, 3 * n).reshape(n, 3)
    c = np.stack([c1_max * u[:, 0], c2_max * (2 * u[:, 1] - 1), c3_max * (2 * u[:, 2] - 1)], 1)
    return np.ascontiguousarray(c.astype(np.float32))


def make_cotangent(seed: int, npix: int) -> np.ndarray:
    """A seeded cotangent dJ/dR in [-1, 1), shape [npix, 3] (float32)."""
    return (2.0 * uniform(seed, 3 * npix) - 1.0).reshape(npix, 3).astype(np.float32)


def sample_pixels(seed: int, total: int, m: int) -> np.ndarray:
    """m distinct flat pixel indices out of ``total`` (sorted, int64)."""
    m = min(m, total)
    keys = splitmix64(seed, total) if total <= 1 << 24 else None
    if keys is not None:
        return np.sort(np.argsort(keys, kind="stable")[:m]).astype(np.int64)
    picks = set()
    off = 0
    while len(picks) < m:
        cand = (uniform(seed, 2 * m, off) * total).astype(np.int64)
        off += 2 * m
        for c in cand.tolist():
            picks.add(c)
            if len(picks) == m:
                break
    return np.array(sorted(picks), dtype=np.int64)


# ---------------------------------------------------------------------------
# Named workloads (the paper's operating point is 2000 strokes at 1024^2,
# Sec. 5.2 "Fitting performance"; the sharper 1/200 relaxation is expressed as
# tau = 0, tau_min = 1/200 in Eq. relax).
# ---------------------------------------------------------------------------
SHARP_TAU, SHARP_TAU_MIN = 0.0, 1.0 / 200.0


def small_program() -> Program:
    """50 strokes, 8-colour palette, r log-uniform in [0.01, 0.08] (rendered at 128^2)."""
    return make_program(50, seed=101, palette_seed=201, k=8, r_lo=0.01, r_hi=0.08)


def operating_program(seed: int = 102, palette_seed: int = 202) -> Program:
    """2000 strokes, 16-colour palette, r log-uniform in [0.003, 0.05] (rendered at 1024^2)."""
    return make_program(2000, seed=seed, palette_seed=palette_seed, k=16, r_lo=0.003, r_hi=0.05)


def operating_target_program() -> Program:
    """Second seeded 2000-stroke program whose hard render is the L2 target."""
    return operating_program(seed=103, palette_seed=202)


def fit_programs() -> tuple[Program, Program]:
    """(initial, target) 2000-stroke programs of the full-fit workload."""
    return operating_program(seed=104, palette_seed=203), operating_program(seed=105, palette_seed=203)


def resolution_program() -> Program:
    """The 2000-stroke program of the resolution-replay sweep (512^2 .. 4096^2)."""
    return operating_program(seed=106, palette_seed=206)
