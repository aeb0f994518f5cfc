"""Seeded synthetic inputs for the hierarchical-grid correlator.

This module only builds inputs: array geometries (the level shapes n_k1 x n_k2
and matrices A_k of Eq. GridEq, Sec. II.D) and antenna voltages (noise plus
plane-wave point sources).  It holds none of the correlator's arithmetic and is
shared by the test-suite, the oracle checks and the benchmark.

Conventions used everywhere in this project:

* A hierarchy is a list of levels, level 1 (finest) first.  Level k has a shape
  (n_k1, n_k2) and a 2x2 matrix A_k = [a_k | a_{k+n}] (row-major), so that the
  antenna with integer index m_k = (m_k1, m_k2) on every level sits at
  r = sum_k A_k m_k (Eq. GridEq; the paper numbers the first axes of the levels
  a_1..a_n and the second axes a_{n+1}..a_{2n}).
* The lattice dimensions are d = 0..2n-1 with sizes
  (n_11, n_12, n_21, n_22, ...): dimension 0 is level 1's first axis.
* Antennas are stored row-major over (level n axis 2, level n axis 1, ...,
  level 1 axis 2, level 1 axis 1): dimension 0 varies fastest.
* Voltages are [C][T][N] complex, interleaved (re, im), either float32 or int8.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np
import torch

SPEED_OF_LIGHT = 299_792_458.0


@dataclass(frozen=True)
class Level:
    """One level of a hierarchical grid: an n1 x n2 block placed by A."""

    n1: int
    n2: int
    A: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 1.0)


@dataclass
class Workload:
    """A named workload: geometry plus the shape and recipe of its voltages."""

    name: str
    levels: List[Level]
    channels: int
    samples: int
    dtype: str  # "cf32" or "ci8"
    n_sources: int
    noise_sigma: float
    source_sigma: float
    seed: int
    freq_lo_hz: float = 150e6
    freq_hi_hz: float = 150e6
    description: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dims(self) -> List[int]:
        return lattice_dims(self.levels)

    @property
    def n_antennas(self) -> int:
        return int(np.prod(self.dims))


def lattice_dims(levels: Sequence[Level]) -> List[int]:
    dims: List[int] = []
    for lv in levels:
        dims += [int(lv.n1), int(lv.n2)]
    return dims


def antenna_indices(levels: Sequence[Level]) -> np.ndarray:
    """Integer lattice index m_d of every antenna, shape [N][2n] (d=0 first)."""
    dims = lattice_dims(levels)
    grids = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]
    return np.ascontiguousarray(grids.T)


def antenna_positions(levels: Sequence[Level]) -> np.ndarray:
    """Physical positions r = sum_k A_k m_k (Eq. GridEq), shape [N][2], metres."""
    m = antenna_indices(levels).astype(np.float64)
    r = np.zeros((m.shape[0], 2))
    for k, lv in enumerate(levels):
        a = np.asarray(lv.A, dtype=np.float64).reshape(2, 2)
        r += m[:, 2 * k:2 * k + 2] @ a.T
    return r


def sheared_rotation(pitch: float, theta: float, shear: float) -> Tuple[float, ...]:
    """A = pitch * R(theta) * [[1, shear], [0, 1]], row-major."""
    c, s = math.cos(theta), math.sin(theta)
    rot = np.array([[c, -s], [s, c]])
    sh = np.array([[1.0, shear], [0.0, 1.0]])
    return tuple(float(v) for v in (pitch * rot @ sh).ravel())


def _diameter(levels: Sequence[Level]) -> float:
    r = antenna_positions(levels)
    span = r.max(axis=0) - r.min(axis=0)
    return float(math.hypot(span[0], span[1])) + 1.0


def hierarchy(shapes: Sequence[Tuple[int, int]], thetas: Sequence[float],
              shears: Sequence[float]) -> List[Level]:
    """Levels whose pitch is 1.25x the diameter of the block below (level 1: 1 m)."""
    levels: List[Level] = []
    for k, ((n1, n2), th, sh) in enumerate(zip(shapes, thetas, shears)):
        pitch = 1.0 if k == 0 else 1.25 * _diameter(levels)
        levels.append(Level(n1, n2, sheared_rotation(pitch, th, sh)))
    return levels


# ---------------------------------------------------------------------------
# Workloads.  Sizes follow the five benchmark configurations; the geometry of
# the fixtures is the paper's own (Sec. II.C, Sec. II.D, Figs. 2-5).
# ---------------------------------------------------------------------------

def _cfg3_levels(seed: int) -> List[Level]:
    rng = np.random.default_rng(seed)
    thetas = rng.uniform(0.0, math.pi, 3)
    shears = rng.uniform(-0.3, 0.3, 3)
    return hierarchy([(16, 16), (8, 8), (4, 4)], thetas, shears)


def workload(name: str) -> Workload:
    if name == "grid16":
        return Workload(
            name, [Level(16, 16)], channels=1, samples=64, dtype="cf32",
            n_sources=3, noise_sigma=1.0, source_sigma=1.0, seed=9090001,
            freq_lo_hz=SPEED_OF_LIGHT / 2.0, freq_hi_hz=SPEED_OF_LIGHT / 2.0,
            description="single-level 16x16 grid, 1 channel x 64 samples, complex64")
    if name == "hier2":
        return Workload(
            name, hierarchy([(16, 16), (8, 8)], [0.0, math.radians(30.0)], [0.0, 0.2]),
            channels=64, samples=1024, dtype="ci8", n_sources=5, noise_sigma=20.0,
            source_sigma=10.0, seed=9090002, freq_lo_hz=100e6, freq_hi_hz=200e6,
            description="2-level 16x16 blocks on an 8x8 rotated/sheared grid (N=16384), "
                        "64 channels x 1024 samples, int8 complex")
    if name == "hier3":
        return Workload(
            name, _cfg3_levels(9090003), channels=16, samples=256, dtype="cf32",
            n_sources=10, noise_sigma=1.0, source_sigma=1.0, seed=9090003,
            freq_lo_hz=100e6, freq_hi_hz=200e6,
            description="3-level 16x16, 8x8, 4x4 hierarchy (N=262144), "
                        "16 channels x 256 samples, complex64")
    if name == "grid1024":
        return Workload(
            name, [Level(1024, 1024)], channels=16, samples=64, dtype="cf32",
            n_sources=20, noise_sigma=1.0, source_sigma=1.0, seed=9090005,
            freq_lo_hz=100e6, freq_hi_hz=200e6,
            description="single-level 1024x1024 grid (N=1048576), 16 channels x 64 samples")
    raise KeyError(name)


WORKLOADS = ("grid16", "hier2", "hier3", "grid1024")


def batch_arrays(n_arrays: int = 48, seed: int = 9090004) -> List[List[Level]]:
    """Uneven independent arrays: half single-level squares with side 8..64, half
    2-level hierarchies of 4x4 tiles on an 8x8 or 16x16 grid, each with a seeded
    rotation and shear; sorted by shape so that equal shapes are adjacent."""
    rng = np.random.default_rng(seed)
    arrays = []
    for a in range(n_arrays):
        th = rng.uniform(0.0, math.pi, 2)
        sh = rng.uniform(-0.3, 0.3, 2)
        if a < n_arrays // 2:
            side = int(rng.choice([8, 16, 32, 64]))
            arrays.append([Level(side, side, sheared_rotation(1.0, th[0], sh[0]))])
        else:
            side = int(rng.choice([8, 16]))
            arrays.append(hierarchy([(4, 4), (side, side)], list(th), list(sh)))
    arrays.sort(key=lambda lv: (len(lv), [(x.n1, x.n2) for x in lv]))
    return arrays


def batch_voltages(arrays: Sequence[Sequence[Level]], channels: int, samples: int,
                   dtype: str = "ci8", device: str | torch.device = "cpu",
                   seed: int = 9090004, n_sources: int = 3) -> List[torch.Tensor]:
    """Per-array voltages [C][T][N_a][2] with noise sigma 20 and point sources."""
    out = []
    for a, levels in enumerate(arrays):
        w = Workload(f"array{a}", list(levels), channels, samples, dtype, n_sources,
                     noise_sigma=20.0, source_sigma=10.0, seed=seed + 101 * a,
                     freq_lo_hz=100e6, freq_hi_hz=200e6)
        out.append(voltages(w, device=device))
    return out


def paper_fixture(name: str) -> List[Level]:
    """Array layouts printed in the paper."""
    if name == "warmup_1d":        # Sec. II.C: x = 1,2,3,7,8,9 as one 9-long row
        return [Level(9, 1)]
    if name == "warmup_2level":    # Sec. II.C/II.D: a_1=(1,0), a_2=(6,0)
        return [Level(3, 1, (1.0, 0.0, 0.0, 1.0)), Level(2, 1, (6.0, 0.0, 0.0, 1.0))]
    if name == "three_level":      # Fig. 1/2: a_1..a_6, hypercube 5x3x3x3x3x3
        return [Level(5, 3, (1.0, 0.0, 0.0, 1.0)),
                Level(3, 3, (8.0, 2.0, 0.0, 8.0)),
                Level(3, 3, (40.0, -10.0, 10.0, 40.0))]
    if name == "blocks":           # Fig. 3: four 16x16 blocks at 200 m
        return [Level(16, 16, (1.0, 0.0, 0.0, 1.0)), Level(2, 2, (200.0, 0.0, 0.0, 200.0))]
    if name == "plank":            # Fig. 4: one 512x32 block
        return [Level(512, 32)]
    if name == "strips":           # Fig. 5: a_1=(16,0) n=32, a_2=(0,1) n=512
        return [Level(32, 512, (16.0, 0.0, 0.0, 1.0))]
    if name == "interleaved":      # Sec. II.D: a_1=(5,0), a_2=(7,0), 4 points each
        return [Level(4, 1, (5.0, 0.0, 0.0, 1.0)), Level(4, 1, (7.0, 0.0, 0.0, 1.0))]
    raise KeyError(name)


# ---------------------------------------------------------------------------
# Voltages
# ---------------------------------------------------------------------------

def _source_directions(gen: torch.Generator, n: int) -> torch.Tensor:
    """(l, m) direction cosines uniform in the unit disk, float64 [n][2]."""
    u = torch.rand(n, generator=gen, dtype=torch.float64)
    phi = torch.rand(n, generator=gen, dtype=torch.float64) * (2 * math.pi)
    rad = torch.sqrt(u)
    return torch.stack([rad * torch.cos(phi), rad * torch.sin(phi)], dim=1)


def channel_frequencies(w: Workload) -> np.ndarray:
    if w.channels == 1:
        return np.array([w.freq_lo_hz])
    return np.linspace(w.freq_lo_hz, w.freq_hi_hz, w.channels)


def voltages(w: Workload, channels: int | None = None, samples: int | None = None,
             device: str | torch.device = "cpu", seed: int | None = None,
             channel_offset: int = 0) -> torch.Tensor:
    """Seeded voltages [C][T][N][2] (float32 or int8) for a workload.

    Each channel c draws from its own generator seeded with seed + c, so a
    channel's samples do not depend on how many channels are generated.
    x_t(r) = noise + sum_s a_{s,t} exp(2 pi i (l_s x + m_s y) / lambda_c).
    int8 voltages are rounded half-to-even and clipped to [-127, 127].
    """
    C = w.channels if channels is None else channels
    T = w.samples if samples is None else samples
    seed = w.seed if seed is None else seed
    device = torch.device(device)
    pos = torch.from_numpy(antenna_positions(w.levels)).to(device)      # [N][2] f64
    N = pos.shape[0]
    freqs = channel_frequencies(w)
    out_dtype = torch.int8 if w.dtype == "ci8" else torch.float32
    out = torch.empty((C, T, N, 2), dtype=out_dtype, device=device)
    dgen = torch.Generator(device="cpu")
    dgen.manual_seed(seed)
    dirs = _source_directions(dgen, w.n_sources).to(device)            # [S][2]
    for ci in range(C):
        c = ci + channel_offset
        gen = torch.Generator(device=device)
        gen.manual_seed(seed * 1000 + c)
        lam = SPEED_OF_LIGHT / float(freqs[c % len(freqs)])
        x = torch.randn((T, N, 2), generator=gen, device=device,
                        dtype=torch.float32) * w.noise_sigma
        if w.n_sources:
            amp = torch.randn((T, w.n_sources, 2), generator=gen, device=device,
                              dtype=torch.float32) * w.source_sigma
            ph = (pos @ dirs.T) * (2 * math.pi / lam)                   # [N][S] f64
            wave = torch.polar(torch.ones_like(ph), ph).to(torch.complex64)
            a = torch.view_as_complex(amp.contiguous())                 # [T][S]
            x = x + torch.view_as_real(a @ wave.T)
        if out_dtype == torch.int8:
            x = torch.clamp(torch.round(x), -127, 127)
        out[ci] = x.to(out_dtype)
    return out


def all_ones(dims: Sequence[int], C: int, T: int, dtype: str = "cf32") -> torch.Tensor:
    """The layout map of Sec. III (one at every antenna), as [C][T][N][2]."""
    N = int(np.prod(dims))
    t = torch.zeros((C, T, N, 2), dtype=torch.int8 if dtype == "ci8" else torch.float32)
    t[..., 0] = 1
    return t


def random_complex(dims: Sequence[int], C: int, T: int, seed: int, dtype: str = "cf32",
                   sigma: float = 1.0) -> torch.Tensor:
    """Plain seeded complex noise [C][T][N][2]."""
    N = int(np.prod(dims))
    gen = torch.Generator().manual_seed(seed)
    x = torch.randn((C, T, N, 2), generator=gen, dtype=torch.float32) * sigma
    if dtype == "ci8":
        return torch.clamp(torch.round(x), -127, 127).to(torch.int8)
    return x
