"""Seeded synthetic inputs for the grid-hopping path.

This module only draws random numbers and packs them with the fixed radar and
grid parameters of the workloads. It holds no part of the method itself: no
sensing function, atom, transform, interpolation or score. Both the FP64 oracle
and the CUDA path read the inputs it makes; each side turns them into a
measurement with its own implementation of the signal model (Sec. II).

Random numbers come from a counter-based SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
stream s under seed k is mix64(key(k, s) + (i + 1) * 0x9E3779B97F4A7C15), so a
draw never depends on how many numbers were drawn before it and the bytes are
identical on every platform. Normals use the Box-Muller transform.

Workloads (all sizes from the paper's measurement set-up, Sec. V: one TX,
f0 = 24 GHz, B = 250 MHz, Tc = 128 us, Ms = Mc = 128, four receivers):

* ``tiny_scene``: 1 TX at the origin, Q = 3 RX on a 10 m circle, Tc = 100 us,
  Ms = 64 x Mc = 32, one unit-modulus target at SNR 20 dB,
  grid 32 x 32 x 8 x 8 over [0, 20]^2 m x [-10, 10]^2 m/s.
* ``paper_frame``: Q = 4 RX spread over 30 m, Ms = 256 x Mc = 128, three
  Rayleigh targets at SNR 10 dB, grid 128 x 128 x 32 x 32 over
  [0, 40]^2 m x [-15, 15]^2 m/s, K = 3 detections.
* ``precision_scene``: Q = 8, Ms = 512 x Mc = 256, five targets at SNR 5 dB,
  grid 256 x 256 x 64 x 64.
* ``batch_scenes``: many frames of uneven size (Q in 3..8, Ms in
  {128, 256, 512}, Mc in {64, 128, 256}, (x, y) sides in {64, 96, 128, 160},
  velocity sides in {16, 24, 32, 40}, 1..5 targets at SNR 0..20 dB), or a
  small variant with the same spread for the oracle.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers: one independent stream per kind of draw.
_S_RX, _S_TGT_POS, _S_TGT_VEL, _S_AMP, _S_PHASE, _S_NOISE, _S_ONGRID, _S_BATCH = range(1, 9)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """n raw 64-bit values of stream ``stream`` under ``seed`` (counter based)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)]) +
                     _GAMMA * np.uint64(stream + 1))[0]
        ctr = np.arange(1, n + 1, dtype=np.uint64)
        return _mix64(key + _GAMMA * ctr)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform on [0, 1), 53 random bits each."""
    return (splitmix64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of uniforms."""
    u = uniform(seed, stream, 2 * n)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def complex_normal(seed: int, stream: int, shape, var: float = 1.0) -> np.ndarray:
    """Circular complex Gaussian CN(0, var) samples of the given shape."""
    n = int(np.prod(shape))
    g = normal(seed, stream, 2 * n)
    return ((g[0::2] + 1j * g[1::2]) * np.sqrt(var / 2.0)).reshape(shape)


@dataclass(frozen=True)
class Radar:
    """FMCW frame parameters (Sec. II): carrier f0 [Hz], bandwidth B [Hz],
    chirp duration Tc [s], Ms samples per chirp, Mc chirps, zero-pad factor."""
    f0: float
    B: float
    Tc: float
    Ms: int
    Mc: int
    pad: int = 4


@dataclass(frozen=True)
class Grid:
    """Cell-centred 4D grid over (x, y, vx, vy): point i of axis a is
    lo[a] + (i + 1/2) * step[a], i = 0 .. n[a]-1. Linear cell index
    ((ix * ny + iy) * nvx + ivx) * nvy + ivy."""
    lo: Tuple[float, float, float, float]
    step: Tuple[float, float, float, float]
    n: Tuple[int, int, int, int]

    @staticmethod
    def from_bounds(lo, hi, n) -> "Grid":
        lo = tuple(float(v) for v in lo)
        n = tuple(int(v) for v in n)
        step = tuple((float(h) - l) / k for l, h, k in zip(lo, hi, n))
        return Grid(lo, step, n)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n, dtype=np.int64))

    def axis(self, a: int) -> np.ndarray:
        return self.lo[a] + (np.arange(self.n[a]) + 0.5) * self.step[a]

    def cell_index(self, ix, iy, ivx, ivy):
        nx, ny, nvx, nvy = self.n
        return ((np.int64(ix) * ny + iy) * nvx + ivx) * nvy + ivy

    def unravel(self, cell):
        nx, ny, nvx, nvy = self.n
        cell = np.int64(cell)
        ivy = cell % nvy
        ivx = (cell // nvy) % nvx
        iy = (cell // (nvy * nvx)) % ny
        ix = cell // (nvy * nvx * ny)
        return int(ix), int(iy), int(ivx), int(ivy)

    def centre(self, cell) -> np.ndarray:
        idx = self.unravel(cell)
        return np.array([self.lo[a] + (idx[a] + 0.5) * self.step[a] for a in range(4)])


@dataclass
class Scene:
    """One frame: geometry, targets, random amplitudes and noise, and the grid.

    targets[t] = (x, y, vx, vy) in m and m/s; alpha[t, q] is the scattering
    coefficient of target t at receiver q; noise[q] is W_q of shape (Mc, Ms).
    """
    name: str
    seed: int
    radar: Radar
    tx: np.ndarray                 # (2,)
    rx: np.ndarray                 # (Q, 2)
    targets: np.ndarray            # (T, 4)
    alpha: np.ndarray              # (T, Q) complex128
    noise: np.ndarray              # (Q, Mc, Ms) complex128
    grid: Grid
    K: int
    snr_db: Optional[float]
    target_cells: Optional[np.ndarray] = field(default=None)  # on-grid scenes only

    @property
    def Q(self) -> int:
        return self.rx.shape[0]

    def noiseless(self) -> "Scene":
        return replace(self, noise=np.zeros_like(self.noise), snr_db=None)


def _noise(seed, Q, radar, snr_db):
    shape = (Q, radar.Mc, radar.Ms)
    if snr_db is None:
        return np.zeros(shape, np.complex128)
    return complex_normal(seed, _S_NOISE, shape, 10.0 ** (-snr_db / 10.0))


def _uniform_box(seed, stream, T, lo, hi):
    u = uniform(seed, stream, 2 * T).reshape(T, 2)
    return lo + (hi - lo) * u


def _unit_phase(seed, shape):
    return np.exp(2j * np.pi * uniform(seed, _S_PHASE, int(np.prod(shape))).reshape(shape))


def _rayleigh_alpha(seed, T, Q):
    mag = np.abs(complex_normal(seed, _S_AMP, (T,), 1.0))
    return mag[:, None] * _unit_phase(seed, (T, Q))


def _ongrid_targets(seed, grid: Grid, T):
    """Targets placed exactly on cell centres, at least 4 cells apart in x, y."""
    idx = []
    u = uniform(seed, _S_ONGRID, 64 * T).reshape(-1, 4)
    for row in u:
        cand = tuple(int(row[a] * grid.n[a]) for a in range(4))
        if all(max(abs(cand[0] - c[0]), abs(cand[1] - c[1])) >= 4 for c in idx):
            idx.append(cand)
        if len(idx) == T:
            break
    cells = np.array([grid.cell_index(*c) for c in idx], dtype=np.int64)
    pts = np.array([[grid.lo[a] + (c[a] + 0.5) * grid.step[a] for a in range(4)] for c in idx])
    return pts, cells


def tiny_scene(seed: int = 1, snr_db: Optional[float] = 20.0, on_grid: bool = False) -> Scene:
    """1 TX at the origin, Q = 3 RX at seeded angles on a 10 m circle,
    Ms = 64 x Mc = 32, Tc = 100 us, one unit-modulus random-phase target."""
    radar = Radar(24e9, 250e6, 100e-6, 64, 32, 4)
    grid = Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (32, 32, 8, 8))
    ang = 2.0 * np.pi * uniform(seed, _S_RX, 3)
    rx = 10.0 * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    cells = None
    if on_grid:
        tg, cells = _ongrid_targets(seed, grid, 1)
    else:
        pos = _uniform_box(seed, _S_TGT_POS, 1, 0.0, 20.0)
        vel = _uniform_box(seed, _S_TGT_VEL, 1, -10.0, 10.0)
        tg = np.concatenate([pos, vel], axis=1)
    alpha = _unit_phase(seed, (1, 3))
    return Scene("tiny", seed, radar, np.zeros(2), rx, tg, alpha,
                 _noise(seed, 3, radar, snr_db), grid, 1, snr_db, cells)


def paper_frame(seed: int = 1, snr_db: Optional[float] = 10.0, on_grid: bool = False,
                T: int = 3) -> Scene:
    """Paper-shaped frame: Q = 4 RX spread over 30 m (x in [-5, 25], y in
    [-3, -1]), Ms = 256 x Mc = 128, Tc = 128 us, T Rayleigh targets in
    [0, 40]^2 m with velocities in [-15, 15]^2 m/s, K = T detections."""
    radar = Radar(24e9, 250e6, 128e-6, 256, 128, 4)
    grid = Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (128, 128, 32, 32))
    u = uniform(seed, _S_RX, 8).reshape(4, 2)
    rx = np.stack([-5.0 + 30.0 * u[:, 0], -3.0 + 2.0 * u[:, 1]], axis=1)
    cells = None
    if on_grid:
        tg, cells = _ongrid_targets(seed, grid, T)
    else:
        pos = _uniform_box(seed, _S_TGT_POS, T, 0.0, 40.0)
        vel = _uniform_box(seed, _S_TGT_VEL, T, -15.0, 15.0)
        tg = np.concatenate([pos, vel], axis=1)
    alpha = _rayleigh_alpha(seed, T, 4)
    return Scene("paper_frame", seed, radar, np.zeros(2), rx, tg, alpha,
                 _noise(seed, 4, radar, snr_db), grid, T, snr_db, cells)


def precision_scene(seed: int = 1, snr_db: Optional[float] = 5.0, on_grid: bool = False) -> Scene:
    """Q = 8 RX spread over 30 m, Ms = 512 x Mc = 256, Tc = 128 us, five
    Rayleigh targets, grid 256 x 256 x 64 x 64 over [0, 40]^2 x [-15, 15]^2."""
    radar = Radar(24e9, 250e6, 128e-6, 512, 256, 4)
    grid = Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (256, 256, 64, 64))
    u = uniform(seed, _S_RX, 16).reshape(8, 2)
    rx = np.stack([-5.0 + 30.0 * u[:, 0], -3.0 + 2.0 * u[:, 1]], axis=1)
    T = 5
    cells = None
    if on_grid:
        tg, cells = _ongrid_targets(seed, grid, T)
    else:
        pos = _uniform_box(seed, _S_TGT_POS, T, 0.0, 40.0)
        vel = _uniform_box(seed, _S_TGT_VEL, T, -15.0, 15.0)
        tg = np.concatenate([pos, vel], axis=1)
    alpha = _rayleigh_alpha(seed, T, 8)
    return Scene("precision", seed, radar, np.zeros(2), rx, tg, alpha,
                 _noise(seed, 8, radar, snr_db), grid, T, snr_db, cells)


def custom_scene(seed: int, radar: Radar, grid: Grid, Q: int, T: int,
                 snr_db: Optional[float] = 10.0, on_grid: bool = False,
                 rx_box=((-5.0, 25.0), (-3.0, -1.0))) -> Scene:
    """A scene of any size (for ragged and edge-case tests): RX uniform in
    rx_box, targets uniform over the grid's extent, Rayleigh amplitudes."""
    u = uniform(seed, _S_RX, 2 * Q).reshape(Q, 2)
    (x0, x1), (y0, y1) = rx_box
    rx = np.stack([x0 + (x1 - x0) * u[:, 0], y0 + (y1 - y0) * u[:, 1]], axis=1)
    cells = None
    if on_grid:
        tg, cells = _ongrid_targets(seed, grid, T)
    else:
        hi = [grid.lo[a] + grid.n[a] * grid.step[a] for a in range(4)]
        p = uniform(seed, _S_TGT_POS, 4 * T).reshape(T, 4)
        tg = np.array(grid.lo) + (np.array(hi) - np.array(grid.lo)) * p
    alpha = _rayleigh_alpha(seed, T, Q)
    return Scene("custom", seed, radar, np.zeros(2), rx, tg, alpha,
                 _noise(seed, Q, radar, snr_db), grid, T, snr_db, cells)


def batch_scenes(seed: int, n: int, small: bool = False):
    """n frames of uneven size; frame i uses seed (seed * 100003 + i) for its
    own draws. ``small`` scales the sizes down (Ms in {32, 64}, Mc in {16, 32},
    (x, y) sides in {8, 12, 16}, velocity sides in {4, 6, 8}) so that the FP64
    oracle can score every frame."""
    u = uniform(seed, _S_BATCH, 8 * n).reshape(n, 8)
    pick = lambda opts, v: opts[min(int(v * len(opts)), len(opts) - 1)]
    frames = []
    for i in range(n):
        Q = 3 + min(int(u[i, 0] * 6), 5)
        if small:
            Ms, Mc = pick((32, 64), u[i, 1]), pick((16, 32), u[i, 2])
            nxy, nv = pick((8, 12, 16), u[i, 3]), pick((4, 6, 8), u[i, 4])
        else:
            Ms, Mc = pick((128, 256, 512), u[i, 1]), pick((64, 128, 256), u[i, 2])
            nxy, nv = pick((64, 96, 128, 160), u[i, 3]), pick((16, 24, 32, 40), u[i, 4])
        T = 1 + min(int(u[i, 5] * 5), 4)
        snr = 20.0 * u[i, 6]
        radar = Radar(24e9, 250e6, 128e-6, Ms, Mc, 4)
        grid = Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (nxy, nxy, nv, nv))
        sc = custom_scene(seed * 100003 + i, radar, grid, Q=Q, T=T, snr_db=snr)
        frames.append(replace(sc, name="batch"))
    return frames
