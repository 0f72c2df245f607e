"""Seeded synthetic inputs for MRF dictionary generating and searching (DGS).

This module is shared by the FP64 oracle (``oracle/``) and the GPU library
(``paper_1506_05393_gb300``). It holds only random draws and data layout: no
Bloch simulation, no correlation, no search. Everything the method computes
lives in those two packages, which never import each other.

Contents
--------
* ``sequence(seed, n)``: the randomised IR-bSSFP acquisition train. The paper's
  own recipe (Perlin-noise flip angles, 0/90/180 degree RF phases, Gaussian TRs;
  *Methods*, Experiment 1) has no published seed or noise parameters, so the
  stand-in recipe used throughout is: flip angle
  ``alpha_j = (-1)^j (10 + 50 |sin(pi j / 250)| + u_j)`` degrees with
  ``u_j ~ U(0, 5)``, ``TR_j ~ U(10.5, 14)`` ms, ``TE_j = TR_j / 2``, preceded
  by an ideal 180 degree inversion and a 20 ms delay. ``sequence_paper`` is a
  seeded stand-in shaped like the paper's recipe (gradient-noise flip angles,
  0/90/180 degree phases, Gaussian TRs), and ``with_pulses`` gives any train
  RF pulses of finite duration (the Appendix's off-resonant RF form).
* ``GRIDS``: the (T1, T2, df) search grids of the workloads, as plain numbers.
* ``phantom_*``: per-voxel true parameters, proton density, global phase and
  standard-normal noise draws.
* ``compose_voxels``: scales clean simulated signals by M0 e^{i phase} and adds
  complex white Gaussian noise at a given SNR (*Methods*, Experiment 4 adds
  white noise to the real and imaginary parts). The clean signals come from
  whichever simulator the caller trusts; this module never simulates.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict

import numpy as np

__all__ = [
    "Sequence", "Grid", "GRIDS", "sequence", "sequence_paper", "with_pulses", "grid_values", "grid_valid_params", "phantom_piecewise",
    "phantom_offgrid", "phantom_ongrid", "noise_draws", "compose_voxels",
    "write_sequence", "read_sequence",
]


@dataclass(frozen=True)
class Sequence:
    """IR-bSSFP train: per-timepoint signed flip (rad), RF phase (rad), TR and TE (ms)."""
    flip_rad: np.ndarray      # (n,) float64, signed: + at j = 0, alternating
    rf_phase_rad: np.ndarray  # (n,) float64, all zero for the alternating-sign recipe
    tr_ms: np.ndarray         # (n,) float64
    te_ms: np.ndarray         # (n,) float64
    inversion: int = 1
    inv_delay_ms: float = 20.0
    pulse_ms: np.ndarray | None = None   # (n,) RF pulse durations in ms; None: hard pulses

    @property
    def n(self) -> int:
        return int(self.flip_rad.shape[0])


def with_pulses(seq: Sequence, tau_ms) -> Sequence:
    """The same train with RF pulses of duration tau_ms (scalar or (n,))."""
    from dataclasses import replace
    return replace(seq, pulse_ms=np.broadcast_to(np.asarray(tau_ms, np.float64), (seq.n,)).copy())


def _gradient_noise_1d(rng, n: int, cell: float) -> np.ndarray:
    """Perlin's gradient noise in one dimension (K. Perlin, "Improving noise",
    SIGGRAPH 2002): a random gradient in [-1, 1] at each lattice point (spacing
    `cell` samples), the contribution g_i (x - i) of the two neighbouring
    lattice points blended with the quintic fade 6t^5 - 15t^4 + 10t^3."""
    x = np.arange(n) / cell
    i0 = np.floor(x).astype(np.int64)
    g = rng.uniform(-1.0, 1.0, int(i0.max()) + 2)
    t = x - i0
    fade = t * t * t * (t * (t * 6.0 - 15.0) + 10.0)
    return (1.0 - fade) * g[i0] * t + fade * g[i0 + 1] * (t - 1.0)


def sequence_paper(seed: int, n: int, pulse_ms=None) -> Sequence:
    """A stand-in for the paper's own train (Methods, Experiment 1), whose
    noise parameters and seed are unpublished: flip angles from 1D gradient
    (Perlin) noise rescaled to 0-79 degrees, RF phases oscillating 0, 90,
    180, 90, 0, ... degrees, TR from Gaussian noise remapped to 0-6 ms plus
    the 14 ms minimum, TE = TR / 2, an ideal inversion and a 20 ms delay;
    optional RF pulse durations. Draw order: gradients, then the TR noise."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    p = _gradient_noise_1d(rng, n, 40.0)
    span = p.max() - p.min()
    deg = 79.0 * (p - p.min()) / span if span > 0 else np.zeros(n)
    g = rng.normal(0.0, 1.0, n)
    gs = g.max() - g.min()
    tr = 14.0 + (6.0 * (g - g.min()) / gs if gs > 0 else np.zeros(n))
    phase = np.deg2rad(np.array([0.0, 90.0, 180.0, 90.0])[np.arange(n) % 4])
    seq = Sequence(flip_rad=np.deg2rad(deg), rf_phase_rad=phase, tr_ms=tr, te_ms=tr / 2.0, inversion=1,
                   inv_delay_ms=20.0)
    return seq if pulse_ms is None else with_pulses(seq, pulse_ms)


def sequence(seed: int, n: int) -> Sequence:
    """The seeded acquisition train (draw order: u first, then TR)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 5.0, n)
    tr = rng.uniform(10.5, 14.0, n)
    j = np.arange(n)
    deg = 10.0 + 50.0 * np.abs(np.sin(np.pi * j / 250.0)) + u
    sign = np.where(j % 2 == 0, 1.0, -1.0)
    flip = np.deg2rad(sign * deg)
    return Sequence(flip_rad=flip.astype(np.float64),
                    rf_phase_rad=np.zeros(n, np.float64),
                    tr_ms=tr.astype(np.float64),
                    te_ms=(tr / 2.0).astype(np.float64),
                    inversion=1, inv_delay_ms=20.0)


def write_sequence(seq: Sequence, path: str) -> None:
    """Little-endian binary: int32 n, int32 inversion, f64 delay, then 4 arrays of n f64."""
    with open(path, "wb") as f:
        np.array([seq.n, seq.inversion], "<i4").tofile(f)
        np.array([seq.inv_delay_ms], "<f8").tofile(f)
        for a in (seq.flip_rad, seq.rf_phase_rad, seq.tr_ms, seq.te_ms):
            np.asarray(a, "<f8").tofile(f)


def read_sequence(path: str) -> Sequence:
    with open(path, "rb") as f:
        n, inv = np.fromfile(f, "<i4", 2)
        delay = float(np.fromfile(f, "<f8", 1)[0])
        arrs = [np.fromfile(f, "<f8", int(n)) for _ in range(4)]
    return Sequence(*arrs, inversion=int(inv), inv_delay_ms=delay)


@dataclass(frozen=True)
class Grid:
    """Uniform (T1, T2, df) grid; value i of an axis is ``min + i * step``.

    An entry is valid iff T2 < T1 (when ``require_t2_lt_t1``). Linear entry
    order: T1 outermost, T2 next, df innermost, valid entries only.
    """
    t1_min: float
    t1_step: float
    n_t1: int
    t2_min: float
    t2_step: float
    n_t2: int
    df_min: float
    df_step: float
    n_df: int
    require_t2_lt_t1: int = 1

    def asdict(self):
        return asdict(self)


def _axis(lo, hi, step):
    return int(round((hi - lo) / step)) + 1


GRIDS = {
    # 16x16 voxels, N = 200
    "tiny": Grid(100.0, 100.0, _axis(100, 2000, 100), 20.0, 20.0, _axis(20, 200, 20),
                 0.0, 1.0, 1),
    # 64x64 voxels, N = 1000, FP32 brute force
    "fp32_brute": Grid(100.0, 20.0, _axis(100, 4000, 20), 10.0, 5.0, _axis(10, 400, 5),
                       -40.0, 2.0, _axis(-40, 40, 2)),
    # same slice, finer grid for the BF16 / FP8 + re-score forms
    "precision": Grid(100.0, 5.0, _axis(100, 4000, 5), 10.0, 2.0, _axis(10, 400, 2),
                      -40.0, 1.0, _axis(-40, 40, 1)),
    # ZOOM only (about 2.4e9 entries, never materialised)
    "zoom_fine": Grid(100.0, 1.0, _axis(100, 4000, 1), 10.0, 0.5, _axis(10, 400, 0.5),
                      -40.0, 0.1, _axis(-40, 40, 0.1)),
}


def grid_values(g: Grid):
    """Axis values, each ``min + i * step`` (never cumulative sums)."""
    t1 = g.t1_min + np.arange(g.n_t1) * g.t1_step
    t2 = g.t2_min + np.arange(g.n_t2) * g.t2_step
    df = g.df_min + np.arange(g.n_df) * g.df_step
    return t1, t2, df


def grid_valid_params(g: Grid):
    """(a, b, c) index arrays of valid entries in linear order (small grids only)."""
    t1, t2, _ = grid_values(g)
    a, b, c = np.meshgrid(np.arange(g.n_t1), np.arange(g.n_t2), np.arange(g.n_df), indexing="ij")
    a, b, c = a.ravel(), b.ravel(), c.ravel()
    if g.require_t2_lt_t1:
        keep = t2[b] < t1[a]
        a, b, c = a[keep], b[keep], c[keep]
    return a.astype(np.int64), b.astype(np.int64), c.astype(np.int64)


def phantom_offgrid(seed: int, v: int, t1_range=(200.0, 3000.0), t2_range=(20.0, 300.0),
                    df_range=(-40.0, 40.0)):
    """Off-grid voxel parameters: T1, T2 log-uniform (resampled until T2 < T1),
    df uniform, M0 ~ U(0.5, 1), global phase ~ U(0, 2 pi). Draw order is fixed."""
    rng = np.random.default_rng(seed)
    t1 = np.exp(rng.uniform(math.log(t1_range[0]), math.log(t1_range[1]), v))
    t2 = np.exp(rng.uniform(math.log(t2_range[0]), math.log(t2_range[1]), v))
    bad = t2 >= t1
    while bad.any():
        k = int(bad.sum())
        t1[bad] = np.exp(rng.uniform(math.log(t1_range[0]), math.log(t1_range[1]), k))
        t2[bad] = np.exp(rng.uniform(math.log(t2_range[0]), math.log(t2_range[1]), k))
        bad = t2 >= t1
    df = rng.uniform(df_range[0], df_range[1], v)
    m0 = rng.uniform(0.5, 1.0, v)
    ph = rng.uniform(0.0, 2.0 * math.pi, v)
    return dict(t1=t1, t2=t2, df=df, m0=m0, phase=ph, rng_state=rng.bit_generator.state)


def phantom_piecewise(seed: int, rows: int, cols: int, classes: int = 5, t1_range=(200.0, 3000.0),
                      t2_range=(20.0, 300.0), df_range=(-40.0, 40.0)):
    """A piecewise-smooth slice (row-major, rows x cols voxels), for searches
    that use spatial neighbours: `classes` tissue classes with T1, T2
    log-uniform (T2 < T1) and df uniform, laid out by the largest of smooth
    random fields (one per class, a sum of Gaussian blobs), then 2 % jitter on
    T1 and T2 and a +-3 Hz df gradient across the slice; M0 ~ U(0.5, 1) and
    global phase ~ U(0, 2 pi) per voxel. Draw order is fixed."""
    rng = np.random.default_rng(seed)
    ct1 = np.exp(rng.uniform(math.log(t1_range[0]), math.log(t1_range[1]), classes))
    ct2 = np.minimum(np.exp(rng.uniform(math.log(t2_range[0]), math.log(t2_range[1]), classes)), 0.8 * ct1)
    cdf = rng.uniform(df_range[0] + 3.0, df_range[1] - 3.0, classes)
    yy, xx = np.mgrid[0:rows, 0:cols].astype(np.float64)
    field = np.zeros((classes, rows, cols))
    for k in range(classes):
        for _ in range(8):
            cy, cx = rng.uniform(0, rows), rng.uniform(0, cols)
            r = rng.uniform(0.08, 0.25) * max(rows, cols)
            field[k] += rng.uniform(0.5, 1.0) * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * r * r))
    label = field.argmax(0).ravel()
    v = rows * cols
    t1 = ct1[label] * (1.0 + 0.02 * rng.uniform(-1, 1, v))
    t2 = ct2[label] * (1.0 + 0.02 * rng.uniform(-1, 1, v))
    df = cdf[label] + 3.0 * (xx.ravel() / max(cols - 1, 1) * 2.0 - 1.0)
    m0 = rng.uniform(0.5, 1.0, v)
    ph = rng.uniform(0.0, 2.0 * math.pi, v)
    return dict(t1=t1, t2=t2, df=df, m0=m0, phase=ph, label=label)


def phantom_ongrid(seed: int, v: int, g: Grid):
    """Voxels placed on random valid grid points, with M0 ~ U(0.5, 1) and phase ~ U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    a, b, c = grid_valid_params(g)
    idx = rng.integers(0, a.shape[0], v)
    t1, t2, df = grid_values(g)
    m0 = rng.uniform(0.5, 1.0, v)
    ph = rng.uniform(0.0, 2.0 * math.pi, v)
    return dict(index=idx, a=a[idx], b=b[idx], c=c[idx], t1=t1[a[idx]], t2=t2[b[idx]],
                df=df[c[idx]], m0=m0, phase=ph)


def noise_draws(seed: int, v: int, n: int):
    """Two (v, n) standard-normal arrays: real then imaginary parts."""
    rng = np.random.default_rng(seed + 7919)
    g_re = rng.standard_normal((v, n))
    g_im = rng.standard_normal((v, n))
    return g_re, g_im


def compose_voxels(clean: np.ndarray, m0: np.ndarray, phase: np.ndarray, g_re: np.ndarray,
                   g_im: np.ndarray, snr: float | None) -> np.ndarray:
    """x_v = m0_v e^{i phase_v} s_v + (sigma_v / sqrt 2)(g + i g') with
    sigma_v = rms_j |m0_v s_v,j| / snr (no noise when snr is None or inf).

    ``clean`` is a (v, n) complex array of simulated signals. Returns complex128.
    """
    s = np.asarray(clean, np.complex128) * (np.asarray(m0)[:, None] * np.exp(1j * np.asarray(phase))[:, None])
    if snr is None or not np.isfinite(snr):
        return s
    sigma = np.sqrt(np.mean(np.abs(s) ** 2, axis=1)) / float(snr)
    return s + (sigma[:, None] / math.sqrt(2.0)) * (g_re + 1j * g_im)
