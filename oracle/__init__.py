"""FP64 CPU oracle for MRF DGS (ctypes wrapper around ``mrf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it. The GPU library never imports it and it
never imports the GPU library; the two share only ``mrf_synth`` (random draws).

Every function follows the paper directly:
  * ``simulate`` / ``simulate_state``: Appendix Eq. A2 with the hard-pulse RF
    form (or, for pulses of finite duration, the Appendix's off-resonant
    effective-field form) and the recovery term of Eq. A1.
  * ``cc``: Eq. 1.
  * ``bruteforce``: argmax of Eq. 1 over every valid grid entry.
  * ``zoom`` / ``zoom_generic``: MRF-ZOOM, Theory (df search steps 1-4, Fig. 1
    1D ZOOM, Fig. 2 2D ZOOM) with the schedule of Experiment 2 steps 1-5.
Parity unpinned: ZOOM on grids too large for exhaustive search (only
local-optimality and windowed brute-force checks apply there).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_mrf.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 16


class OrSeq(C.Structure):
    _fields_ = [("n", C.c_int32), ("flip", C.POINTER(C.c_double)), ("phase", C.POINTER(C.c_double)),
                ("tr", C.POINTER(C.c_double)), ("te", C.POINTER(C.c_double)),
                ("inversion", C.c_int32), ("inv_delay", C.c_double), ("pulse", C.POINTER(C.c_double))]


class OrGrid(C.Structure):
    _fields_ = [("t1_min", C.c_double), ("t1_step", C.c_double), ("n_t1", C.c_int32),
                ("t2_min", C.c_double), ("t2_step", C.c_double), ("n_t2", C.c_int32),
                ("df_min", C.c_double), ("df_step", C.c_double), ("n_df", C.c_int32),
                ("require_t2_lt_t1", C.c_int32)]


class OrZoomOpts(C.Structure):
    _fields_ = [("omega_hz", C.c_double), ("t1_init_ms", C.c_double), ("t2_init_ms", C.c_double),
                ("s1a_step_frac", C.c_double), ("s1b_half_frac", C.c_double),
                ("s1b_step_frac", C.c_double), ("s3_half_frac", C.c_double),
                ("n_s2", C.c_int32), ("s2_t1_ms", C.c_double * MAX_LEVELS),
                ("s2_t2_ms", C.c_double * MAX_LEVELS), ("n_s4", C.c_int32),
                ("s4_param", C.c_int32 * MAX_LEVELS), ("s4_ms", C.c_double * MAX_LEVELS)]


SCORE_FN = C.CFUNCTYPE(C.c_double, C.c_void_p, C.c_int32, C.c_int32, C.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, C11, OpenMP, no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        lp = C.POINTER(C.c_int64)
        L.or_simulate_state.argtypes = [C.POINTER(OrSeq), C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.or_simulate.argtypes = [C.POINTER(OrSeq), C.c_int64, dp, dp, dp, dp]
        L.or_cc.argtypes = [C.c_int32, dp, dp]
        L.or_cc.restype = C.c_double
        L.or_grid_count.argtypes = [C.POINTER(OrGrid)]
        L.or_grid_count.restype = C.c_int64
        L.or_grid_index.argtypes = [C.POINTER(OrGrid), C.c_int32, C.c_int32, C.c_int32]
        L.or_grid_index.restype = C.c_int64
        L.or_grid_params.argtypes = [C.POINTER(OrGrid), C.c_int64, ip, ip, ip]
        L.or_grid_params.restype = C.c_int64
        L.or_bruteforce.argtypes = [C.POINTER(OrSeq), C.POINTER(OrGrid), dp, C.c_int64, C.c_int32, lp, dp, dp, dp]
        L.or_zoom_generic.argtypes = [C.POINTER(OrGrid), C.POINTER(OrZoomOpts), C.c_double, SCORE_FN, C.c_void_p,
                                      ip, dp, ip, dp, C.c_int32, ip, ip, dp]
        L.or_zoom.argtypes = [C.POINTER(OrSeq), C.POINTER(OrGrid), C.POINTER(OrZoomOpts), dp, C.c_int64,
                              ip, dp, dp, dp, ip, dp]
        L.or_smooth.argtypes = [C.c_int32, C.c_int64, dp, C.c_int32, C.c_double, dp]
        L.or_bruteforce_smooth.argtypes = [C.POINTER(OrSeq), C.POINTER(OrGrid), dp, C.c_int64, C.c_int32, C.c_int32,
                                           C.c_double, lp, dp, dp, dp]
        L.or_refine_generic.argtypes = [C.POINTER(OrGrid), C.c_int32, SCORE_FN, C.c_void_p, ip, dp, ip, dp]
        L.or_refine.argtypes = [C.POINTER(OrSeq), C.POINTER(OrGrid), dp, C.c_int64, C.c_int32, ip, dp, dp, dp, ip, dp]
        L.or_default_omega.argtypes = [C.POINTER(OrSeq)]
        L.or_default_omega.restype = C.c_double
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class _SeqHandle:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, seq):
        self.flip = np.ascontiguousarray(seq.flip_rad, np.float64)
        self.phase = np.ascontiguousarray(seq.rf_phase_rad, np.float64) if seq.rf_phase_rad is not None else None
        self.tr = np.ascontiguousarray(seq.tr_ms, np.float64)
        self.te = np.ascontiguousarray(seq.te_ms, np.float64)
        pulse = getattr(seq, "pulse_ms", None)
        self.pulse = np.ascontiguousarray(pulse, np.float64) if pulse is not None else None
        self.c = OrSeq(int(self.flip.shape[0]), _dp(self.flip),
                       _dp(self.phase) if self.phase is not None else C.POINTER(C.c_double)(),
                       _dp(self.tr), _dp(self.te), int(seq.inversion), float(seq.inv_delay_ms),
                       _dp(self.pulse) if self.pulse is not None else C.POINTER(C.c_double)())


def _grid(g) -> OrGrid:
    return OrGrid(g.t1_min, g.t1_step, g.n_t1, g.t2_min, g.t2_step, g.n_t2,
                  g.df_min, g.df_step, g.n_df, g.require_t2_lt_t1)


def default_zoom_opts(**kw) -> OrZoomOpts:
    """Experiment 2 schedule: df search (coarse step 6/7 omega, window +-omega
    at omega/20, probes at k omega), 2D ZOOM at 200 then 100 ms, df refinement
    over +-omega/2 at the finest step, 1D ZOOMs T1@100, T2@100, T1@50/20/10,
    T2@50/20/10, final 2D ZOOM at the finest step. Start at T1/T2 = 1000/100 ms."""
    o = OrZoomOpts()
    o.omega_hz = kw.get("omega_hz", 0.0)
    o.t1_init_ms = kw.get("t1_init_ms", 1000.0)
    o.t2_init_ms = kw.get("t2_init_ms", 100.0)
    o.s1a_step_frac = kw.get("s1a_step_frac", 6.0 / 7.0)
    o.s1b_half_frac = kw.get("s1b_half_frac", 1.0)
    o.s1b_step_frac = kw.get("s1b_step_frac", 1.0 / 20.0)
    o.s3_half_frac = kw.get("s3_half_frac", 0.5)
    s2 = kw.get("s2", [(200.0, 200.0), (100.0, 100.0)])
    o.n_s2 = len(s2)
    for i, (h1, h2) in enumerate(s2):
        o.s2_t1_ms[i] = h1
        o.s2_t2_ms[i] = h2
    s4 = kw.get("s4", [(0, 100.0), (1, 100.0), (0, 50.0), (0, 20.0), (0, 10.0),
                       (1, 50.0), (1, 20.0), (1, 10.0)])
    o.n_s4 = len(s4)
    for i, (p, h) in enumerate(s4):
        o.s4_param[i] = p
        o.s4_ms[i] = h
    return o


def num_threads() -> int:
    return int(lib().or_num_threads())


def simulate_state(seq, t1, t2, df, m_init=None):
    """(signal (n,) complex128, state (n, 3)) of one fingerprint."""
    h = _SeqHandle(seq)
    n = h.c.n
    sig = np.zeros(2 * n)
    st = np.zeros(3 * n)
    mi = None
    if m_init is not None:
        mi = np.ascontiguousarray(m_init, np.float64)
    rc = lib().or_simulate_state(C.byref(h.c), float(t1), float(t2), float(df),
                                 _dp(mi) if mi is not None else C.POINTER(C.c_double)(), _dp(sig), _dp(st))
    assert rc == 0
    return sig[0::2] + 1j * sig[1::2], st.reshape(n, 3)


def simulate(seq, t1, t2, df):
    """(count, n) complex128 fingerprints for parameter arrays."""
    t1 = np.ascontiguousarray(np.atleast_1d(t1), np.float64)
    t2 = np.ascontiguousarray(np.broadcast_to(t2, t1.shape), np.float64)
    df = np.ascontiguousarray(np.broadcast_to(df, t1.shape), np.float64)
    h = _SeqHandle(seq)
    n = h.c.n
    out = np.zeros((t1.shape[0], n, 2))
    rc = lib().or_simulate(C.byref(h.c), t1.shape[0], _dp(t1), _dp(t2), _dp(df), _dp(out))
    assert rc == 0
    return out[..., 0] + 1j * out[..., 1]


def _interleave(x):
    x = np.asarray(x, np.complex128)
    out = np.empty(x.shape + (2,))
    out[..., 0] = x.real
    out[..., 1] = x.imag
    return np.ascontiguousarray(out)


def cc(x, d) -> float:
    xi, di = _interleave(x), _interleave(d)
    return float(lib().or_cc(xi.shape[0], _dp(xi), _dp(di)))


def grid_count(g) -> int:
    return int(lib().or_grid_count(C.byref(_grid(g))))


def grid_index(g, a, b, c) -> int:
    return int(lib().or_grid_index(C.byref(_grid(g)), int(a), int(b), int(c)))


def grid_params(g):
    gc = _grid(g)
    n = int(lib().or_grid_count(C.byref(gc)))
    a = np.zeros(n, np.int32)
    b = np.zeros(n, np.int32)
    c = np.zeros(n, np.int32)
    lib().or_grid_params(C.byref(gc), n, _ip(a), _ip(b), _ip(c))
    return a, b, c


def bruteforce(seq, g, x, k: int = 1, smooth=None):
    """Top-k by Eq. 1 for each voxel. Returns dict(idx (V,k), cc (V,k), m0 (V,), phase (V,)).
    smooth = (width, sigma): the dictionary entries are smoothed first (x is used as given)."""
    h = _SeqHandle(seq)
    xi = _interleave(np.atleast_2d(x))
    V = xi.shape[0]
    idx = np.zeros((V, k), np.int64)
    ccs = np.zeros((V, k))
    m0 = np.zeros(V)
    ph = np.zeros(V)
    lp = C.POINTER(C.c_int64)
    if smooth is None:
        rc = lib().or_bruteforce(C.byref(h.c), C.byref(_grid(g)), _dp(xi), V, k, idx.ctypes.data_as(lp), _dp(ccs),
                                 _dp(m0), _dp(ph))
    else:
        rc = lib().or_bruteforce_smooth(C.byref(h.c), C.byref(_grid(g)), _dp(xi), V, k, int(smooth[0]),
                                        float(smooth[1]), idx.ctypes.data_as(lp), _dp(ccs), _dp(m0), _dp(ph))
    if rc != 0:
        raise RuntimeError(f"or_bruteforce failed: {rc}")
    return dict(idx=idx, cc=ccs, m0=m0, phase=ph)


def smooth(x, width: int, sigma: float = 1.0):
    """Temporal smoothing of V x n complex timecourses (Experiment 4)."""
    x2 = np.atleast_2d(np.asarray(x, np.complex128))
    V, n = x2.shape
    xi = _interleave(x2)
    out = np.zeros_like(xi)
    rc = lib().or_smooth(n, V, _dp(xi), int(width), float(sigma), _dp(out))
    if rc != 0:
        raise RuntimeError(f"or_smooth failed: {rc}")
    return out[..., 0] + 1j * out[..., 1]


def default_omega(seq) -> float:
    return float(lib().or_default_omega(C.byref(_SeqHandle(seq).c)))


def zoom(seq, g, x, opts=None):
    """MRF-ZOOM per voxel. Returns dict(abc (V,3), cc, m0, phase, evaluated, min_margin)."""
    h = _SeqHandle(seq)
    xi = _interleave(np.atleast_2d(x))
    V = xi.shape[0]
    o = opts if opts is not None else default_zoom_opts()
    abc = np.zeros((V, 3), np.int32)
    ccs = np.zeros(V)
    m0 = np.zeros(V)
    ph = np.zeros(V)
    ev = np.zeros(V, np.int32)
    mm = np.zeros(V)
    rc = lib().or_zoom(C.byref(h.c), C.byref(_grid(g)), C.byref(o), _dp(xi), V,
                       _ip(abc), _dp(ccs), _dp(m0), _dp(ph), _ip(ev), _dp(mm))
    if rc != 0:
        raise RuntimeError(f"or_zoom failed: {rc}")
    return dict(abc=abc, cc=ccs, m0=m0, phase=ph, evaluated=ev, min_margin=mm)


class _SubGrid:
    """A grid restricted to index boxes [a_lo, a_hi] x [b_lo, b_hi] x [c_lo, c_hi]
    of `g` (same steps; first values those of the box's first points)."""

    def __init__(self, g, a_lo, a_hi, b_lo, b_hi, c_lo, c_hi):
        self.t1_min, self.t1_step, self.n_t1 = g.t1_min + a_lo * g.t1_step, g.t1_step, a_hi - a_lo + 1
        self.t2_min, self.t2_step, self.n_t2 = g.t2_min + b_lo * g.t2_step, g.t2_step, b_hi - b_lo + 1
        self.df_min, self.df_step, self.n_df = g.df_min + c_lo * g.df_step, g.df_step, c_hi - c_lo + 1
        self.require_t2_lt_t1 = g.require_t2_lt_t1


def prior_box(g, abc_p, half):
    """Index box of the grid points within `half` = (T1, T2, df) half-widths of
    the preceding voxel's grid point abc_p, overlapped with the grid (Methods,
    Experiment 3: the ranges T1p +- 3000, T2p +- 800, dfp +- 150 overlapped
    with the original searching ranges)."""
    h = [int(math.floor(w / st + 1e-9)) for w, st in zip(half, (g.t1_step, g.t2_step, g.df_step))]
    n = (g.n_t1, g.n_t2, g.n_df)
    return [(max(0, int(abc_p[k]) - h[k]), min(n[k] - 1, int(abc_p[k]) + h[k])) for k in range(3)]


def zoom_prior_one(seq, g, x, abc_p, half=(3000.0, 800.0, 150.0), start_from_prior=True, opts=None):
    """One voxel's MRF-ZOOM under the spatial-neighbour prior (Methods,
    Experiment 3): the search runs on the grid overlapped with the ranges
    around the preceding voxel's result abc_p, as a search on that sub-grid
    of its own; with start_from_prior the ZOOM starts at the preceding voxel's
    (T1, T2) (Theory, 1D ZOOM: the initial centre may be the parameter value
    of the neighbouring voxel), else at the options' start clipped into the
    ranges. Returns zoom()'s dict for this voxel (global indices) plus `box`."""
    (a0, a1), (b0, b1), (c0, c1) = prior_box(g, abc_p, half)
    sub = _SubGrid(g, a0, a1, b0, b1, c0, c1)
    o = opts if opts is not None else default_zoom_opts()
    if start_from_prior:
        o2 = OrZoomOpts()
        C.pointer(o2)[0] = o
        o2.t1_init_ms = g.t1_min + int(abc_p[0]) * g.t1_step
        o2.t2_init_ms = g.t2_min + int(abc_p[1]) * g.t2_step
        o = o2
    r = zoom(seq, sub, np.atleast_2d(x), o)
    out = {k: r[k][0] for k in ("cc", "m0", "phase", "evaluated", "min_margin")}
    out["abc"] = r["abc"][0] + np.array([a0, b0, c0], np.int32)
    out["box"] = np.array([a0, a1, b0, b1, c0, c1], np.int32)
    return out


def zoom_prior(seq, g, x, chain=None, half=(3000.0, 800.0, 150.0), start_from_prior=True, opts=None):
    """MRF-ZOOM with the spatial-neighbour prior (Methods, Experiment 3), in
    the voxels' given (raster) order: each voxel's search is bounded by, and
    (with start_from_prior) started from, the result of the voxel before it.
    chain = None is the paper's single chain through all voxels; chain = L
    cuts the voxels into consecutive chains of L, the first voxel of each
    searched on the whole grid like the first voxel of the slice. A plain
    sequential loop; returns zoom()'s dict (global indices) plus `box`."""
    x = np.atleast_2d(x)
    V = x.shape[0]
    L = V if chain is None else int(chain)
    if L < 1:
        raise ValueError("chain length must be >= 1")
    out = dict(abc=np.zeros((V, 3), np.int32), cc=np.zeros(V), m0=np.zeros(V), phase=np.zeros(V),
               evaluated=np.zeros(V, np.int32), min_margin=np.zeros(V), box=np.zeros((V, 6), np.int32))
    for v in range(V):
        if v % L == 0:
            r = zoom(seq, g, x[v:v + 1], opts)
            r = {k: r[k][0] for k in r}
            r["box"] = np.array([0, g.n_t1 - 1, 0, g.n_t2 - 1, 0, g.n_df - 1], np.int32)
        else:
            r = zoom_prior_one(seq, g, x[v], out["abc"][v - 1], half, start_from_prior, opts)
        for k in out:
            out[k][v] = r[k]
    return out


def zoom_generic(g, score, omega, opts=None, trace_cap=100000):
    """ZOOM over a Python score(a, b, c) -> float (test hook for the stage machine)."""
    o = opts if opts is not None else default_zoom_opts()
    cb = SCORE_FN(lambda _ctx, a, b, c: float(score(a, b, c)))
    abc = np.zeros(3, np.int32)
    ccv = np.zeros(1)
    ev = np.zeros(1, np.int32)
    mm = np.zeros(1)
    tn = np.zeros(1, np.int32)
    tr = np.zeros((trace_cap, 4), np.int32)
    tcc = np.zeros(trace_cap)
    rc = lib().or_zoom_generic(C.byref(_grid(g)), C.byref(o), float(omega), cb, None,
                               _ip(abc), _dp(ccv), _ip(ev), _dp(mm), trace_cap, _ip(tn), _ip(tr), _dp(tcc))
    if rc != 0:
        raise RuntimeError(f"or_zoom_generic failed: {rc}")
    n = min(int(tn[0]), trace_cap)
    return dict(abc=tuple(int(v) for v in abc), cc=float(ccv[0]), evaluated=int(ev[0]),
                min_margin=float(mm[0]), trace=tr[:n].copy(), trace_cc=tcc[:n].copy())


def refine_generic(g, score, start, max_moves=1 << 20):
    """Windowed refinement over a Python score(a, b, c) -> float (test hook)."""
    cb = SCORE_FN(lambda _ctx, a, b, c: float(score(a, b, c)))
    abc = np.array(start, np.int32)
    ccv = np.zeros(1)
    ev = np.zeros(1, np.int32)
    mm = np.zeros(1)
    rc = lib().or_refine_generic(C.byref(_grid(g)), int(max_moves), cb, None, _ip(abc), _dp(ccv), _ip(ev), _dp(mm))
    if rc != 0:
        raise RuntimeError(f"or_refine_generic failed: {rc}")
    return dict(abc=tuple(int(v) for v in abc), cc=float(ccv[0]), evaluated=int(ev[0]), min_margin=float(mm[0]))


def refine(seq, g, x, start_abc, max_moves=1 << 20):
    """Windowed refinement per voxel from start_abc (V, 3). Returns dict(abc,
    cc, m0, phase, evaluated, min_margin)."""
    h = _SeqHandle(seq)
    xi = _interleave(np.atleast_2d(x))
    V = xi.shape[0]
    abc = np.ascontiguousarray(np.asarray(start_abc, np.int32).reshape(V, 3)).copy()
    ccs = np.zeros(V)
    m0 = np.zeros(V)
    ph = np.zeros(V)
    ev = np.zeros(V, np.int32)
    mm = np.zeros(V)
    rc = lib().or_refine(C.byref(h.c), C.byref(_grid(g)), _dp(xi), V, int(max_moves), _ip(abc), _dp(ccs), _dp(m0),
                         _dp(ph), _ip(ev), _dp(mm))
    if rc != 0:
        raise RuntimeError(f"or_refine failed: {rc}")
    return dict(abc=abc, cc=ccs, m0=m0, phase=ph, evaluated=ev, min_margin=mm)
