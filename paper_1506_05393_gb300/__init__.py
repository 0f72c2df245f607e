"""GB300 (sm_103a) MRF dictionary generating and searching -- Python binding.

A thin ctypes layer over ``libmrf_gb300.so`` (C ABI in ``include/mrf.h``):
argument marshalling only. Every computation runs in the library's CUDA
kernels; there is no CPU fallback, and importing this module on a machine
without the built library raises.

Method: Z. Wang, "MRF-ZOOM: A Fast Dictionary Searching Algorithm for
Magnetic Resonance Fingerprinting" -- Bloch-simulated fingerprints (Appendix,
Eq. A2), complex correlation (Eq. 1), brute-force DGS and MRF-ZOOM (Theory;
Methods, Experiment 2).

The functions named ``mrf_*`` mirror the C entry points one to one. Device
buffers are passed as torch CUDA tensors (their ``data_ptr()``), streams as
``torch.cuda.Stream`` (or None for the current stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MRF_OK, MRF_PENDING = 0, 1
MRF_E_INVALID, MRF_E_NOMEM, MRF_E_BUDGET, MRF_E_TIMEOUT = -1, -2, -3, -4
MRF_E_CUDA, MRF_E_NOTFOUND, MRF_E_UNSUPPORTED = -5, -6, -7
MRF_F32, MRF_BF16, MRF_FP8E4M3 = 0, 1, 2
MRF_MODE_BRUTE, MRF_MODE_ZOOM = 0, 1
ZOOM_MAX_LEVELS = 16

_ERRNAMES = {MRF_E_INVALID: "MRF_E_INVALID", MRF_E_NOMEM: "MRF_E_NOMEM", MRF_E_BUDGET: "MRF_E_BUDGET",
             MRF_E_TIMEOUT: "MRF_E_TIMEOUT", MRF_E_CUDA: "MRF_E_CUDA", MRF_E_NOTFOUND: "MRF_E_NOTFOUND",
             MRF_E_UNSUPPORTED: "MRF_E_UNSUPPORTED"}


class MrfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


# ----------------------------------------------------------------------------- structs

class SequenceDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("flip_rad", C.POINTER(C.c_double)), ("rf_phase_rad", C.POINTER(C.c_double)),
                ("tr_ms", C.POINTER(C.c_double)), ("te_ms", C.POINTER(C.c_double)),
                ("inversion", C.c_int32), ("inv_delay_ms", C.c_double), ("pulse_ms", C.POINTER(C.c_double))]


class GridDesc(C.Structure):
    _fields_ = [("t1_min", C.c_double), ("t1_step", C.c_double), ("n_t1", C.c_int32),
                ("t2_min", C.c_double), ("t2_step", C.c_double), ("n_t2", C.c_int32),
                ("df_min", C.c_double), ("df_step", C.c_double), ("n_df", C.c_int32),
                ("require_t2_lt_t1", C.c_int32)]


class DictInfo(C.Structure):
    _fields_ = [("entries", C.c_int64), ("n", C.c_int32), ("ld", C.c_int32), ("dtype", C.c_int32),
                ("hi_dev", C.c_void_p), ("lo_dev", C.c_void_p), ("norm_dev", C.c_void_p),
                ("scale_dev", C.c_void_p), ("bytes", C.c_size_t), ("smooth_width", C.c_int32),
                ("smooth_sigma", C.c_double)]


class MatchOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("top_k", C.c_int32), ("rescore", C.c_int32)]


class ZoomOpts(C.Structure):
    _fields_ = [("omega_hz", C.c_double), ("t1_init_ms", C.c_double), ("t2_init_ms", C.c_double),
                ("s1a_step_frac", C.c_double), ("s1b_half_frac", C.c_double), ("s1b_step_frac", C.c_double),
                ("s3_half_frac", C.c_double), ("n_s2", C.c_int32),
                ("s2_t1_ms", C.c_double * ZOOM_MAX_LEVELS), ("s2_t2_ms", C.c_double * ZOOM_MAX_LEVELS),
                ("n_s4", C.c_int32), ("s4_param", C.c_int32 * ZOOM_MAX_LEVELS),
                ("s4_ms", C.c_double * ZOOM_MAX_LEVELS), ("prior_chain", C.c_int32), ("prior_start", C.c_int32),
                ("prior_t1_ms", C.c_double), ("prior_t2_ms", C.c_double), ("prior_df_hz", C.c_double)]


class Request(C.Structure):
    _fields_ = [("mode", C.c_int32), ("dict", C.c_void_p), ("match", MatchOpts), ("seq", C.c_void_p),
                ("grid", C.POINTER(GridDesc)), ("zoom", C.POINTER(ZoomOpts)), ("fp_host", C.c_void_p),
                ("V", C.c_int64)]


class ServeConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("max_batch_voxels", C.c_int32), ("request_bytes_budget", C.c_size_t)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("rejected", C.c_uint64), ("cancelled", C.c_uint64), ("launches", C.c_uint64),
                ("queued_now", C.c_uint64), ("running_now", C.c_uint64),
                ("request_bytes_in_use", C.c_size_t), ("request_bytes_peak", C.c_size_t)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("dictgen_launches", C.c_uint64), ("matcher_launches", C.c_uint64),
                ("zoom_launches", C.c_uint64), ("dictgen_ms", C.c_double), ("matcher_ms", C.c_double),
                ("zoom_ms", C.c_double), ("dictgen_timed", C.c_uint64), ("matcher_timed", C.c_uint64),
                ("zoom_timed", C.c_uint64), ("zoomline_launches", C.c_uint64), ("zoomline_ms", C.c_double),
                ("zoomline_timed", C.c_uint64), ("zoomline_pairs", C.c_uint64), ("zoomline_entries", C.c_uint64),
                ("zoom_rounds", C.c_uint64), ("zoom_candidates", C.c_uint64), ("zoom_max_voxel_rounds", C.c_uint64)]


# one mrf_result (56 bytes, 8-byte aligned)
RESULT_DTYPE = np.dtype([("index", "<i8"), ("i_t1", "<i4"), ("i_t2", "<i4"), ("i_df", "<i4"),
                         ("t1_ms", "<f4"), ("t2_ms", "<f4"), ("df_hz", "<f4"), ("cc", "<f4"), ("m0", "<f4"),
                         ("phase", "<f4"), ("entries_evaluated", "<i4"), ("min_margin", "<f4")], align=True)
assert RESULT_DTYPE.itemsize == 56

# ----------------------------------------------------------------------------- library

_lib = None
EXPORTS = [
    "mrf_last_error", "mrf_version", "mrf_ctx_create", "mrf_ctx_destroy", "mrf_ctx_memory", "mrf_stream_sync",
    "mrf_sequence_load", "mrf_sequence_free", "mrf_grid_count", "mrf_grid_unravel", "mrf_simulate",
    "mrf_dict_generate", "mrf_dict_free", "mrf_dict_query", "mrf_match_bruteforce", "mrf_match_bruteforce_grid",
    "mrf_match_topk",
    "mrf_zoom_opts_default", "mrf_zoom_search", "mrf_serve_start", "mrf_serve_submit", "mrf_serve_poll",
    "mrf_serve_cancel", "mrf_serve_get_stats", "mrf_serve_stop", "mrf_profile_enable", "mrf_profile_read",
    "mrf_zoom_search_static", "mrf_zoom_search_dict", "mrf_refine", "mrf_smooth", "mrf_dict_smooth",
    "mrf_dict_free_async", "mrf_sequence_free_async", "mrf_fp32_fma_rate", "mrf_mma_rate", "mrf_match_bruteforce_fused",
]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libmrf_gb300.so missing at {path}: the MRF library has no CPU fallback")
        L = C.CDLL(path)
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        L.mrf_last_error.restype = C.c_char_p
        L.mrf_version.restype = C.c_char_p
        L.mrf_ctx_create.argtypes = [C.c_int, sz, C.POINTER(vp)]
        L.mrf_ctx_destroy.argtypes = [vp]
        L.mrf_ctx_destroy.restype = None
        L.mrf_ctx_memory.argtypes = [vp, C.POINTER(sz), C.POINTER(sz)]
        L.mrf_stream_sync.argtypes = [vp, vp]
        L.mrf_sequence_load.argtypes = [vp, C.POINTER(SequenceDesc), C.POINTER(vp)]
        L.mrf_sequence_free.argtypes = [vp, vp]
        L.mrf_grid_count.argtypes = [C.POINTER(GridDesc)]
        L.mrf_grid_count.restype = i64
        L.mrf_grid_unravel.argtypes = [C.POINTER(GridDesc), i64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.mrf_simulate.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
        L.mrf_dict_generate.argtypes = [vp, vp, C.POINTER(GridDesc), C.c_int, vp, C.POINTER(vp)]
        L.mrf_dict_free.argtypes = [vp, vp]
        L.mrf_dict_query.argtypes = [vp, C.POINTER(DictInfo)]
        L.mrf_match_bruteforce.argtypes = [vp, vp, vp, i64, C.POINTER(MatchOpts), vp, vp]
        L.mrf_match_topk.argtypes = [vp, vp, vp, i64, i32, i32, vp, vp, vp]
        L.mrf_match_bruteforce_grid.argtypes = [vp, vp, C.POINTER(GridDesc), C.POINTER(MatchOpts), i64, vp, i64, vp,
                                                vp]
        L.mrf_match_bruteforce_fused.argtypes = [vp, vp, C.POINTER(GridDesc), C.POINTER(MatchOpts), vp, i64, vp, vp]
        L.mrf_zoom_opts_default.argtypes = [C.POINTER(ZoomOpts)]
        L.mrf_zoom_opts_default.restype = None
        L.mrf_zoom_search.argtypes = [vp, vp, C.POINTER(GridDesc), C.POINTER(ZoomOpts), vp, i64, vp, vp]
        L.mrf_refine.argtypes = [vp, vp, C.POINTER(GridDesc), vp, i64, i32, vp, vp]
        L.mrf_smooth.argtypes = [vp, vp, vp, i64, i32, i32, C.c_double, vp]
        L.mrf_dict_free_async.argtypes = [vp, vp, vp]
        L.mrf_sequence_free_async.argtypes = [vp, vp, vp]
        L.mrf_dict_smooth.argtypes = [vp, vp, i32, C.c_double, vp]
        L.mrf_serve_start.argtypes = [vp, C.POINTER(ServeConfig)]
        L.mrf_serve_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
        L.mrf_serve_poll.argtypes = [vp, C.c_uint64, i32, vp]
        L.mrf_serve_cancel.argtypes = [vp, C.c_uint64]
        L.mrf_serve_get_stats.argtypes = [vp, C.POINTER(ServeStats)]
        L.mrf_serve_stop.argtypes = [vp]
        L.mrf_profile_enable.argtypes = [vp, C.c_int]
        L.mrf_profile_read.argtypes = [vp, C.POINTER(Profile), C.c_int]
        L.mrf_fp32_fma_rate.argtypes = [vp, C.POINTER(C.c_double)]
        L.mrf_mma_rate.argtypes = [vp, C.c_int32, C.POINTER(C.c_double)]
        L.mrf_zoom_search_static.argtypes = [vp, vp, C.POINTER(GridDesc), C.POINTER(ZoomOpts), vp, i64, vp, vp]
        L.mrf_zoom_search_dict.argtypes = [vp, vp, C.POINTER(ZoomOpts), vp, i64, vp, vp]
        _lib = L
    return _lib


def last_error() -> str:
    return lib().mrf_last_error().decode()


def check(rc: int, what: str = "") -> int:
    if rc < 0:
        raise MrfError(rc, f"{what}: {last_error()}" if what else last_error())
    return rc


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p()


def grid_desc(g) -> GridDesc:
    """GridDesc from any object with the grid fields (e.g. mrf_synth.Grid)."""
    return GridDesc(g.t1_min, g.t1_step, g.n_t1, g.t2_min, g.t2_step, g.n_t2, g.df_min, g.df_step, g.n_df,
                    int(g.require_t2_lt_t1))


# ----------------------------------------------------------------------------- C entry points

def mrf_version() -> str:
    return lib().mrf_version().decode()


def mrf_ctx_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = C.c_void_p()
    check(lib().mrf_ctx_create(device, hbm_budget_bytes, C.byref(h)), "mrf_ctx_create")
    return h


def mrf_ctx_destroy(ctx) -> None:
    lib().mrf_ctx_destroy(ctx)


def mrf_ctx_memory(ctx):
    u, b = C.c_size_t(), C.c_size_t()
    check(lib().mrf_ctx_memory(ctx, C.byref(u), C.byref(b)), "mrf_ctx_memory")
    return u.value, b.value


def mrf_stream_sync(ctx, stream=None) -> int:
    return check(lib().mrf_stream_sync(ctx, _stream_ptr(stream)), "mrf_stream_sync")


class _SeqArrays:
    def __init__(self, seq):
        self.flip = np.ascontiguousarray(seq.flip_rad, np.float64)
        ph = getattr(seq, "rf_phase_rad", None)
        self.phase = None if ph is None else np.ascontiguousarray(ph, np.float64)
        self.tr = np.ascontiguousarray(seq.tr_ms, np.float64)
        self.te = np.ascontiguousarray(seq.te_ms, np.float64)
        pu = getattr(seq, "pulse_ms", None)
        self.pulse = None if pu is None else np.ascontiguousarray(pu, np.float64)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else C.POINTER(C.c_double)()
        self.desc = SequenceDesc(int(self.flip.shape[0]), dp(self.flip), dp(self.phase), dp(self.tr), dp(self.te),
                                 int(seq.inversion), float(seq.inv_delay_ms), dp(self.pulse))


def mrf_sequence_load(ctx, seq):
    """seq: object with flip_rad, rf_phase_rad (or None), tr_ms, te_ms, inversion, inv_delay_ms
    and optionally pulse_ms (RF pulse durations, None for hard pulses)."""
    arr = _SeqArrays(seq)
    h = C.c_void_p()
    check(lib().mrf_sequence_load(ctx, C.byref(arr.desc), C.byref(h)), "mrf_sequence_load")
    return h


def mrf_sequence_free(ctx, seq) -> None:
    check(lib().mrf_sequence_free(ctx, seq), "mrf_sequence_free")


def mrf_grid_count(grid) -> int:
    return check(int(lib().mrf_grid_count(C.byref(grid_desc(grid)))), "mrf_grid_count")


def mrf_grid_unravel(grid, index: int):
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    check(lib().mrf_grid_unravel(C.byref(grid_desc(grid)), int(index), C.byref(a), C.byref(b), C.byref(c)),
          "mrf_grid_unravel")
    return a.value, b.value, c.value


def mrf_simulate(ctx, seq, t1, t2, df, out, stream=None) -> None:
    """t1/t2/df: float32 CUDA tensors (count,); out: complex64 CUDA tensor (count, n)."""
    check(lib().mrf_simulate(ctx, seq, t1.numel(), _ptr(t1), _ptr(t2), _ptr(df), _ptr(out), _stream_ptr(stream)),
          "mrf_simulate")


def mrf_dict_generate(ctx, seq, grid, dtype: int, stream=None):
    h = C.c_void_p()
    g = grid_desc(grid)
    check(lib().mrf_dict_generate(ctx, seq, C.byref(g), dtype, _stream_ptr(stream), C.byref(h)), "mrf_dict_generate")
    return h


def mrf_dict_free(ctx, d) -> None:
    check(lib().mrf_dict_free(ctx, d), "mrf_dict_free")


def mrf_smooth(ctx, fp_in, fp_out, width: int, sigma: float = 1.0, stream=None) -> None:
    """Temporal smoothing of V x n complex64 CUDA tensors (distinct in and out)."""
    V, n = fp_in.shape
    check(lib().mrf_smooth(ctx, _ptr(fp_in), _ptr(fp_out), V, n, int(width), float(sigma), _stream_ptr(stream)),
          "mrf_smooth")


def mrf_dict_smooth(ctx, d, width: int, sigma: float = 1.0, stream=None) -> None:
    """Smooth a generated MRF_F32 or BF16 dictionary in place."""
    check(lib().mrf_dict_smooth(ctx, d, int(width), float(sigma), _stream_ptr(stream)), "mrf_dict_smooth")


def mrf_dict_free_async(ctx, d, stream=None) -> None:
    """Release a dictionary in the order of `stream` (its uses must be enqueued there)."""
    check(lib().mrf_dict_free_async(ctx, d, _stream_ptr(stream)), "mrf_dict_free_async")


def mrf_sequence_free_async(ctx, seq, stream=None) -> None:
    """Release a sequence in the order of `stream` (its uses must be enqueued there)."""
    check(lib().mrf_sequence_free_async(ctx, seq, _stream_ptr(stream)), "mrf_sequence_free_async")


def mrf_dict_query(d) -> DictInfo:
    info = DictInfo()
    check(lib().mrf_dict_query(d, C.byref(info)), "mrf_dict_query")
    return info


def mrf_match_bruteforce(ctx, d, fp, opts: MatchOpts, out, stream=None) -> None:
    """fp: complex64 CUDA tensor (V, n); out: uint8 CUDA tensor of V * 56 bytes."""
    V = fp.shape[0] if fp is not None else 0
    check(lib().mrf_match_bruteforce(ctx, d, _ptr(fp), V, C.byref(opts), _ptr(out), _stream_ptr(stream)),
          "mrf_match_bruteforce")


def mrf_match_bruteforce_grid(ctx, seq, grid, fp, opts: MatchOpts, out, chunk_entries: int = 0, stream=None) -> None:
    """Brute force over a grid without a resident dictionary (ranges of T1 rows
    generated, matched and released in turn). fp: complex64 CUDA tensor (V, n)."""
    g = grid_desc(grid)
    V = fp.shape[0] if fp is not None else 0
    check(lib().mrf_match_bruteforce_grid(ctx, seq, C.byref(g), C.byref(opts), int(chunk_entries), _ptr(fp), V,
                                          _ptr(out), _stream_ptr(stream)), "mrf_match_bruteforce_grid")


def mrf_match_bruteforce_fused(ctx, seq, grid, fp, opts: MatchOpts, out, stream=None) -> None:
    """Brute force with every dictionary tile generated inside the matcher (no
    dictionary stored). fp: complex64 CUDA tensor (V, n)."""
    g = grid_desc(grid)
    V = fp.shape[0] if fp is not None else 0
    check(lib().mrf_match_bruteforce_fused(ctx, seq, C.byref(g), C.byref(opts), _ptr(fp), V, _ptr(out),
                                           _stream_ptr(stream)), "mrf_match_bruteforce_fused")


def mrf_match_topk(ctx, d, fp, precision: int, top_k: int, idx, cc2, stream=None) -> None:
    check(lib().mrf_match_topk(ctx, d, _ptr(fp), fp.shape[0], precision, top_k, _ptr(idx), _ptr(cc2),
                               _stream_ptr(stream)), "mrf_match_topk")


def mrf_zoom_opts_default() -> ZoomOpts:
    o = ZoomOpts()
    lib().mrf_zoom_opts_default(C.byref(o))
    return o


def mrf_zoom_search(ctx, seq, grid, opts, fp, out, stream=None) -> None:
    g = grid_desc(grid)
    check(lib().mrf_zoom_search(ctx, seq, C.byref(g), C.byref(opts) if opts is not None else None, _ptr(fp),
                                fp.shape[0], _ptr(out), _stream_ptr(stream)), "mrf_zoom_search")


def mrf_refine(ctx, seq, grid, fp, res, max_moves=1 << 20, stream=None) -> None:
    """Windowed refinement of the results in res (in place) from their grid points."""
    g = grid_desc(grid)
    check(lib().mrf_refine(ctx, seq, C.byref(g), _ptr(fp), fp.shape[0], int(max_moves), _ptr(res),
                           _stream_ptr(stream)), "mrf_refine")


def mrf_zoom_search_dict(ctx, d, opts, fp, out, stream=None) -> None:
    """MRF-ZOOM with every candidate's CC read from the resident dictionary d."""
    check(lib().mrf_zoom_search_dict(ctx, d, C.byref(opts) if opts is not None else None, _ptr(fp), fp.shape[0],
                                     _ptr(out), _stream_ptr(stream)), "mrf_zoom_search_dict")


def mrf_zoom_search_static(ctx, seq, grid, opts, fp, out, stream=None) -> None:
    """mrf_zoom_search with its scratch in the library's fixed device array (no allocation)."""
    g = grid_desc(grid)
    check(lib().mrf_zoom_search_static(ctx, seq, C.byref(g), C.byref(opts) if opts is not None else None, _ptr(fp),
                                       fp.shape[0], _ptr(out), _stream_ptr(stream)), "mrf_zoom_search_static")


def mrf_serve_start(ctx, max_inflight=2, max_batch_voxels=16384, request_bytes_budget=0) -> None:
    cfg = ServeConfig(max_inflight, max_batch_voxels, request_bytes_budget)
    check(lib().mrf_serve_start(ctx, C.byref(cfg)), "mrf_serve_start")


def mrf_serve_submit(ctx, req: Request) -> int:
    t = C.c_uint64()
    check(lib().mrf_serve_submit(ctx, C.byref(req), C.byref(t)), "mrf_serve_submit")
    return t.value


def mrf_serve_poll(ctx, ticket: int, timeout_ms: int, out_host: np.ndarray) -> int:
    """out_host: RESULT_DTYPE array of V elements. Returns MRF_OK or MRF_PENDING; raises on errors."""
    return check(lib().mrf_serve_poll(ctx, ticket, timeout_ms, out_host.ctypes.data_as(C.c_void_p)),
                 "mrf_serve_poll")


def mrf_serve_poll_rc(ctx, ticket: int, timeout_ms: int, out_host: np.ndarray) -> int:
    """Like mrf_serve_poll but returns the raw status code."""
    return int(lib().mrf_serve_poll(ctx, ticket, timeout_ms, out_host.ctypes.data_as(C.c_void_p)))


def mrf_serve_cancel(ctx, ticket: int) -> int:
    return int(lib().mrf_serve_cancel(ctx, ticket))


def mrf_serve_get_stats(ctx) -> ServeStats:
    s = ServeStats()
    check(lib().mrf_serve_get_stats(ctx, C.byref(s)), "mrf_serve_get_stats")
    return s


def mrf_serve_stop(ctx) -> None:
    check(lib().mrf_serve_stop(ctx), "mrf_serve_stop")


def mrf_profile_enable(ctx, on: bool = True) -> None:
    check(lib().mrf_profile_enable(ctx, 1 if on else 0), "mrf_profile_enable")


def mrf_fp32_fma_rate(ctx) -> float:
    """Measured FP32 FMA rate of the device, TFLOP/s."""
    t = C.c_double()
    check(lib().mrf_fp32_fma_rate(ctx, C.byref(t)), "mrf_fp32_fma_rate")
    return float(t.value)


def mrf_mma_rate(ctx, precision) -> float:
    """Measured dense tensor-core rate of the matcher's MMA shape (MRF_BF16 or MRF_FP8E4M3), TFLOP/s."""
    t = C.c_double()
    check(lib().mrf_mma_rate(ctx, int(precision), C.byref(t)), "mrf_mma_rate")
    return float(t.value)


def mrf_profile_read(ctx, reset: bool = False) -> Profile:
    p = Profile()
    check(lib().mrf_profile_read(ctx, C.byref(p), 1 if reset else 0), "mrf_profile_read")
    return p


# ----------------------------------------------------------------------------- helpers

def results_to_numpy(out) -> np.ndarray:
    """Copy a device result buffer (uint8 tensor) into a RESULT_DTYPE array."""
    raw = out.detach().cpu().numpy().view(np.uint8)
    return raw.view(RESULT_DTYPE)


def empty_results(V: int, device="cuda"):
    import torch
    return torch.empty(max(V, 1) * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)


def match_opts(precision: int = MRF_F32, top_k: int = 4, rescore: int = 1) -> MatchOpts:
    return MatchOpts(precision, top_k, rescore)


def zoom_opts(**kw) -> ZoomOpts:
    """Experiment 2 defaults with keyword overrides (s2=[(t1, t2)...], s4=[(param, ms)...])."""
    o = mrf_zoom_opts_default()
    for k in ("omega_hz", "t1_init_ms", "t2_init_ms", "s1a_step_frac", "s1b_half_frac", "s1b_step_frac",
              "s3_half_frac"):
        if k in kw:
            setattr(o, k, float(kw[k]))
    if "s2" in kw:
        o.n_s2 = len(kw["s2"])
        for i, (a, b) in enumerate(kw["s2"]):
            o.s2_t1_ms[i], o.s2_t2_ms[i] = a, b
    if "s4" in kw:
        o.n_s4 = len(kw["s4"])
        for i, (p, h) in enumerate(kw["s4"]):
            o.s4_param[i], o.s4_ms[i] = p, h
    if "prior" in kw:   # (chain length, (T1, T2, df) half-widths[, start from the prior 1/0])
        chain, half = kw["prior"][:2]
        o.prior_chain = int(chain)
        o.prior_start = int(kw["prior"][2]) if len(kw["prior"]) > 2 else 1
        o.prior_t1_ms, o.prior_t2_ms, o.prior_df_hz = (float(v) for v in half)
    return o
