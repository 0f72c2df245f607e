"""RF pulses of finite duration on the GPU (Appendix: the off-resonant form
R_z(phi) R_y(beta) R_x(alpha') R_y(-beta) R_z(-phi), which depends on each
candidate's df) against the FP64 oracle, through every simulator: the
fingerprint kernel, dictionary generation (every stored precision), brute
force with its re-score, MRF-ZOOM (the split search with step 3 batched by
line, and the single-kernel search) and the windowed refinement.

Bars as for hard pulses: fingerprints within 1e-5 relative L2; CC within
1e-5; indices identical except where the oracle's top-two gap (brute force)
or smallest decision margin (ZOOM, refinement) is below 1e-6."""
import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import F32_STORE_TOL, offgrid_voxels, rel_l2
from test_gpu_bloch import _dict_rows, _gpu_simulate
from test_gpu_match import _compare as _compare_brute
from test_gpu_match import _run as _run_brute
from test_gpu_refine import _compare as _compare_refine
from test_gpu_refine import _gpu_refine, _starts_from_truth
from test_gpu_zoom import _compare as _compare_zoom
from test_gpu_zoom import _gpu_zoom

pytestmark = pytest.mark.gpu


def _seqs():
    """The paper-shaped train (0/90/180 degree phases) with 1 ms pulses, the
    alternating-sign train with 2 ms pulses and TE = 0.3 TR, and per-pulse
    durations of 0-3 ms, some zero (hard)."""
    p = S.sequence_paper(21, 300, 1.0)
    b = S.sequence(22, 300)
    alt = S.with_pulses(S.Sequence(b.flip_rad, b.rf_phase_rad, b.tr_ms, b.tr_ms * 0.3, 1, 20.0), 2.0)
    rng = np.random.default_rng(23)
    tau = np.where(rng.uniform(size=300) < 0.2, 0.0, rng.uniform(0.2, 3.0, 300))
    mixed = S.with_pulses(S.sequence(24, 300), tau)
    return {"paper_1ms": p, "alternating_2ms_asym": alt, "alternating_mixed": mixed}


SEQS = _seqs()


@pytest.mark.parametrize("kind", list(SEQS))
def test_finite_pulse_fingerprints(M, ctx, oracle_lib, kind):
    """Fingerprints at random parameters (df up to +-60 Hz, beyond the
    workloads' +-40 Hz), the oracle evaluated at the FP32 values the GPU
    kernel receives."""
    seq = SEQS[kind]
    p = S.phantom_offgrid(61, 384, t1_range=(100.0, 4000.0), t2_range=(10.0, 400.0), df_range=(-60.0, 60.0))
    p = {k: np.asarray(p[k], np.float32).astype(np.float64) for k in ("t1", "t2", "df")}
    gpu = _gpu_simulate(M, ctx, seq, p["t1"], p["t2"], p["df"])
    ref = oracle_lib.simulate(seq, p["t1"], p["t2"], p["df"])
    err = rel_l2(gpu, ref)
    assert err.max() < 1e-5, f"{kind}: max rel L2 {err.max():.3g}"
    # the pulses matter: against the same train with hard pulses the fingerprints differ
    hard = oracle_lib.simulate(S.Sequence(seq.flip_rad, seq.rf_phase_rad, seq.tr_ms, seq.te_ms, seq.inversion,
                                          seq.inv_delay_ms), p["t1"], p["t2"], p["df"])
    assert np.median(rel_l2(hard, ref)) > 1e-3


def test_zero_pulse_durations_are_the_hard_pulse_bit_for_bit(M, ctx, oracle_lib):
    seq = S.sequence_paper(25, 200)
    p = S.phantom_offgrid(62, 96)
    a = _gpu_simulate(M, ctx, seq, p["t1"], p["t2"], p["df"])
    b = _gpu_simulate(M, ctx, S.with_pulses(seq, 0.0), p["t1"], p["t2"], p["df"])
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("dtype,tol", [(0, F32_STORE_TOL), (1, 3e-3), (2, 7e-2)])
def test_finite_pulse_dictionary(M, ctx, oracle_lib, dtype, tol):
    """Rows, norms and padding of a dictionary on a grid with a df axis
    (each entry's RF rotation from its own df)."""
    seq = SEQS["paper_1ms"]
    g = S.Grid(100.0, 150.0, 20, 20.0, 30.0, 10, -60.0, 15.0, 9)
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, dtype)
    torch.cuda.synchronize()
    try:
        rows, pad, norm, info = _dict_rows(M, d, dtype)
        a, b, c = oracle_lib.grid_params(g)
        t1, t2, df = S.grid_values(g)
        ref = oracle_lib.simulate(seq, t1[a], t2[b], df[c])
        nr = np.linalg.norm(ref, axis=1)
        err = rel_l2(rows, ref / nr[:, None])
        assert err.max() < tol, f"dtype {dtype}: max rel L2 {err.max():.3g}"
        np.testing.assert_allclose(norm, nr, rtol=1e-5)
        assert np.all(pad == 0)
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_finite_pulse_bruteforce(M, ctx, oracle_lib):
    """FP32-equivalent brute force with its FP32 re-simulation / FP64
    re-score over several 256-entry tiles (ragged tail) against the oracle."""
    seq = SEQS["alternating_2ms_asym"]
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -30.0, 6.0, 11)
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
    try:
        ph, x = offgrid_voxels(oracle_lib, seq, 96, 25.0, 63, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                               df_range=(-28.0, 28.0))
        ref = oracle_lib.bruteforce(seq, g, x, k=2)
        res = _run_brute(M, ctx, d, x, M.MRF_F32, 4, 1)
        diff, exc = _compare_brute(res, ref, "finite pulse brute force")
        print(f"finite pulse brute force: differ={diff} excused={exc}")
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


@pytest.mark.parametrize("grid", ["fp32_brute", "precision"])
def test_finite_pulse_zoom(M, ctx, oracle_lib, grid):
    """MRF-ZOOM with finite pulses: on the 614,508-entry grid (every step in
    the packed kernel) and on the 12M-entry grid, whose 1 Hz df step makes the
    step-3 window long enough for the batched line kernel; against the oracle,
    and the single-kernel search bit for bit."""
    import ctypes as C
    seq = SEQS["paper_1ms"]
    g = S.GRIDS[grid]
    ph, x = offgrid_voxels(oracle_lib, seq, 48, 20.0, 64)
    res = _gpu_zoom(M, ctx, seq, g, x)
    ref = oracle_lib.zoom(seq, g, x)
    diff, exc = _compare_zoom(oracle_lib, g, res, ref, f"finite pulse zoom {grid}")
    print(f"finite pulse zoom {grid}: differ={diff} excused={exc}")
    h = M.mrf_sequence_load(ctx, seq)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        gd, zo = M.grid_desc(g), M.zoom_opts()
        M.check(M.lib().mrf_zoom_search_static(ctx, h, C.byref(gd), C.byref(zo), C.c_void_p(fp.data_ptr()),
                                               x.shape[0], C.c_void_p(out.data_ptr()), None), "zoom static")
        M.mrf_stream_sync(ctx)
        one = M.results_to_numpy(out)[: x.shape[0]]
        for f in res.dtype.names:
            assert np.array_equal(np.ascontiguousarray(one[f]).view(np.uint8),
                                  np.ascontiguousarray(res[f]).view(np.uint8)), f
    finally:
        M.mrf_sequence_free(ctx, h)


def test_finite_pulse_refine(M, ctx, oracle_lib):
    seq = SEQS["alternating_mixed"]
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 64, 20.0, 65)
    abc = _starts_from_truth(g, ph, 66)
    res = _gpu_refine(M, ctx, seq, g, x, abc)
    ref = oracle_lib.refine(seq, g, x, abc)
    _compare_refine(oracle_lib, g, res, ref, "finite pulse refine")
