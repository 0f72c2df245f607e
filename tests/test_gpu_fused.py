"""Brute force with generated dictionary tiles (mrf_match_bruteforce_fused:
the Bloch recurrence run inside the tensor-core matcher, no dictionary
stored) against the FP64 oracle's brute force (Theory: argmax of Eq. 1 over
every grid entry), and against the resident-dictionary search.

Bar as for mrf_match_bruteforce: CC within 1e-5; index identical except
where the oracle's top-two CC gap is below 1e-6."""
import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import offgrid_voxels, ongrid_voxels
from test_gpu_match import _compare

pytestmark = pytest.mark.gpu


def _fused(M, ctx, seq, g, x, precision, top_k, rescore=1):
    h = M.mrf_sequence_load(ctx, seq)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        M.mrf_match_bruteforce_fused(ctx, h, g, fp, M.match_opts(precision, top_k, rescore), out)
        M.mrf_stream_sync(ctx)
        return M.results_to_numpy(out)[: x.shape[0]]
    finally:
        M.mrf_sequence_free(ctx, h)


def _resident(M, ctx, seq, g, x, precision, top_k, rescore=1):
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, precision)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        M.mrf_match_bruteforce(ctx, d, fp, M.match_opts(precision, top_k, rescore), out)
        M.mrf_stream_sync(ctx)
        return M.results_to_numpy(out)[: x.shape[0]]
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_fused_tiny_recovers_on_grid_voxels(M, ctx, oracle_lib):
    """Noise-free on-grid voxels (Experiment 2): found exactly, CC 1, M0 the
    applied scale (one tile, most of it past the 193 entries)."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    ph, x = ongrid_voxels(oracle_lib, seq, g, 64, None, 200)
    res = _fused(M, ctx, seq, g, x, M.MRF_F32, 4)
    a, b, c = oracle_lib.grid_params(g)
    assert (a[res["index"]] == ph["a"]).all() and (b[res["index"]] == ph["b"]).all()
    np.testing.assert_allclose(res["cc"], 1.0, atol=1e-5)
    np.testing.assert_allclose(res["m0"], ph["m0"], rtol=1e-4)
    assert (res["entries_evaluated"] == 193).all()


@pytest.mark.parametrize("n", [200, 37])
def test_fused_ragged_against_oracle(M, ctx, oracle_lib, n):
    """Several 256-entry tiles with a ragged tail, V = 150 (three voxel units
    of 64, the last ragged), N = 200 and N = 37 (a K block cut by the end of
    the sequence): FP32-equivalent, top-4 + re-score."""
    seq = S.sequence(2, n)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    ph, x = offgrid_voxels(oracle_lib, seq, 150, 25.0, 7, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-11.0, 11.0))
    ref = oracle_lib.bruteforce(seq, g, x, k=2)
    res = _fused(M, ctx, seq, g, x, M.MRF_F32, 4)
    diff, exc = _compare(res, ref, f"fused F32 N={n}")
    print(f"fused F32 N={n}: differ={diff} excused={exc}")
    assert (res["entries_evaluated"] == oracle_lib.grid_count(g)).all()


def test_fused_general_rf_and_finite_pulses_against_oracle(M, ctx, oracle_lib):
    """The table-free simulation with the general RF rotation: the paper-
    shaped train (0/90/180 degree phases) with 1 ms pulses."""
    seq = S.sequence_paper(31, 300, 1.0)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -30.0, 6.0, 11)
    ph, x = offgrid_voxels(oracle_lib, seq, 96, 25.0, 8, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-28.0, 28.0))
    ref = oracle_lib.bruteforce(seq, g, x, k=2)
    res = _fused(M, ctx, seq, g, x, M.MRF_F32, 4)
    diff, exc = _compare(res, ref, "fused F32, finite pulses")
    print(f"fused F32 finite pulses: differ={diff} excused={exc}")


def test_fused_bf16_rescore(M, ctx, oracle_lib):
    """BF16 tiles (raw entries, FP32 column scales) with top-32 and the FP64
    re-score: the returned entries' CCs are the oracle's, and nearly every
    voxel agrees with the oracle's brute force."""
    seq = S.sequence(2, 200)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    ph, x = offgrid_voxels(oracle_lib, seq, 150, 25.0, 9, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-11.0, 11.0))
    ref = oracle_lib.bruteforce(seq, g, x, k=2)
    res = _fused(M, ctx, seq, g, x, M.MRF_BF16, 32)
    t1, t2, df = S.grid_values(g)
    a, b, c = oracle_lib.grid_params(g)
    dd = oracle_lib.simulate(seq, t1[a[res["index"]]], t2[b[res["index"]]], df[c[res["index"]]])
    occ = np.abs(np.sum(dd.conj() * x, 1)) / (np.linalg.norm(dd, axis=1) * np.linalg.norm(x, axis=1))
    assert np.abs(res["cc"] - occ).max() < 1e-5
    agree = np.mean(res["index"] == ref["idx"][:, 0])
    print(f"fused BF16 top-32: agreement {agree:.3f}")
    assert agree >= 0.9


def test_fused_equals_resident_at_full_size_sampled(M, ctx, oracle_lib):
    """The 614,508-entry grid (N = 1000), 256 voxels of the 64x64 slice: the
    fused search against the resident FP32-equivalent search (same indices
    wherever the resident search's top-two gap is at least 1e-6, CC within
    1e-5), and 4 voxels against the oracle's exhaustive search."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 256, 20.0, 101)
    fused = _fused(M, ctx, seq, g, x, M.MRF_F32, 4)
    res = _resident(M, ctx, seq, g, x, M.MRF_F32, 4)
    sure = res["min_margin"] >= 1e-6
    assert (fused["index"] == res["index"])[sure].all()
    same = fused["index"] == res["index"]
    assert np.abs(fused["cc"][same] - res["cc"][same]).max() < 1e-5
    pick = np.random.default_rng(3).choice(256, 4, replace=False)
    ref = oracle_lib.bruteforce(seq, g, x[pick], k=2)
    _compare(fused[pick], ref, "fused full size")
    print(f"fused vs resident at full size: same index {same.mean():.4f} ({int(sure.sum())} firm)")


def test_fused_options_checked(M, ctx):
    import ctypes as C
    seq = S.sequence(0, 50)
    h = M.mrf_sequence_load(ctx, seq)
    try:
        g = M.grid_desc(S.GRIDS["tiny"])
        fp = torch.zeros((4, 50), dtype=torch.complex64, device="cuda")
        out = M.empty_results(4)
        L = M.lib()
        for o in (M.match_opts(M.MRF_FP8E4M3, 8, 1), M.match_opts(M.MRF_F32, 3, 1), M.match_opts(M.MRF_F32, 4, 2)):
            rc = L.mrf_match_bruteforce_fused(ctx, h, C.byref(g), C.byref(o), C.c_void_p(fp.data_ptr()), 4,
                                              C.c_void_p(out.data_ptr()), None)
            assert rc == M.MRF_E_INVALID
    finally:
        M.mrf_sequence_free(ctx, h)


@pytest.mark.parametrize("V", [1, 65])
def test_fused_ragged_voxel_counts(M, ctx, oracle_lib, V):
    """One voxel, and one voxel past a 64-voxel unit: the padding rows of the
    voxel operand take no part."""
    seq = S.sequence(2, 200)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    ph, x = offgrid_voxels(oracle_lib, seq, V, 25.0, 10, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-11.0, 11.0))
    ref = oracle_lib.bruteforce(seq, g, x, k=2)
    res = _fused(M, ctx, seq, g, x, M.MRF_F32, 4)
    _compare(res, ref, f"fused V={V}")
