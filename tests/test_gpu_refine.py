"""GPU windowed refinement (mrf_refine) against the FP64 oracle's refinement
(Results, Experiment 2: brute force in a window around an answer, repeated as
a hill climb over the 26-point grid neighbourhood).

Bar: final grid point identical except where the oracle's smallest decision
margin is below 1e-6 (counted); CC within 1e-5; evaluation counts identical
where no margin is below 1e-5. Start points come from the phantoms' true
parameters (nearest grid point plus seeded offsets), from the FP8 top-k
re-score and from ZOOM."""
import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import offgrid_voxels

pytestmark = pytest.mark.gpu

MARGIN_EXCUSE = 1e-6


def _starts_from_truth(g, ph, seed, spread=3):
    t1, t2, df = S.grid_values(g)
    a = np.clip(np.rint((ph["t1"] - g.t1_min) / g.t1_step).astype(int), 0, g.n_t1 - 1)
    b = np.clip(np.rint((ph["t2"] - g.t2_min) / g.t2_step).astype(int), 0, g.n_t2 - 1)
    c = np.clip(np.rint((ph["df"] - g.df_min) / g.df_step).astype(int), 0, g.n_df - 1)
    rng = np.random.default_rng(seed)
    abc = np.stack([a, b, c], 1) + rng.integers(-spread, spread + 1, (len(a), 3))
    abc = np.clip(abc, 0, [g.n_t1 - 1, g.n_t2 - 1, g.n_df - 1])
    if g.require_t2_lt_t1:
        abc[:, 1] = np.minimum(abc[:, 1], np.searchsorted(t2, t1[abc[:, 0]]) - 1)
    return abc


def _gpu_refine(M, ctx, seq, g, x, abc, prior=None):
    h = M.mrf_sequence_load(ctx, seq)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        V = x.shape[0]
        res = np.zeros(V, M.RESULT_DTYPE) if prior is None else prior.copy()
        if prior is None:
            res["index"] = 1
            res["entries_evaluated"] = 0
            res["min_margin"] = -1.0
        res["i_t1"], res["i_t2"], res["i_df"] = abc[:, 0], abc[:, 1], abc[:, 2]
        out = torch.from_numpy(res.view(np.uint8)).cuda()
        M.mrf_refine(ctx, h, g, fp, out)
        M.mrf_stream_sync(ctx)
        return M.results_to_numpy(out)[:V]
    finally:
        M.mrf_sequence_free(ctx, h)


def _compare(orc, g, res, ref, label, base_evaluated=0):
    abc = np.stack([res["i_t1"], res["i_t2"], res["i_df"]], 1)
    same = (abc == ref["abc"]).all(1)
    excused = ref["min_margin"] < MARGIN_EXCUSE
    bad = ~same & ~excused
    assert not bad.any(), (f"{label}: {int(bad.sum())} voxels differ with margin >= {MARGIN_EXCUSE}: "
                           f"gpu {abc[bad][:4].tolist()} oracle {ref['abc'][bad][:4].tolist()}")
    assert np.abs(res["cc"][same] - ref["cc"][same]).max() < 1e-5
    idx = np.array([orc.grid_index(g, *p) for p in ref["abc"]])
    assert (res["index"][same] == idx[same]).all()
    np.testing.assert_allclose(res["m0"][same], ref["m0"][same], rtol=1e-4)
    firm = same & (ref["min_margin"] >= 1e-5)
    assert (res["entries_evaluated"][firm] == base_evaluated + ref["evaluated"][firm]).all()
    return int((~same).sum()), int(excused.sum())


def test_refine_from_perturbed_truth_3d(M, ctx, oracle_lib):
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 96, 20.0, 121)
    abc = _starts_from_truth(g, ph, 5)
    res = _gpu_refine(M, ctx, seq, g, x, abc)
    ref = oracle_lib.refine(seq, g, x, abc)
    diff, exc = _compare(oracle_lib, g, res, ref, "perturbed 3d")
    print(f"refine 3d: differ={diff} excused={exc} mean evaluated={ref['evaluated'].mean():.1f}")


def test_refine_on_single_df_grid_and_general_rf(M, ctx, oracle_lib):
    """n_df = 1 (the df neighbours are off the grid) and a sequence with
    general RF phases and TE != TR / 2."""
    import math
    base = S.sequence(5, 160)
    rng = np.random.default_rng(23)
    seq = S.Sequence(base.flip_rad, rng.uniform(0, 2 * math.pi, 160), base.tr_ms, base.tr_ms * 0.35, 1, 20.0)
    g = S.Grid(200.0, 25.0, 50, 20.0, 8.0, 30, 0.0, 1.0, 1)
    ph, x = offgrid_voxels(oracle_lib, seq, 40, 30.0, 66, t1_range=(300.0, 1300.0), t2_range=(30.0, 220.0),
                           df_range=(0.0, 0.0))
    abc = _starts_from_truth(g, ph, 8, spread=4)
    res = _gpu_refine(M, ctx, seq, g, x, abc)
    ref = oracle_lib.refine(seq, g, x, abc)
    _compare(oracle_lib, g, res, ref, "single df")


def test_refine_after_fp8_rescore_improves_agreement(M, ctx, oracle_lib):
    """Low-precision brute force + re-score, then refinement from its answer:
    parity with the oracle's refinement from the same points, and agreement
    with the exhaustive FP64 optimum no worse than before."""
    seq = S.sequence(2, 200)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    ph, x = offgrid_voxels(oracle_lib, seq, 120, 25.0, 7, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-11.0, 11.0))
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, M.MRF_FP8E4M3)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        M.mrf_match_bruteforce(ctx, d, fp, M.match_opts(M.MRF_FP8E4M3, 8, 1), out)
        M.mrf_stream_sync(ctx)
        first = M.results_to_numpy(out)[: x.shape[0]].copy()
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)
    abc = np.stack([first["i_t1"], first["i_t2"], first["i_df"]], 1)
    res = _gpu_refine(M, ctx, seq, g, x, abc, prior=first)
    ref = oracle_lib.refine(seq, g, x, abc)
    D = oracle_lib.grid_count(g)
    _compare(oracle_lib, g, res, ref, "after fp8", base_evaluated=D)
    bf = oracle_lib.bruteforce(seq, g, x, k=1)
    before = np.mean(first["index"] == bf["idx"][:, 0])
    after = np.mean(res["index"] == bf["idx"][:, 0])
    print(f"fp8 top-8 + re-score: agreement {before:.3f} -> after refinement {after:.3f}")
    assert after >= before


def test_refine_after_zoom(M, ctx, oracle_lib):
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 64, 20.0, 141)
    h = M.mrf_sequence_load(ctx, seq)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        M.mrf_zoom_search(ctx, h, g, M.zoom_opts(), fp, out)
        M.mrf_stream_sync(ctx)
        z = M.results_to_numpy(out)[: x.shape[0]].copy()
    finally:
        M.mrf_sequence_free(ctx, h)
    abc = np.stack([z["i_t1"], z["i_t2"], z["i_df"]], 1)
    res = _gpu_refine(M, ctx, seq, g, x, abc, prior=z)
    ref = oracle_lib.refine(seq, g, x, abc)
    # the ZOOM margins carry over: compare the refinement's own decisions
    prior_free = z.copy()
    prior_free["min_margin"] = -1.0
    res2 = _gpu_refine(M, ctx, seq, g, x, abc, prior=prior_free)
    assert (res2["i_t1"] == res["i_t1"]).all() and (res2["index"] == res["index"]).all()
    abc2 = np.stack([res2["i_t1"], res2["i_t2"], res2["i_df"]], 1)
    same = (abc2 == ref["abc"]).all(1)
    assert (same | (ref["min_margin"] < MARGIN_EXCUSE)).all()
    assert (res["cc"] >= z["cc"] - 1e-5).all()
    print(f"zoom + refinement: moved {int((abc2 != abc).any(1).sum())}/{len(abc)} voxels")


def test_refine_leaves_unmatched_voxels_and_rejects_bad_arguments(M, ctx):
    import ctypes as C
    seq = S.sequence(0, 50)
    g = S.GRIDS["tiny"]
    h = M.mrf_sequence_load(ctx, seq)
    try:
        x = torch.ones((3, 50), dtype=torch.complex64, device="cuda")
        res = np.zeros(3, M.RESULT_DTYPE)
        res["index"] = [-1, 5, -1]
        res["i_t1"], res["i_t2"], res["i_df"] = [0, 40, 0], [0, 0, 0], [0, 0, 0]   # voxel 1: T1 index off the grid
        res["cc"] = [0.25, 0.5, 0.75]
        out = torch.from_numpy(res.view(np.uint8)).cuda()
        M.mrf_refine(ctx, h, g, x, out)
        M.mrf_stream_sync(ctx)
        back = M.results_to_numpy(out)[:3]
        np.testing.assert_array_equal(back, res)
        gd = M.grid_desc(g)
        assert M.lib().mrf_refine(ctx, h, C.byref(gd), C.c_void_p(x.data_ptr()), 3, 0, C.c_void_p(out.data_ptr()),
                                  None) == M.MRF_E_INVALID
        assert M.lib().mrf_refine(ctx, h, C.byref(gd), None, 0, 4, None, None) == M.MRF_OK
    finally:
        M.mrf_sequence_free(ctx, h)
