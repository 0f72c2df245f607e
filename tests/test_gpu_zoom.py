"""GPU MRF-ZOOM against the FP64 oracle's ZOOM (Theory: df search, 1D and
2D ZOOM; Methods, Experiment 2 steps 1-5).

Bar: final grid point identical except where the oracle trace's smallest
decision margin is below 1e-6 (counted); CC within 1e-5; where the final
points agree and no margin is close, the number of candidate evaluations is
identical too (same trace length)."""
import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import offgrid_voxels, ongrid_voxels

pytestmark = pytest.mark.gpu

MARGIN_EXCUSE = 1e-6


def _gpu_zoom(M, ctx, seq, g, x, **kw):
    h = M.mrf_sequence_load(ctx, seq)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        M.mrf_zoom_search(ctx, h, g, M.zoom_opts(**kw), fp, out)
        M.mrf_stream_sync(ctx)
        return M.results_to_numpy(out)[: x.shape[0]]
    finally:
        M.mrf_sequence_free(ctx, h)


def _compare(orc, g, res, ref, label):
    abc = np.stack([res["i_t1"], res["i_t2"], res["i_df"]], 1)
    same = (abc == ref["abc"]).all(1)
    excused = ref["min_margin"] < MARGIN_EXCUSE
    bad = ~same & ~excused
    assert not bad.any(), (f"{label}: {bad.sum()} voxels differ with margin >= {MARGIN_EXCUSE}: "
                           f"gpu {abc[bad][:4].tolist()} oracle {ref['abc'][bad][:4].tolist()} "
                           f"margin {ref['min_margin'][bad][:4]}")
    assert np.abs(res["cc"][same] - ref["cc"][same]).max() < 1e-5
    idx = np.array([orc.grid_index(g, *p) for p in ref["abc"]])
    assert (res["index"][same] == idx[same]).all()
    firm = same & (ref["min_margin"] >= 1e-5)
    assert (res["entries_evaluated"][firm] == ref["evaluated"][firm]).all()
    return int((~same).sum()), int(excused.sum())


def test_zoom_tiny_on_grid(M, ctx, oracle_lib):
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    ph, x = ongrid_voxels(oracle_lib, seq, g, 256, 30.0, 100)
    res = _gpu_zoom(M, ctx, seq, g, x)
    ref = oracle_lib.zoom(seq, g, x)
    diff, exc = _compare(oracle_lib, g, res, ref, "tiny")
    print(f"zoom tiny: differ={diff} excused={exc}")


def test_zoom_noise_free_recovery(M, ctx, oracle_lib):
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    ph, x = ongrid_voxels(oracle_lib, seq, g, 64, None, 200)
    res = _gpu_zoom(M, ctx, seq, g, x)
    assert (res["i_t1"] == ph["a"]).all() and (res["i_t2"] == ph["b"]).all()
    np.testing.assert_allclose(res["cc"], 1.0, atol=1e-5)
    np.testing.assert_allclose(res["m0"], ph["m0"], rtol=1e-4)


def test_zoom_3d_grid_offgrid_voxels(M, ctx, oracle_lib):
    """df searched too: the full df stage machine (steps 1a-1c, 3)."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 96, 20.0, 101)
    res = _gpu_zoom(M, ctx, seq, g, x)
    ref = oracle_lib.zoom(seq, g, x)
    diff, exc = _compare(oracle_lib, g, res, ref, "fp32_brute grid")
    print(f"zoom 3d: differ={diff} excused={exc}")


def test_zoom_fine_grid_subset(M, ctx, oracle_lib):
    """The 2.4e9-entry grid (1 ms / 0.5 ms / 0.1 Hz) on a 16x16 voxel subset.
    Decisions there separate candidates by less than 1e-6, so the traces may
    part; what must hold: CC of the GPU result within 1e-5 of the oracle's,
    and the GPU's final point is a local optimum of the oracle's FP64 CC at
    the finest step (up to 1e-6)."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["zoom_fine"]
    ph, x = offgrid_voxels(oracle_lib, seq, 256, 20.0, 103)
    res = _gpu_zoom(M, ctx, seq, g, x)
    ref = oracle_lib.zoom(seq, g, x)
    abc = np.stack([res["i_t1"], res["i_t2"], res["i_df"]], 1)
    same = (abc == ref["abc"]).all(1)
    firm = ref["min_margin"] >= MARGIN_EXCUSE
    assert (same | ~firm).all()
    assert np.abs(res["cc"] - ref["cc"]).max() < 1e-5
    t1, t2, df = S.grid_values(g)
    pts, owner = [], []
    for v in range(0, 256, 4):
        a, b, c = abc[v]
        for da in (-1, 0, 1):
            for db in (-1, 0, 1):
                aa, bb = a + da, b + db
                if 0 <= aa < g.n_t1 and 0 <= bb < g.n_t2 and t2[bb] < t1[aa]:
                    pts.append((aa, bb, c, da == 0 and db == 0))
                    owner.append(v)
    pts = np.array(pts)
    d = oracle_lib.simulate(seq, t1[pts[:, 0]], t2[pts[:, 1]], df[pts[:, 2]])
    owner = np.array(owner)
    cc = np.abs(np.sum(d.conj() * x[owner], 1)) / (np.linalg.norm(d, axis=1) * np.linalg.norm(x[owner], axis=1))
    for v in np.unique(owner):
        sel = owner == v
        centre = cc[sel & (pts[:, 3] == 1)][0]
        assert cc[sel].max() <= centre + 1e-6
        assert abs(centre - res["cc"][v]) < 1e-5
    print(f"zoom fine: same={int(same.sum())}/256 firm={int(firm.sum())} "
          f"max |dCC|={np.abs(res['cc'] - ref['cc']).max():.2e} mean evaluated={ref['evaluated'].mean():.0f}")


def test_zoom_full_slice_sampled(M, ctx, oracle_lib):
    """The benchmark's ZOOM workload: a 128x128 slice (16,384 voxels, SNR 20) on
    the 2.4e9-entry grid in one call. A voxel's answer does not depend on the
    batch: 48 sampled voxels searched alone return the same bits. Those voxels
    against the oracle's ZOOM: the same final point wherever the oracle's
    smallest decision margin is at least 1e-6, CC within 1e-5."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["zoom_fine"]
    _, x = offgrid_voxels(oracle_lib, seq, 128 * 128, 20.0, 103)
    res = _gpu_zoom(M, ctx, seq, g, x)
    pick = np.sort(np.random.default_rng(8).choice(x.shape[0], 48, replace=False))
    alone = _gpu_zoom(M, ctx, seq, g, x[pick])
    for f in ("i_t1", "i_t2", "i_df", "entries_evaluated"):
        np.testing.assert_array_equal(res[f][pick], alone[f], err_msg=f)
    for f in ("cc", "m0", "phase", "min_margin"):
        np.testing.assert_array_equal(res[f][pick].view(np.uint32), alone[f].view(np.uint32), err_msg=f)
    ref = oracle_lib.zoom(seq, g, x[pick])
    abc = np.stack([res["i_t1"][pick], res["i_t2"][pick], res["i_df"][pick]], 1)
    same = (abc == ref["abc"]).all(1)
    firm = ref["min_margin"] >= MARGIN_EXCUSE
    assert (same | ~firm).all()
    assert np.abs(res["cc"][pick] - ref["cc"]).max() < 1e-5
    assert (res["index"] >= 0).all()
    print(f"zoom full slice: same={int(same.sum())}/48 firm={int(firm.sum())}")


def test_zoom_custom_schedule_and_general_rf(M, ctx, oracle_lib):
    import math
    base = S.sequence(5, 300)
    rng = np.random.default_rng(17)
    seq = S.Sequence(base.flip_rad, rng.uniform(0, 2 * math.pi, 300), base.tr_ms, base.tr_ms * 0.4, 1, 20.0)
    g = S.Grid(200.0, 10.0, 120, 20.0, 4.0, 60, -20.0, 0.5, 81)
    ph, x = offgrid_voxels(oracle_lib, seq, 40, 30.0, 55, t1_range=(300.0, 1200.0), t2_range=(30.0, 200.0),
                           df_range=(-15.0, 15.0))
    kw = dict(t1_init_ms=700.0, t2_init_ms=80.0, s2=[(150.0, 60.0), (60.0, 24.0)], s4=[(0, 40.0), (1, 16.0), (0, 20.0), (1, 8.0)])
    res = _gpu_zoom(M, ctx, seq, g, x, **kw)
    ref = oracle_lib.zoom(seq, g, x, oracle_lib.default_zoom_opts(**kw))
    _compare(oracle_lib, g, res, ref, "custom")


def test_zoom_empty_batch(M, ctx):
    import ctypes as C
    seq = S.sequence(0, 50)
    h = M.mrf_sequence_load(ctx, seq)
    try:
        g = M.grid_desc(S.GRIDS["tiny"])
        assert M.lib().mrf_zoom_search(ctx, h, C.byref(g), None, None, 0, None, None) == M.MRF_OK
    finally:
        M.mrf_sequence_free(ctx, h)


def _gpu_zoom_dict(M, ctx, seq, g, x, dtype):
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, dtype)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        out = M.empty_results(x.shape[0])
        M.mrf_zoom_search_dict(ctx, d, M.zoom_opts(), fp, out)
        M.mrf_stream_sync(ctx)
        return M.results_to_numpy(out)[: x.shape[0]]
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_zoom_over_dictionary_tiny(M, ctx, oracle_lib):
    """Experiment 2's full-dictionary ZOOM: same search, CC read from the
    resident FP32-equivalent dictionary."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    ph, x = ongrid_voxels(oracle_lib, seq, g, 256, 30.0, 100)
    res = _gpu_zoom_dict(M, ctx, seq, g, x, M.MRF_F32)
    ref = oracle_lib.zoom(seq, g, x)
    _compare(oracle_lib, g, res, ref, "dict tiny")
    np.testing.assert_allclose(res["m0"], ref["m0"], rtol=1e-4)


def test_zoom_over_dictionary_3d(M, ctx, oracle_lib):
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 96, 20.0, 101)
    res = _gpu_zoom_dict(M, ctx, seq, g, x, M.MRF_F32)
    ref = oracle_lib.zoom(seq, g, x)
    diff, exc = _compare(oracle_lib, g, res, ref, "dict 3d")
    print(f"zoom dict 3d: differ={diff} excused={exc}")


def test_zoom_over_bf16_dictionary_runs(M, ctx, oracle_lib):
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 64, 20.0, 131)
    res = _gpu_zoom_dict(M, ctx, seq, g, x, M.MRF_BF16)
    ref = oracle_lib.zoom(seq, g, x)
    # bf16 CC is within about 1e-3 of the FP64 CC of the same entry
    t1, t2, df = S.grid_values(g)
    a, b, c = res["i_t1"], res["i_t2"], res["i_df"]
    d = oracle_lib.simulate(seq, t1[a], t2[b], df[c])
    occ = np.abs(np.sum(d.conj() * x, 1)) / (np.linalg.norm(d, axis=1) * np.linalg.norm(x, axis=1))
    assert np.abs(res["cc"] - occ).max() < 5e-3
    print(f"zoom bf16 dict: agreement with the FP64 ZOOM {np.mean((np.stack([a, b, c], 1) == ref['abc']).all(1)):.3f}")


def test_zoom_dict_rejects_fp8(M, ctx):
    import ctypes as C
    seq = S.sequence(0, 64)
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, S.GRIDS["tiny"], M.MRF_FP8E4M3)
    try:
        fp = torch.zeros((2, 64), dtype=torch.complex64, device="cuda")
        out = M.empty_results(2)
        rc = M.lib().mrf_zoom_search_dict(ctx, d, None, C.c_void_p(fp.data_ptr()), 2, C.c_void_p(out.data_ptr()), None)
        assert rc == M.MRF_E_UNSUPPORTED
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def _zoom_both(M, ctx, seq, grid, x, **kw):
    """mrf_zoom_search (step 3 batched by (T1, T2) line) and the single-kernel
    search of mrf_zoom_search_static on the same voxels."""
    import ctypes as C
    L = M.lib()
    h = M.mrf_sequence_load(ctx, seq)
    try:
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        g = M.grid_desc(grid)
        o = M.zoom_opts(**kw)
        res = []
        for fn in (L.mrf_zoom_search, L.mrf_zoom_search_static):
            out = M.empty_results(x.shape[0])
            rc = fn(ctx, h, C.byref(g), C.byref(o), C.c_void_p(fp.data_ptr()), x.shape[0],
                    C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == M.MRF_OK, M.last_error()
            M.mrf_stream_sync(ctx)
            res.append(M.results_to_numpy(out)[: x.shape[0]])
        return res
    finally:
        M.mrf_sequence_free(ctx, h)


@pytest.mark.parametrize("grid,v,seed", [("precision", 600, 11), ("zoom_fine", 160, 12), ("precision", 1, 13),
                                         ("precision", 17, 14)])
def test_zoom_batched_step3_equals_per_voxel_scan(M, ctx, oracle_lib, grid, v, seed):
    """Step 3 batched over the voxels sharing (T1, T2) computes every CC with
    the per-voxel kernel's FP32 operations in the same order, so the two
    searches agree bit for bit: same decisions, evaluation counts, margins and
    CC. Covers several lines, lines of more than one 16-voxel tile, a single
    voxel, windows clipped at both ends of the df axis and the 7 chunks of
    the 801-point df axis."""
    seq = S.sequence(1, 1000)
    ph, x = offgrid_voxels(oracle_lib, seq, v, 20.0, seed)
    split, single = _zoom_both(M, ctx, seq, S.GRIDS[grid], x)
    for f in ("index", "i_t1", "i_t2", "i_df", "entries_evaluated"):
        assert np.array_equal(split[f], single[f]), f
    for f in ("cc", "min_margin", "m0", "phase"):
        assert np.array_equal(split[f].view(np.uint32), single[f].view(np.uint32)), f


def test_zoom_batched_step3_general_rf_against_oracle(M, ctx, oracle_lib):
    """The other instantiations of the line kernel (general RF rotation, TE not
    half of TR) on a grid whose windows cover 3 chunks, against the oracle and
    against the per-voxel kernel."""
    import math
    base = S.sequence(5, 300)
    rng = np.random.default_rng(21)
    seq = S.Sequence(base.flip_rad, rng.uniform(0, 2 * math.pi, 300), base.tr_ms, base.tr_ms * 0.4, 1, 20.0)
    g = S.Grid(200.0, 20.0, 60, 20.0, 8.0, 30, -40.0, 0.25, 321)
    ph, x = offgrid_voxels(oracle_lib, seq, 48, 30.0, 57, t1_range=(300.0, 1200.0), t2_range=(30.0, 200.0),
                           df_range=(-38.0, 38.0))
    split, single = _zoom_both(M, ctx, seq, g, x)
    for f in ("index", "entries_evaluated"):
        assert np.array_equal(split[f], single[f]), f
    assert np.array_equal(split["cc"].view(np.uint32), single["cc"].view(np.uint32))
    ref = oracle_lib.zoom(seq, g, x)
    _compare(oracle_lib, g, split, ref, "general rf, 321 df")


@pytest.mark.parametrize("grid,s3", [("fp32_brute", 0.0), ("fp32_brute", 0.02), ("precision", 0.4)])
def test_zoom_step3_narrow_or_empty_window(M, ctx, oracle_lib, grid, s3):
    """Step-3 windows of the centre alone (s3_half_frac 0: no scan) and of a
    few positions (both on the single-kernel path: fewer than 64 positions),
    and windows of 71 positions clipped by the df axis on the batched path,
    against the oracle."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS[grid]
    ph, x = offgrid_voxels(oracle_lib, seq, 64, 20.0, 202)
    res = _gpu_zoom(M, ctx, seq, g, x, s3_half_frac=s3)
    ref = oracle_lib.zoom(seq, g, x, oracle_lib.default_zoom_opts(s3_half_frac=s3))
    _compare(oracle_lib, g, res, ref, f"s3_half_frac={s3}")


def _piecewise_voxels(orc, seq, rows, cols, seed, snr=30.0):
    ph = S.phantom_piecewise(seed, rows, cols)
    clean = orc.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    g_re, g_im = S.noise_draws(seed, rows * cols, seq.n)
    return ph, S.compose_voxels(clean, ph["m0"], ph["phase"], g_re, g_im, snr)


def _compare_chains(orc, g, res, ref, L, half, label):
    """GPU prior chains against the oracle's: within each chain of L voxels,
    voxel by voxel, the final point must match (CC within 1e-5, same index,
    same evaluation count where margins exceed 1e-5) until the first voxel
    the oracle's margin excuses (< 1e-6) and the GPU answers differently;
    the rest of that chain starts from another result and is not compared.
    Every GPU result lies in the box around its own predecessor's result."""
    V = res.shape[0]
    abc = np.stack([res["i_t1"], res["i_t2"], res["i_df"]], 1)
    h = [int(np.floor(w / s + 1e-9)) for w, s in zip(half, (g.t1_step, g.t2_step, g.df_step))]
    compared, cut = 0, 0
    for c0 in range(0, V, L):
        for v in range(c0, min(c0 + L, V)):
            if v > c0:
                assert (np.abs(abc[v] - abc[v - 1]) <= h).all(), f"{label}: voxel {v} outside its prior box"
            if not (abc[v] == ref["abc"][v]).all():
                assert ref["min_margin"][v] < MARGIN_EXCUSE, (
                    f"{label}: voxel {v} differs with margin {ref['min_margin'][v]}: "
                    f"gpu {abc[v].tolist()} oracle {ref['abc'][v].tolist()}")
                cut += min(c0 + L, V) - v
                break
            compared += 1
            assert abs(res["cc"][v] - ref["cc"][v]) < 1e-5
            assert res["index"][v] == orc.grid_index(g, *ref["abc"][v])
            if ref["min_margin"][v] >= 1e-5:
                assert res["entries_evaluated"][v] == ref["evaluated"][v], f"{label}: voxel {v} evaluations"
    return compared, cut


def test_zoom_prior_single_chain_against_oracle(M, ctx, oracle_lib):
    """The paper's spatial-neighbour prior (Methods, Experiment 3) as its
    single chain through an 8 x 8 piecewise-smooth slice in raster order,
    with the paper's windows (T1p +- 3000 ms, T2p +- 800 ms, dfp +- 150 Hz)
    and each search started at the preceding voxel's result: against the
    oracle's chain."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = _piecewise_voxels(oracle_lib, seq, 8, 8, 31)
    half = (3000.0, 800.0, 150.0)
    res = _gpu_zoom(M, ctx, seq, g, x, prior=(64, half))
    ref = oracle_lib.zoom_prior(seq, g, x, half=half)
    compared, cut = _compare_chains(oracle_lib, g, res, ref, 64, half, "single chain")
    print(f"zoom prior, one chain of 64: compared={compared} after an excused divergence={cut}")
    assert compared >= 16


@pytest.mark.parametrize("half,start", [((3000.0, 800.0, 150.0), 1), ((200.0, 30.0, 6.0), 1),
                                        ((200.0, 30.0, 6.0), 0)])
def test_zoom_prior_chains_against_oracle(M, ctx, oracle_lib, half, start):
    """Chains of one row (16 voxels) through a 16 x 16 piecewise-smooth slice:
    the paper's windows and narrow ones that bound most searches, started at
    the preceding voxel's result or at the options' start clipped into the
    box; against the oracle's chains."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = _piecewise_voxels(oracle_lib, seq, 16, 16, 32)
    res = _gpu_zoom(M, ctx, seq, g, x, prior=(16, half, start))
    ref = oracle_lib.zoom_prior(seq, g, x, chain=16, half=half, start_from_prior=bool(start))
    compared, cut = _compare_chains(oracle_lib, g, res, ref, 16, half, f"chains {half} start={start}")
    print(f"zoom prior chains {half} start={start}: compared={compared} cut={cut}")
    assert compared >= 128


def test_zoom_prior_covering_the_grid_is_the_plain_search(M, ctx, oracle_lib):
    """Windows wider than every axis and the start left at the options'
    start: every search runs on the whole grid from the same point, so the
    results are those of the plain search bit for bit (chains of 13 voxels,
    a ragged last chain)."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 13 * 7 + 5, 20.0, 33)
    plain = _gpu_zoom(M, ctx, seq, g, x)
    pri = _gpu_zoom(M, ctx, seq, g, x, prior=(13, (1e6, 1e6, 1e6), 0))
    for f in ("index", "entries_evaluated"):
        assert np.array_equal(plain[f], pri[f]), f
    assert np.array_equal(plain["cc"].view(np.uint32), pri["cc"].view(np.uint32))


def test_zoom_prior_started_at_the_optimum(M, ctx, oracle_lib):
    """Noise-free voxels of one on-grid tissue in a chain: every voxel after
    the first starts at its own optimum, so no decision moves and each needs
    the 25 evaluations the oracle pin counts by hand on the tiny grid."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    rng = np.random.default_rng(11)
    clean = oracle_lib.simulate(seq, np.full(9, 1400.0), np.full(9, 100.0), np.zeros(9))
    x = clean * (rng.uniform(0.5, 1.0, 9) * np.exp(1j * rng.uniform(0, 2 * np.pi, 9)))[:, None]
    res = _gpu_zoom(M, ctx, seq, g, x, prior=(9, (3000.0, 800.0, 150.0)))
    assert list(res["i_t1"]) == [13] * 9 and list(res["i_t2"]) == [4] * 9
    assert list(res["entries_evaluated"][1:]) == [25] * 8
    np.testing.assert_allclose(res["cc"], 1.0, atol=1e-5)


def test_zoom_prior_options_checked(M, ctx):
    import ctypes as C
    seq = S.sequence(0, 50)
    h = M.mrf_sequence_load(ctx, seq)
    try:
        g = M.grid_desc(S.GRIDS["tiny"])
        fp = torch.zeros((4, 50), dtype=torch.complex64, device="cuda")
        out = M.empty_results(4)
        L = M.lib()
        for kw in (dict(prior=(-1, (3000.0, 800.0, 150.0))), dict(prior=(2, (3000.0, 800.0, 150.0), 2)),
                   dict(prior=(2, (-1.0, 800.0, 150.0))), dict(prior=(2, (3000.0, float("inf"), 150.0)))):
            o = M.zoom_opts(**kw)
            rc = L.mrf_zoom_search(ctx, h, C.byref(g), C.byref(o), C.c_void_p(fp.data_ptr()), 4,
                                   C.c_void_p(out.data_ptr()), None)
            assert rc == M.MRF_E_INVALID
        o = M.zoom_opts(prior=(2, (3000.0, 800.0, 150.0)))
        rc = L.mrf_zoom_search_static(ctx, h, C.byref(g), C.byref(o), C.c_void_p(fp.data_ptr()), 4,
                                      C.c_void_p(out.data_ptr()), None)
        assert rc == M.MRF_E_UNSUPPORTED
    finally:
        M.mrf_sequence_free(ctx, h)


def test_zoom_work_counters(M, ctx, oracle_lib):
    """The profile's ZOOM work counters after one search on a grid whose step
    3 runs batched: step-3 positions are part of the evaluation count, the
    line kernel simulated candidates, the packed kernel ran rounds and
    simulated candidates, both were timed once, and a reset clears
    everything."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["precision"]
    ph, x = offgrid_voxels(oracle_lib, seq, 48, 20.0, 41)
    M.mrf_profile_read(ctx, reset=True)
    M.mrf_profile_enable(ctx, True)
    res = _gpu_zoom(M, ctx, seq, g, x)
    M.mrf_profile_enable(ctx, False)
    p = M.mrf_profile_read(ctx, reset=True)
    ev = int(res["entries_evaluated"].sum())
    assert 0 < p.zoomline_pairs < ev
    assert p.zoomline_entries > 0
    assert p.zoom_rounds > 0 and p.zoom_candidates > 0 and p.zoom_max_voxel_rounds > 0
    assert p.zoom_timed == 1 and p.zoomline_timed == 1 and p.zoom_ms > p.zoomline_ms > 0
    q = M.mrf_profile_read(ctx)
    assert q.zoomline_pairs == 0 and q.zoom_rounds == 0 and q.zoom_timed == 0


def test_zoom_prior_edge_chains(M, ctx, oracle_lib):
    """Chains of one voxel are the plain search bit for bit (every voxel is a
    chain's first); a single voxel, and a chain longer than the slice, are
    the oracle's chain."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 21, 20.0, 34)
    plain = _gpu_zoom(M, ctx, seq, g, x)
    one = _gpu_zoom(M, ctx, seq, g, x, prior=(1, (200.0, 30.0, 6.0)))
    for f in ("index", "entries_evaluated"):
        assert np.array_equal(plain[f], one[f]), f
    assert np.array_equal(plain["cc"].view(np.uint32), one["cc"].view(np.uint32))
    half = (200.0, 30.0, 6.0)
    for V, L in ((1, 1), (21, 1000)):
        res = _gpu_zoom(M, ctx, seq, g, x[:V], prior=(L, half))
        ref = oracle_lib.zoom_prior(seq, g, x[:V], chain=min(L, V), half=half)
        compared, cut = _compare_chains(oracle_lib, g, res, ref, min(L, V), half, f"V={V} chain={L}")
        assert compared >= 1
