"""GPU brute-force DGS (tensor-core matcher + re-score) against the FP64
oracle's brute force (Theory: argmax of Eq. 1 over every grid entry).

Bar: CC within 1e-5 absolute; matched index identical except where the
oracle's top-two CC gap is below 1e-6 (those are counted and reported)."""
import math

import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import offgrid_voxels, ongrid_voxels

pytestmark = pytest.mark.gpu

GAP_EXCUSE = 1e-6
CC_TOL = 1e-5


def _run(M, ctx, d, x, precision, top_k, rescore):
    fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    out = M.empty_results(x.shape[0])
    M.mrf_match_bruteforce(ctx, d, fp, M.match_opts(precision, top_k, rescore), out)
    M.mrf_stream_sync(ctx)
    return M.results_to_numpy(out)[: x.shape[0]]


def _topk(M, ctx, d, x, precision, k):
    fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    idx = torch.empty((x.shape[0], k), dtype=torch.int64, device="cuda")
    cc2 = torch.empty((x.shape[0], k), dtype=torch.float32, device="cuda")
    M.mrf_match_topk(ctx, d, fp, precision, k, idx, cc2)
    M.mrf_stream_sync(ctx)
    return idx.cpu().numpy(), cc2.cpu().numpy()


def _compare(res, ref, label):
    gap = ref["cc"][:, 0] - ref["cc"][:, 1]
    same = res["index"] == ref["idx"][:, 0]
    excused = gap < GAP_EXCUSE
    bad = ~same & ~excused
    assert not bad.any(), (f"{label}: {bad.sum()} voxels differ with gap >= {GAP_EXCUSE}: "
                           f"gpu {res['index'][bad][:5]} oracle {ref['idx'][bad, 0][:5]} gap {gap[bad][:5]}")
    ok = same
    assert np.abs(res["cc"][ok] - ref["cc"][ok, 0]).max() < CC_TOL
    return int((~same).sum()), int(excused.sum())


@pytest.fixture(scope="module")
def tiny(M, ctx, oracle_lib):
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    h = M.mrf_sequence_load(ctx, seq)
    dicts = {dt: M.mrf_dict_generate(ctx, h, g, dt) for dt in (M.MRF_F32, M.MRF_BF16, M.MRF_FP8E4M3)}
    ph, x = ongrid_voxels(oracle_lib, seq, g, 256, 30.0, 100)
    ref = oracle_lib.bruteforce(seq, g, x, k=8)
    yield dict(seq=seq, grid=g, h=h, dicts=dicts, x=x, ph=ph, ref=ref)
    for d in dicts.values():
        M.mrf_dict_free(ctx, d)
    M.mrf_sequence_free(ctx, h)


@pytest.fixture(scope="module")
def ragged(M, ctx, oracle_lib):
    """Several 256-entry tiles with a ragged tail, and V not a multiple of 64."""
    seq = S.sequence(2, 200)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    h = M.mrf_sequence_load(ctx, seq)
    dicts = {dt: M.mrf_dict_generate(ctx, h, g, dt) for dt in (M.MRF_F32, M.MRF_BF16, M.MRF_FP8E4M3)}
    ph, x = offgrid_voxels(oracle_lib, seq, 150, 25.0, 7, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-11.0, 11.0))
    ref = oracle_lib.bruteforce(seq, g, x, k=8)
    yield dict(seq=seq, grid=g, h=h, dicts=dicts, x=x, ph=ph, ref=ref, D=oracle_lib.grid_count(g))
    for d in dicts.values():
        M.mrf_dict_free(ctx, d)
    M.mrf_sequence_free(ctx, h)


def test_tiny_fp32_recovers_on_grid_voxels(M, ctx, tiny):
    res = _run(M, ctx, tiny["dicts"][M.MRF_F32], tiny["x"], M.MRF_F32, 4, 1)
    _compare(res, tiny["ref"], "tiny fp32")
    np.testing.assert_allclose(res["m0"], tiny["ref"]["m0"], rtol=1e-4)
    dphi = np.angle(np.exp(1j * (res["phase"] - tiny["ref"]["phase"])))
    assert np.abs(dphi).max() < 1e-4
    assert (res["entries_evaluated"] == 193).all()


def test_tiny_topk_lists(M, ctx, tiny):
    idx, cc2 = _topk(M, ctx, tiny["dicts"][M.MRF_F32], tiny["x"], M.MRF_F32, 8)
    ref = tiny["ref"]
    np.testing.assert_allclose(np.sqrt(np.maximum(cc2, 0)), ref["cc"], atol=1e-5)
    # where consecutive oracle CCs are well separated, the order must agree
    sep = np.diff(ref["cc"], axis=1) < -1e-5
    for v in range(idx.shape[0]):
        for q in range(7):
            if sep[v, : q + 1].all():
                assert idx[v, q] == ref["idx"][v, q]


def acc_bound(n, precision):
    """Bound on the FP32 accumulation error of a tensor-core CC of unit
    vectors over n timepoints: each MMA adds its products to the accumulator
    with an error of at most one unit in the last place of the running sum
    (whose magnitude stays below sum |x_j d_j| <= 1), so each of Re and Im is
    off by at most steps * 2^-23 and the CC by sqrt(2) times that. Steps per
    result: 2n / 16 fp16 or bf16 MMAs, 2n / 32 e4m3 ones (two per K block in
    the MRF_F32 split form)."""
    k16, k32 = -(-2 * n // 16), -(-2 * n // 32)
    steps = {0: k16 + 2 * k32, 1: k16, 2: k32}[precision]
    return math.sqrt(2) * steps * 2.0 ** -23


# Rigorous bound on |CC_approx - CC| for unit vectors: each operand rounded
# with unit roundoff u gives a per-component error <= (2u + u^2) ||x|| ||d||,
# so |CC_approx - CC| <= sqrt(2) (2u + u^2), plus the accumulation (acc_bound).
# MRF_F32 (fp16 product plus e4m3 products of the two fp16 residuals, each
# residual <= 2^-11 of its operand, e4m3 unit roundoff 2^-4): per component
# <= (2^-22 + 2 * 2^-11 * (2^-3 + 2^-8)) |x_j d_j|.
EPS_STORE = {0: math.sqrt(2) * (2 ** -22 + 2 ** -10 * (2 ** -3 + 2 ** -8)),
             1: math.sqrt(2) * (2 * 2 ** -9 + 2 ** -18),
             2: math.sqrt(2) * (2 * 2 ** -4 + 2 ** -8)}


def eps_bound(n, precision):
    return EPS_STORE[precision] + acc_bound(n, precision)


def _rescore_reference(orc, seq, g, x, cand):
    """FP64 CC of every candidate (oracle simulation), best with ties to the smaller index."""
    t1, t2, df = S.grid_values(g)
    a, b, c = orc.grid_params(g)
    best = np.full(x.shape[0], -1)
    gap = np.full(x.shape[0], np.inf)
    for v in range(x.shape[0]):
        ids = cand[v][cand[v] >= 0]
        d = orc.simulate(seq, t1[a[ids]], t2[b[ids]], df[c[ids]])
        cc = np.abs(d.conj() @ x[v]) / (np.linalg.norm(d, axis=1) * np.linalg.norm(x[v]))
        order = np.lexsort((ids, -cc))
        best[v] = ids[order[0]]
        if len(ids) > 1:
            gap[v] = cc[order[0]] - cc[order[1]]
    return best, gap


@pytest.mark.parametrize("precision,top_k", [(0, 1), (0, 4), (1, 8), (1, 32), (2, 8), (2, 32)])
def test_ragged_all_precisions(M, ctx, oracle_lib, ragged, precision, top_k):
    d = ragged["dicts"][precision]
    res = _run(M, ctx, d, ragged["x"], precision, top_k, 1)
    assert (res["entries_evaluated"] == ragged["D"]).all()
    ref = ragged["ref"]
    if precision == 0:
        diff, exc = _compare(res, ref, f"ragged p{precision} k{top_k}")
        print(f"ragged precision={precision} k={top_k}: differ={diff} excused={exc}")
        return
    # the re-score must return the FP64 best of its own candidate list
    cand, cc2 = _topk(M, ctx, d, ragged["x"], precision, top_k)
    best, cgap = _rescore_reference(oracle_lib, ragged["seq"], ragged["grid"], ragged["x"], cand)
    wrong = (res["index"] != best) & (cgap >= GAP_EXCUSE)
    assert not wrong.any(), f"re-score picked a non-best candidate for {int(wrong.sum())} voxels"
    # CC of the returned entry within 1e-5 of the oracle's CC of that entry
    t1, t2, df = S.grid_values(ragged["grid"])
    a, b, c = oracle_lib.grid_params(ragged["grid"])
    dd = oracle_lib.simulate(ragged["seq"], t1[a[res["index"]]], t2[b[res["index"]]], df[c[res["index"]]])
    x = ragged["x"]
    occ = np.abs(np.sum(dd.conj() * x, 1)) / (np.linalg.norm(dd, axis=1) * np.linalg.norm(x, axis=1))
    assert np.abs(res["cc"] - occ).max() < CC_TOL
    # certificate: a_1 - a_k > 2 eps means no entry outside the list can win
    a1 = np.sqrt(np.maximum(cc2[:, 0], 0))
    ak = np.sqrt(np.maximum(cc2[:, -1], 0))
    cert = (a1 - ak > 2 * eps_bound(ragged["seq"].n, precision)) | (cand[:, -1] < 0)
    gap = ref["cc"][:, 0] - ref["cc"][:, 1]
    agree = res["index"] == ref["idx"][:, 0]
    assert (agree | ~cert | (gap < GAP_EXCUSE)).all(), "a certified voxel disagrees with the oracle"
    rate = agree.mean()
    print(f"ragged precision={precision} k={top_k}: agreement={rate:.3f} certified={int(cert.sum())}/{len(cert)}")
    assert rate >= (0.9 if precision == 1 else 0.5)


def test_ragged_no_rescore_keeps_tensor_core_rank1(M, ctx, ragged):
    idx, _ = _topk(M, ctx, ragged["dicts"][M.MRF_BF16], ragged["x"], M.MRF_BF16, 1)
    res = _run(M, ctx, ragged["dicts"][M.MRF_BF16], ragged["x"], M.MRF_BF16, 1, 0)
    assert (res["index"] == idx[:, 0]).all()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_seeded_topk_head_equals_unseeded_list(M, ctx, oracle_lib, precision):
    """Top-k lists with k >= 8 over a dictionary of at least 4 x 256 x 64
    entries start from a per-voxel bound, the k-th best CC^2 of every 64th
    entry; values below it cannot be among the k best. The head of such a
    list must therefore equal, bit for bit, the top-4 list that the same
    arithmetic gives without a bound."""
    seq = S.sequence(3, 200)
    g = S.Grid(100.0, 20.0, 96, 10.0, 10.0, 40, -20.0, 2.0, 21)
    assert oracle_lib.grid_count(g) >= 4 * 256 * 64
    ph, x = offgrid_voxels(oracle_lib, seq, 200, 20.0, 17, t1_range=(150.0, 1900.0), t2_range=(15.0, 380.0),
                           df_range=(-18.0, 18.0))
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, precision)
    try:
        i32, c32 = _topk(M, ctx, d, x, precision, 32)
        i4, c4 = _topk(M, ctx, d, x, precision, 4)
        np.testing.assert_array_equal(i32[:, :4], i4)
        np.testing.assert_array_equal(c32[:, :4], c4)
        assert (np.diff(c32, axis=1) <= 0).all()
        assert all(len(set(r)) == 32 for r in i32)
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_topk_larger_than_dictionary(M, ctx, oracle_lib):
    seq = S.sequence(3, 64)
    g = S.Grid(300.0, 100.0, 4, 20.0, 40.0, 3, 0.0, 1.0, 1)   # 12 entries
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
    try:
        ph, x = offgrid_voxels(oracle_lib, seq, 5, 30.0, 9, t1_range=(300.0, 600.0), t2_range=(20.0, 100.0),
                               df_range=(-0.1, 0.1))
        idx, cc2 = _topk(M, ctx, d, x, M.MRF_F32, 32)
        assert (idx[:, 12:] == -1).all() and (idx[:, :12] >= 0).all()
        assert sorted(idx[0, :12].tolist()) == list(range(12))
        res = _run(M, ctx, d, x, M.MRF_F32, 32, 1)
        ref = oracle_lib.bruteforce(seq, g, x, k=2)
        assert (res["index"] == ref["idx"][:, 0]).all()
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_empty_and_invalid_calls(M, ctx, tiny):
    d = tiny["dicts"][M.MRF_F32]
    out = M.empty_results(1)
    L = M.lib()
    import ctypes as C
    o = M.match_opts(M.MRF_F32, 4, 1)
    assert L.mrf_match_bruteforce(ctx, d, None, 0, C.byref(o), None, None) == M.MRF_OK
    bad = M.match_opts(M.MRF_BF16, 4, 1)
    fp = torch.zeros((1, 200), dtype=torch.complex64, device="cuda")
    assert L.mrf_match_bruteforce(ctx, d, C.c_void_p(fp.data_ptr()), 1, C.byref(bad), C.c_void_p(out.data_ptr()), None) == M.MRF_E_INVALID
    bad = M.match_opts(M.MRF_F32, 3, 1)
    assert L.mrf_match_bruteforce(ctx, d, C.c_void_p(fp.data_ptr()), 1, C.byref(bad), C.c_void_p(out.data_ptr()), None) == M.MRF_E_INVALID


def test_zero_voxel_gives_no_match(M, ctx, tiny):
    x = np.zeros((3, 200), np.complex128)
    x[1] = tiny["x"][0]
    res = _run(M, ctx, tiny["dicts"][M.MRF_F32], x, M.MRF_F32, 4, 1)
    assert res["index"][0] == -1 and res["index"][2] == -1
    assert res["index"][1] == tiny["ref"]["idx"][0, 0]


def test_full_size_fp32_sampled(M, ctx, oracle_lib):
    """64x64 slice, N = 1000, 614,508 entries (the benchmark workload): all
    4096 voxels matched on the GPU, 12 sampled voxels checked against the
    oracle's exhaustive search."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    ph, x = offgrid_voxels(oracle_lib, seq, 4096, 20.0, 101)
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
    try:
        res = _run(M, ctx, d, x, M.MRF_F32, 4, 1)
        pick = np.random.default_rng(5).choice(4096, 12, replace=False)
        ref = oracle_lib.bruteforce(seq, g, x[pick], k=2)
        diff, exc = _compare(res[pick], ref, "full fp32")
        print(f"full-size fp32: differ={diff} excused={exc} of 12")
        assert (res["index"] >= 0).all()
        # the tensor core's own CCs (no re-score) of 64 voxels' top-4 lists
        # against the oracle's CC of the same entries: within the accumulation
        # bound (the values run low, about 1e-5 on average at N = 1000, as
        # accumulation that rounds toward zero would make them) plus the 1e-5
        # CC bar for the stored values and the FP32 simulation
        sub = np.random.default_rng(6).choice(4096, 64, replace=False)
        idx, cc2 = _topk(M, ctx, d, x[sub], M.MRF_F32, 4)
        t1, t2, df = S.grid_values(g)
        a, b, c = oracle_lib.grid_params(g)
        flat = idx.reshape(-1)
        dd = oracle_lib.simulate(seq, t1[a[flat]], t2[b[flat]], df[c[flat]]).reshape(64, 4, -1)
        xs = x[sub][:, None, :]
        occ = np.abs(np.sum(dd.conj() * xs, -1)) / (np.linalg.norm(dd, axis=-1) * np.linalg.norm(xs, axis=-1))
        err = np.abs(np.sqrt(np.maximum(cc2, 0)) - occ)
        print(f"full-size fp32 raw top-4 CC: max error {err.max():.3g}")
        assert err.max() < CC_TOL + acc_bound(1000, M.MRF_F32)
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_full_size_precision_grid_sampled(M, ctx, oracle_lib):
    """64x64 slice, N = 1000, 12,024,855 entries (the BF16 / FP8 benchmark
    workload): BF16 top-8 and FP8 top-32 with the re-score on all 4096 voxels,
    against the FP32-equivalent brute force over the same grid (in ranges, no
    resident dictionary): never above its CC, the returned entries' CCs equal
    to the oracle's for 8 sampled voxels, and after the windowed refinement
    its index wherever its top-two gap is at least 1e-6."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["precision"]
    _, x = offgrid_voxels(oracle_lib, seq, 4096, 20.0, 101)
    h = M.mrf_sequence_load(ctx, seq)
    try:
        ref = _run_grid(M, ctx, h, g, x, M.MRF_F32, 4, 0)
        sure = ref["min_margin"] >= GAP_EXCUSE
        # the FP32-equivalent brute force over the whole grid pinned to the oracle's exhaustive search
        # on 4 voxels (12,024,855 FP64 fingerprints simulated once, every entry correlated)
        pick4 = np.random.default_rng(7).choice(4096, 4, replace=False)
        orc = oracle_lib.bruteforce(seq, g, x[pick4], k=2)
        diff, exc = _compare(ref[pick4], orc, "12M-entry grid, FP32-equivalent brute force in ranges")
        print(f"12M-entry grid vs the oracle's exhaustive search: differ={diff} excused={exc} of 4")
        t1, t2, df = S.grid_values(g)
        a, b, c = oracle_lib.grid_params(g)
        pick = np.random.default_rng(6).choice(4096, 8, replace=False)
        fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        for dt, k, floor in ((M.MRF_BF16, 8, 0.98), (M.MRF_FP8E4M3, 32, 0.97)):
            d = M.mrf_dict_generate(ctx, h, g, dt)
            out = M.empty_results(4096)
            try:
                M.mrf_match_bruteforce(ctx, d, fp, M.match_opts(dt, k, 1), out)
                M.mrf_stream_sync(ctx)
                res = M.results_to_numpy(out)[:4096].copy()
                M.mrf_refine(ctx, h, g, fp, out)
                M.mrf_stream_sync(ctx)
                ref2 = M.results_to_numpy(out)[:4096]
            finally:
                M.mrf_dict_free(ctx, d)
            assert (res["entries_evaluated"] == ref["entries_evaluated"]).all()
            # never above the FP32-equivalent brute force's CC (the maximum over every entry)
            assert (res["cc"] <= ref["cc"] + 2e-6).all()
            assert (ref2["cc"] <= ref["cc"] + 2e-6).all()
            i = res["index"][pick]
            dd = oracle_lib.simulate(seq, t1[a[i]], t2[b[i]], df[c[i]])
            xx = x[pick]
            occ = np.abs(np.sum(dd.conj() * xx, 1)) / (np.linalg.norm(dd, axis=1) * np.linalg.norm(xx, axis=1))
            assert np.abs(res["cc"][pick] - occ).max() < CC_TOL
            agree = (res["index"] == ref["index"])[sure].mean()
            agree2 = (ref2["index"] == ref["index"])[sure].mean()
            print(f"  oracle exhaustive on 4 voxels: re-scored index equal {int((res['index'][pick4] == orc['idx'][:, 0]).sum())}"
                  f"/4, after refinement {int((ref2['index'][pick4] == orc['idx'][:, 0]).sum())}/4")
            print(f"full-size 12M dtype={dt} top-{k}: agreement with FP32 brute force {agree:.4f}, after "
                  f"refinement {agree2:.4f} ({int(sure.sum())} voxels with a gap >= 1e-6)")
            assert agree2 >= floor
    finally:
        M.mrf_sequence_free(ctx, h)


def _run_grid(M, ctx, h, grid, x, precision, top_k, chunk):
    fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    out = M.empty_results(x.shape[0])
    M.mrf_match_bruteforce_grid(ctx, h, grid, fp, M.match_opts(precision, top_k, 1), out, chunk)
    M.mrf_stream_sync(ctx)
    return M.results_to_numpy(out)[: x.shape[0]]


def _row_entries(oracle_lib, g):
    a, _, _ = oracle_lib.grid_params(g)
    return int(np.bincount(a).max())


@pytest.mark.parametrize("rows", [0, 1, 3])
def test_chunked_grid_fp32_against_oracle(M, ctx, oracle_lib, ragged, rows):
    """Brute force over ranges of whole T1 rows (one range; one row per range;
    about three rows per range): whole-grid indices, parameters and counts,
    and the oracle's answer (Theory: argmax of Eq. 1 over every entry)."""
    g = ragged["grid"]
    chunk = 0 if rows == 0 else rows * _row_entries(oracle_lib, g) + 5
    res = _run_grid(M, ctx, ragged["h"], g, ragged["x"], M.MRF_F32, 4, chunk)
    assert (res["entries_evaluated"] == ragged["D"]).all()
    a, b, c = oracle_lib.grid_params(g)
    t1, t2, df = S.grid_values(g)
    i = res["index"]
    assert ((i >= 0) & (i < ragged["D"])).all()
    assert (a[i] == res["i_t1"]).all() and (b[i] == res["i_t2"]).all() and (c[i] == res["i_df"]).all()
    np.testing.assert_array_equal(res["t1_ms"], t1[a[i]].astype(np.float32))
    np.testing.assert_array_equal(res["t2_ms"], t2[b[i]].astype(np.float32))
    diff, exc = _compare(res, ragged["ref"], f"chunked rows={rows}")
    print(f"chunked rows={rows}: differ={diff} excused={exc}")
    assert (res["min_margin"] >= 0).all()


def test_chunked_grid_single_range_equals_resident(M, ctx, ragged):
    """With one range the chunked search is the resident search, bit for bit."""
    res = _run_grid(M, ctx, ragged["h"], ragged["grid"], ragged["x"], M.MRF_F32, 4, 0)
    ref = _run(M, ctx, ragged["dicts"][M.MRF_F32], ragged["x"], M.MRF_F32, 4, 1)
    for f in ("index", "i_t1", "i_t2", "i_df", "entries_evaluated"):
        np.testing.assert_array_equal(res[f], ref[f], err_msg=f)
    for f in ("cc", "m0", "phase"):
        np.testing.assert_array_equal(res[f].view(np.uint32), ref[f].view(np.uint32), err_msg=f)
    np.testing.assert_allclose(res["min_margin"], ref["min_margin"], atol=1e-7)


@pytest.mark.parametrize("precision,top_k", [(1, 8), (2, 32)])
def test_chunked_grid_low_precision(M, ctx, oracle_lib, ragged, precision, top_k):
    """BF16 / FP8 ranges with the FP32 re-score: the returned entry's CC is the
    oracle's CC of that entry, and agreement with the oracle's argmax is at
    least the resident search's."""
    g = ragged["grid"]
    res = _run_grid(M, ctx, ragged["h"], g, ragged["x"], precision, top_k, 2 * _row_entries(oracle_lib, g))
    t1, t2, df = S.grid_values(g)
    a, b, c = oracle_lib.grid_params(g)
    i = res["index"]
    dd = oracle_lib.simulate(ragged["seq"], t1[a[i]], t2[b[i]], df[c[i]])
    x = ragged["x"]
    occ = np.abs(np.sum(dd.conj() * x, 1)) / (np.linalg.norm(dd, axis=1) * np.linalg.norm(x, axis=1))
    assert np.abs(res["cc"] - occ).max() < CC_TOL
    ref = ragged["ref"]
    agree = (i == ref["idx"][:, 0]).mean()
    resident = (_run(M, ctx, ragged["dicts"][precision], x, precision, top_k, 1)["index"] == ref["idx"][:, 0]).mean()
    print(f"chunked precision={precision} k={top_k}: agreement {agree:.3f} (resident {resident:.3f})")
    assert agree >= resident - 1e-9


def test_chunked_grid_invalid_and_empty_calls(M, ctx, oracle_lib, ragged):
    import ctypes as C
    g = ragged["grid"]
    x = torch.from_numpy(np.ascontiguousarray(ragged["x"][:4].astype(np.complex64))).cuda()
    out = M.empty_results(4)
    L = M.lib()
    gd = M.grid_desc(g)
    opts = M.match_opts(M.MRF_F32, 4, 1)
    small = _row_entries(oracle_lib, g) - 1
    for chunk in (-1, small):
        rc = L.mrf_match_bruteforce_grid(ctx, ragged["h"], C.byref(gd), C.byref(opts), chunk,
                                         C.c_void_p(x.data_ptr()), 4, C.c_void_p(out.data_ptr()), None)
        assert rc == M.MRF_E_INVALID, chunk
    bad = M.match_opts(M.MRF_F32, 3, 1)
    rc = L.mrf_match_bruteforce_grid(ctx, ragged["h"], C.byref(gd), C.byref(bad), 0, C.c_void_p(x.data_ptr()), 4,
                                     C.c_void_p(out.data_ptr()), None)
    assert rc == M.MRF_E_INVALID
    rc = L.mrf_match_bruteforce_grid(ctx, ragged["h"], C.byref(gd), C.byref(opts), 0, None, 0, None, None)
    assert rc == M.MRF_OK
    # a voxel of zeros matches nothing, in every range
    z = np.zeros((2, ragged["seq"].n), np.complex64)
    res = _run_grid(M, ctx, ragged["h"], g, z, M.MRF_F32, 4, 2 * _row_entries(oracle_lib, g))
    assert (res["index"] == -1).all()
