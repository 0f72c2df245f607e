"""GPU temporal smoothing (Methods, Experiment 4) against the FP64 oracle:
mrf_smooth on fingerprints, mrf_dict_smooth on a generated dictionary (entries
within the MRF_F32 storage bound, 2^-15 + 1e-5 relative L2), and brute force with
both sides smoothed (indices identical except where the oracle's top-two gap
is below 1e-6; CC within 1e-5)."""
import ctypes as C

import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import F32_STORE_TOL, offgrid_voxels, rel_l2
from test_gpu_bloch import _dict_rows

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("width,sigma", [(1, 1.0), (3, 1.0), (5, 1.0), (5, 0.7)])
def test_smooth_fingerprints(M, ctx, oracle_lib, width, sigma):
    rng = np.random.default_rng(width * 10 + int(sigma * 10))
    x = (rng.normal(size=(37, 203)) + 1j * rng.normal(size=(37, 203))).astype(np.complex64)
    xin = torch.from_numpy(x).cuda()
    xout = torch.empty_like(xin)
    M.mrf_smooth(ctx, xin, xout, width, sigma)
    torch.cuda.synchronize()
    ref = oracle_lib.smooth(x.astype(np.complex128), width, sigma)
    assert np.abs(xout.cpu().numpy() - ref).max() < 2e-6


@pytest.mark.parametrize("dtype,width,tol", [(0, 3, F32_STORE_TOL), (0, 5, F32_STORE_TOL), (1, 3, 4e-3)])
def test_dictionary_smoothing_matches_oracle(M, ctx, oracle_lib, dtype, width, tol):
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, dtype)
    try:
        M.mrf_dict_smooth(ctx, d, width, 1.0)
        torch.cuda.synchronize()
        rows, pad, norm, info = _dict_rows(M, d, dtype)
        assert info.smooth_width == width and info.smooth_sigma == 1.0
        a, b, c = oracle_lib.grid_params(g)
        t1, t2, df = S.grid_values(g)
        raw = oracle_lib.simulate(seq, t1[a], t2[b], df[c])
        sm = oracle_lib.smooth(raw, width, 1.0)
        refn = sm / np.linalg.norm(sm, axis=1, keepdims=True)
        assert rel_l2(rows, refn).max() < tol
        assert np.abs(pad).max() == 0.0
        np.testing.assert_allclose(norm, np.linalg.norm(sm, axis=1), rtol=max(tol, 1e-5))
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


@pytest.mark.parametrize("width", [3, 5])
def test_bruteforce_with_both_sides_smoothed(M, ctx, oracle_lib, width):
    seq = S.sequence(2, 200)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    ph, x = offgrid_voxels(oracle_lib, seq, 90, 15.0, 77, t1_range=(200.0, 1700.0), t2_range=(15.0, 300.0),
                           df_range=(-11.0, 11.0))
    xs_ref = oracle_lib.smooth(x, width, 1.0)
    ref = oracle_lib.bruteforce(seq, g, xs_ref, k=2, smooth=(width, 1.0))
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
    try:
        M.mrf_dict_smooth(ctx, d, width, 1.0)
        xin = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
        xs = torch.empty_like(xin)
        M.mrf_smooth(ctx, xin, xs, width, 1.0)
        out = M.empty_results(x.shape[0])
        M.mrf_match_bruteforce(ctx, d, xs, M.match_opts(M.MRF_F32, 4, 1), out)
        M.mrf_stream_sync(ctx)
        res = M.results_to_numpy(out)[: x.shape[0]]
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)
    gap = ref["cc"][:, 0] - ref["cc"][:, 1]
    same = res["index"] == ref["idx"][:, 0]
    assert (same | (gap < 1e-6)).all()
    assert np.abs(res["cc"][same] - ref["cc"][same, 0]).max() < 1e-5
    np.testing.assert_allclose(res["m0"][same], ref["m0"][same], rtol=1e-4)
    plain = oracle_lib.bruteforce(seq, g, x, k=1)
    print(f"smoothing width {width}: index agreement {same.mean():.3f}; "
          f"differs from the unsmoothed match for {int((ref['idx'][:, 0] != plain['idx'][:, 0]).sum())} voxels")


def test_smoothing_rejects_bad_arguments(M, ctx):
    seq = S.sequence(0, 50)
    h = M.mrf_sequence_load(ctx, seq)
    d8 = M.mrf_dict_generate(ctx, h, S.GRIDS["tiny"], M.MRF_FP8E4M3)
    d32 = M.mrf_dict_generate(ctx, h, S.GRIDS["tiny"], M.MRF_F32)
    try:
        L = M.lib()
        assert L.mrf_dict_smooth(ctx, d8, 3, 1.0, None) == M.MRF_E_UNSUPPORTED
        assert L.mrf_dict_smooth(ctx, d32, 4, 1.0, None) == M.MRF_E_INVALID
        assert L.mrf_dict_smooth(ctx, d32, 3, 0.0, None) == M.MRF_E_INVALID
        assert L.mrf_dict_smooth(ctx, d32, 3, 1.0, None) == M.MRF_OK
        assert L.mrf_dict_smooth(ctx, d32, 3, 1.0, None) == M.MRF_E_INVALID      # already smoothed
        x = torch.zeros((2, 50), dtype=torch.complex64, device="cuda")
        p = C.c_void_p(x.data_ptr())
        assert L.mrf_smooth(ctx, p, p, 2, 50, 3, 1.0, None) == M.MRF_E_INVALID   # in place
        assert L.mrf_smooth(ctx, None, None, 0, 50, 3, 1.0, None) == M.MRF_OK
    finally:
        M.mrf_dict_free(ctx, d8)
        M.mrf_dict_free(ctx, d32)
        M.mrf_sequence_free(ctx, h)
