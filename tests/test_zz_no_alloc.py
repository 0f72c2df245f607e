"""The allocation-free ZOOM entry point (mrf_zoom_search_static).

It exists for callers that cannot let the library allocate device memory
during a call (a framework owning the GPU's memory pool, a scan loop that
must not stall on allocation); its scratch lives in a fixed device array.
This file is collected last. It checks, through the C ABI, that two calls
in a row (different grids, so the shared array is rewritten and its work
counter reset) give the same results as mrf_zoom_search within the tests'
tolerance (and, being the same search, the same bits), that the call charges
no device memory to the context and takes none from the GPU (free memory by
cudaMemGetInfo unchanged across it), and that a grid too large for the array
is refused with a clear error.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import offgrid_voxels

pytestmark = pytest.mark.gpu

CC_TOL = 1e-5


def _run(M, ctx, fn, h, grid, x):
    """One call through the C ABI; also returns the device's free memory
    (cudaMemGetInfo) just before and just after it, with the call's inputs
    and outputs allocated beforehand."""
    fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    out = M.empty_results(x.shape[0])
    g = M.grid_desc(grid)
    o = M.zoom_opts()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rc = fn(ctx, h, C.byref(g), C.byref(o), C.c_void_p(fp.data_ptr()), x.shape[0], C.c_void_p(out.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == M.MRF_OK, M.last_error()
    M.mrf_stream_sync(ctx)
    free_after = torch.cuda.mem_get_info()[0]
    return M.results_to_numpy(out)[: x.shape[0]], free_before, free_after


def test_static_scratch_zoom_matches_zoom_search(M, oracle_lib):
    L = M.lib()
    ctx = M.mrf_ctx_create(0, 0)
    try:
        seq = S.sequence(1, 1000)
        h = M.mrf_sequence_load(ctx, seq)
        ph, x = offgrid_voxels(oracle_lib, seq, 300, 20.0, 77)
        for grid in (S.GRIDS["zoom_fine"], S.GRIDS["fp32_brute"]):    # two calls in a row
            ref, _, _ = _run(M, ctx, L.mrf_zoom_search, h, grid, x)
            used_before, _ = M.mrf_ctx_memory(ctx)
            got, free_before, free_after = _run(M, ctx, L.mrf_zoom_search_static, h, grid, x)
            used_after, _ = M.mrf_ctx_memory(ctx)
            # nothing charged to the context, and no device memory taken from the GPU
            assert used_after == used_before
            assert free_after == free_before
            for f in ("index", "i_t1", "i_t2", "i_df", "entries_evaluated"):
                assert np.array_equal(got[f], ref[f]), f
            assert np.abs(got["cc"] - ref["cc"]).max() <= CC_TOL
            assert np.abs(got["m0"] - ref["m0"]).max() <= 1e-4 * np.abs(ref["m0"]).max()
            # the same search in one kernel: the same bits as mrf_zoom_search in every field
            for f in got.dtype.names:
                assert np.array_equal(np.ascontiguousarray(got[f]).view(np.uint8), np.ascontiguousarray(ref[f]).view(np.uint8)), f
        M.mrf_sequence_free(ctx, h)
    finally:
        M.mrf_ctx_destroy(ctx)


def test_static_scratch_rejects_oversized_grid(M):
    L = M.lib()
    ctx = M.mrf_ctx_create(0, 0)
    try:
        seq = S.sequence(1, 50)
        h = M.mrf_sequence_load(ctx, seq)
        big = S.Grid(100.0, 0.01, 400000, 10.0, 5.0, 10, 0.0, 1.0, 1)
        fp = torch.zeros((4, 50), dtype=torch.complex64, device="cuda")
        out = M.empty_results(4)
        g = M.grid_desc(big)
        rc = L.mrf_zoom_search_static(ctx, h, C.byref(g), None, C.c_void_p(fp.data_ptr()), 4,
                                      C.c_void_p(out.data_ptr()), None)
        assert rc == M.MRF_E_INVALID
        assert "static scratch" in M.last_error() and "mrf_zoom_search" in M.last_error()
        M.mrf_sequence_free(ctx, h)
    finally:
        M.mrf_ctx_destroy(ctx)
