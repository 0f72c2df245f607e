"""Serving loop: continuous batching over resident dictionaries.

Each request's result must be identical whether it runs alone (direct
C-ABI call) or batched with others; admission respects the HBM budget;
cancellation, polling and oversized requests behave as documented."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

import mrf_synth as S
from helpers import offgrid_voxels

pytestmark = pytest.mark.gpu

FIELDS = ["index", "i_t1", "i_t2", "i_df", "cc", "m0", "phase", "entries_evaluated", "min_margin"]


def _request(M, mode, x, dict_h=None, opts=None, seq_h=None, grid=None, zoom=None):
    x = np.ascontiguousarray(x.astype(np.complex64))
    r = M.Request()
    r.mode = mode
    r.dict = dict_h.value if dict_h is not None else None
    if opts is not None:
        r.match = opts
    r.seq = seq_h.value if seq_h is not None else None
    keep = [x]
    if grid is not None:
        gd = M.grid_desc(grid)
        keep.append(gd)
        r.grid = C.pointer(gd)
    if zoom is not None:
        keep.append(zoom)
        r.zoom = C.pointer(zoom)
    r.fp_host = x.ctypes.data
    r.V = x.shape[0]
    return r, keep


def _alone(M, ctx, mode, x, dict_h=None, opts=None, seq_h=None, grid=None, zoom=None):
    fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    out = M.empty_results(x.shape[0])
    if mode == M.MRF_MODE_BRUTE:
        M.mrf_match_bruteforce(ctx, dict_h, fp, opts, out)
    else:
        M.mrf_zoom_search(ctx, seq_h, grid, zoom, fp, out)
    M.mrf_stream_sync(ctx)
    return M.results_to_numpy(out)[: x.shape[0]]


@pytest.fixture(scope="module")
def setup(M, oracle_lib):
    ctx = M.mrf_ctx_create(0, 0)
    seq = S.sequence(2, 200)
    g = S.Grid(150.0, 45.0, 37, 12.0, 9.0, 33, -12.0, 3.0, 9)
    h = M.mrf_sequence_load(ctx, seq)
    d32 = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
    d16 = M.mrf_dict_generate(ctx, h, g, M.MRF_BF16)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    xs = []
    for i, v in enumerate([16, 70, 256, 5, 130, 64, 33, 200]):
        ph, x = offgrid_voxels(oracle_lib, seq, v, 25.0, 300 + i, t1_range=(200.0, 1700.0),
                               t2_range=(15.0, 300.0), df_range=(-11.0, 11.0))
        xs.append(x)
    yield dict(ctx=ctx, seq=seq, grid=g, h=h, d32=d32, d16=d16, xs=xs)
    M.mrf_dict_free(ctx, d32)
    M.mrf_dict_free(ctx, d16)
    M.mrf_sequence_free(ctx, h)
    M.mrf_ctx_destroy(ctx)


def _specs(M, st):
    o32 = M.match_opts(M.MRF_F32, 4, 1)
    o16 = M.match_opts(M.MRF_BF16, 8, 1)
    zo = M.zoom_opts()
    specs = []
    for i, x in enumerate(st["xs"]):
        kind = i % 3
        if kind == 0:
            specs.append(dict(mode=M.MRF_MODE_BRUTE, x=x, dict_h=st["d32"], opts=o32))
        elif kind == 1:
            specs.append(dict(mode=M.MRF_MODE_BRUTE, x=x, dict_h=st["d16"], opts=o16))
        else:
            specs.append(dict(mode=M.MRF_MODE_ZOOM, x=x, seq_h=st["h"], grid=st["grid"], zoom=zo))
    return specs


def test_results_identical_alone_and_in_the_mix(M, setup):
    ctx = setup["ctx"]
    specs = _specs(M, setup)
    alone = [_alone(M, ctx, **sp) for sp in specs]
    M.mrf_serve_start(ctx, max_inflight=3, max_batch_voxels=400)
    try:
        tickets, keep = [], []
        for sp in specs + specs[::-1]:          # every request twice, mixed order
            r, k = _request(M, **sp)
            keep.append(k)
            tickets.append(M.mrf_serve_submit(ctx, r))
        outs = []
        for t, sp in zip(tickets, specs + specs[::-1]):
            o = np.zeros(sp["x"].shape[0], M.RESULT_DTYPE)
            M.mrf_serve_poll(ctx, t, 60000, o)
            outs.append(o)
        for o, a in zip(outs[: len(specs)] + outs[len(specs):][::-1], alone + alone):
            for f in FIELDS:
                assert np.array_equal(o[f], a[f]), f
        st = M.mrf_serve_get_stats(ctx)
        assert st.completed == 2 * len(specs) and st.queued_now == 0 and st.running_now == 0
        assert st.launches < 2 * len(specs)        # requests were batched together
    finally:
        M.mrf_serve_stop(ctx)


def test_budget_admission_and_rejection(M, oracle_lib, setup):
    """A context whose budget leaves room for about one batch at a time:
    requests wait for memory instead of failing; one that can never fit is
    rejected at submit."""
    seq, g = setup["seq"], setup["grid"]
    ctx = M.mrf_ctx_create(0, 0)
    try:
        h = M.mrf_sequence_load(ctx, seq)
        d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
        torch.cuda.synchronize()
        used, _ = M.mrf_ctx_memory(ctx)
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)
        M.mrf_ctx_destroy(ctx)
        # same objects in a budgeted context
        ctx = M.mrf_ctx_create(0, used + 4 * 1024 * 1024)
        h = M.mrf_sequence_load(ctx, seq)
        d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
        torch.cuda.synchronize()
        M.mrf_serve_start(ctx, max_inflight=4, max_batch_voxels=256)
        o32 = M.match_opts(M.MRF_F32, 4, 1)
        xs = setup["xs"]
        big = np.tile(xs[2], (200, 1))             # 51,200 voxels: cannot fit the budget
        r, keep = _request(M, M.MRF_MODE_BRUTE, big, dict_h=d, opts=o32)
        with pytest.raises(M.MrfError) as ei:
            M.mrf_serve_submit(ctx, r)
        assert ei.value.code == M.MRF_E_BUDGET
        tickets, keeps = [], []
        for x in xs:
            r, k = _request(M, M.MRF_MODE_BRUTE, x, dict_h=d, opts=o32)
            keeps.append(k)
            tickets.append(M.mrf_serve_submit(ctx, r))
        for t, x in zip(tickets, xs):
            o = np.zeros(x.shape[0], M.RESULT_DTYPE)
            M.mrf_serve_poll(ctx, t, 60000, o)
            a = _alone(M, ctx, M.MRF_MODE_BRUTE, x, dict_h=d, opts=o32)
            assert np.array_equal(o["index"], a["index"])
        st = M.mrf_serve_get_stats(ctx)
        assert st.rejected == 1 and st.completed == len(xs)
        u, b = M.mrf_ctx_memory(ctx)
        assert st.request_bytes_peak <= b
        M.mrf_serve_stop(ctx)
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)
    finally:
        M.mrf_ctx_destroy(ctx)


def test_poll_cancel_and_unknown_ticket(M, setup):
    ctx = setup["ctx"]
    M.mrf_serve_start(ctx, max_inflight=1, max_batch_voxels=64)
    try:
        sp = _specs(M, setup)[2]                  # a ZOOM request
        tickets, keep = [], []
        for _ in range(6):
            r, k = _request(M, **sp)
            keep.append(k)
            tickets.append(M.mrf_serve_submit(ctx, r))
        last = tickets[-1]
        rc = M.mrf_serve_cancel(ctx, last)
        assert rc in (M.MRF_OK, M.MRF_E_NOTFOUND)
        o = np.zeros(sp["x"].shape[0], M.RESULT_DTYPE)
        if rc == M.MRF_OK:
            assert M.mrf_serve_poll_rc(ctx, last, 0, o) == M.MRF_E_NOTFOUND
        first = M.mrf_serve_poll_rc(ctx, tickets[0], 0, o)
        assert first in (M.MRF_OK, M.MRF_PENDING)
        for t in tickets[:-1]:
            rc2 = M.MRF_PENDING
            t0 = time.time()
            while rc2 == M.MRF_PENDING and time.time() - t0 < 60:
                rc2 = M.mrf_serve_poll_rc(ctx, t, 100, o)
                if rc2 == M.MRF_E_TIMEOUT:
                    rc2 = M.MRF_PENDING
            assert rc2 == M.MRF_OK or (t == tickets[0] and first == M.MRF_OK and rc2 == M.MRF_E_NOTFOUND)
        assert M.mrf_serve_poll_rc(ctx, 987654321, 0, o) == M.MRF_E_NOTFOUND
    finally:
        M.mrf_serve_stop(ctx)
