"""The bounds-checked build (MRF_BUILD_VARIANT=check compiles the library with
-DMRF_CHECK into its own folder): dictionary generation (both kernels, every
dtype, row padding past N), brute force in every precision, the chunked brute
force, ZOOM, refinement and smoothing run with every device index check on,
leave the context's error flag clear (mrf_stream_sync raises otherwise), and
return the same bits as the normal build."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, math, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import paper_1506_05393_gb300 as M
import mrf_synth as S


class View:
    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def dev_bytes(ptr, nbytes):
    return torch.as_tensor(View(ptr, nbytes), device="cuda").cpu().numpy().tobytes()


h = hashlib.sha1()
ctx = M.mrf_ctx_create(0, 0)
g = S.Grid(100.0, 100.0, 20, 20.0, 20.0, 10, -20.0, 5.0, 9)
base = S.sequence(3, 201)
rng = np.random.default_rng(91)
seqs = [base, S.Sequence(base.flip_rad, rng.uniform(0, 2 * math.pi, 201), base.tr_ms, base.tr_ms * 0.3, 1, 15.0)]
for seq in seqs:
    sh = M.mrf_sequence_load(ctx, seq)
    # voxels: GPU-simulated fingerprints at off-grid parameters plus noise
    ph = S.phantom_offgrid(7, 70, t1_range=(150.0, 1900.0), t2_range=(25.0, 190.0), df_range=(-18.0, 18.0))
    T = [torch.tensor(np.asarray(ph[k], np.float32)).cuda() for k in ("t1", "t2", "df")]
    clean = torch.empty((70, seq.n), dtype=torch.complex64, device="cuda")
    M.mrf_simulate(ctx, sh, T[0], T[1], T[2], clean)
    M.mrf_stream_sync(ctx)
    gr, gi = S.noise_draws(7, 70, seq.n)
    x = S.compose_voxels(clean.cpu().numpy().astype(np.complex128), ph["m0"], ph["phase"], gr, gi, 25.0)
    fp = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    h.update(clean.cpu().numpy().tobytes())
    for dt, k in ((M.MRF_F32, 4), (M.MRF_BF16, 8), (M.MRF_FP8E4M3, 32)):
        d = M.mrf_dict_generate(ctx, sh, g, dt)
        M.mrf_stream_sync(ctx)
        info = M.mrf_dict_query(d)
        eb = 1 if dt == M.MRF_FP8E4M3 else 2
        h.update(dev_bytes(info.hi_dev, info.entries * info.ld * eb))
        if info.lo_dev:
            h.update(dev_bytes(info.lo_dev, info.entries * info.ld * eb))
        h.update(dev_bytes(info.norm_dev, 4 * info.entries) + dev_bytes(info.scale_dev, 4 * info.entries))
        out = M.empty_results(70)
        M.mrf_match_bruteforce(ctx, d, fp, M.match_opts(dt, k, 1), out)
        M.mrf_stream_sync(ctx)
        h.update(out.cpu().numpy().tobytes())
        M.mrf_refine(ctx, sh, g, fp, out)
        M.mrf_stream_sync(ctx)
        h.update(out.cpu().numpy().tobytes())
        if dt != M.MRF_FP8E4M3:
            M.mrf_zoom_search_dict(ctx, d, M.zoom_opts(), fp, out)
            M.mrf_stream_sync(ctx)
            h.update(out.cpu().numpy().tobytes())
        M.mrf_dict_free(ctx, d)
        M.mrf_match_bruteforce_grid(ctx, sh, g, fp, M.match_opts(dt, k, 1), out, 300)
        M.mrf_stream_sync(ctx)
        h.update(out.cpu().numpy().tobytes())
    out = M.empty_results(70)
    M.mrf_zoom_search(ctx, sh, g, M.zoom_opts(), fp, out)
    M.mrf_stream_sync(ctx)
    h.update(out.cpu().numpy().tobytes())
    sm = torch.empty_like(fp)
    M.mrf_smooth(ctx, fp, sm, 3, 1.0)
    M.mrf_stream_sync(ctx)
    h.update(sm.cpu().numpy().tobytes())
    M.mrf_sequence_free(ctx, sh)
M.mrf_ctx_destroy(ctx)
print("DIGEST", h.hexdigest())
"""


def _digest(variant):
    env = dict(os.environ, MRF_BUILD_VARIANT=variant)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + SCRIPT], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, f"variant {variant!r}:\n{r.stdout[-2000:]}\n{r.stderr[-4000:]}"
    line = [l for l in r.stdout.splitlines() if l.startswith("DIGEST ")]
    assert line, r.stdout[-2000:]
    return line[-1].split()[1]


def test_bounds_checked_build_runs_clean_and_returns_the_same_bits():
    checked = _digest("check")
    plain = _digest("")
    assert checked == plain
