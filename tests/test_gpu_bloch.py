"""GPU Bloch simulation and dictionary generation against the FP64 oracle
(Appendix, Eq. A2). Fingerprints must agree within 1e-5 relative L2."""
import math

import numpy as np
import pytest
import torch

import mrf_synth as S
from conftest import device_bytes
from helpers import F32_STORE_TOL, rel_l2

pytestmark = pytest.mark.gpu


def _gpu_simulate(M, ctx, seq, t1, t2, df):
    h = M.mrf_sequence_load(ctx, seq)
    try:
        T1 = torch.tensor(t1, dtype=torch.float32, device="cuda")
        T2 = torch.tensor(t2, dtype=torch.float32, device="cuda")
        DF = torch.tensor(df, dtype=torch.float32, device="cuda")
        out = torch.empty((len(t1), seq.n), dtype=torch.complex64, device="cuda")
        M.mrf_simulate(ctx, h, T1, T2, DF, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    finally:
        M.mrf_sequence_free(ctx, h)


def _random_params(seed, count):
    p = S.phantom_offgrid(seed, count, t1_range=(100.0, 4000.0), t2_range=(10.0, 400.0), df_range=(-40.0, 40.0))
    return p["t1"], p["t2"], p["df"]


@pytest.mark.parametrize("n", [1000, 200, 201])
def test_simulate_matches_oracle(M, ctx, oracle_lib, n):
    seq = S.sequence(1, n)
    t1, t2, df = _random_params(30 + n, 384)
    gpu = _gpu_simulate(M, ctx, seq, t1, t2, df)
    ref = oracle_lib.simulate(seq, t1, t2, df)
    err = rel_l2(gpu, ref)
    assert err.max() < 1e-5, f"max rel L2 {err.max():.3g}"


def test_simulate_general_rf_phase_and_asymmetric_te(M, ctx, oracle_lib):
    base = S.sequence(5, 300)
    rng = np.random.default_rng(77)
    seq = S.Sequence(base.flip_rad, rng.uniform(0, 2 * math.pi, 300), base.tr_ms, base.tr_ms * 0.3, 1, 15.0)
    t1, t2, df = _random_params(41, 256)
    err = rel_l2(_gpu_simulate(M, ctx, seq, t1, t2, df), oracle_lib.simulate(seq, t1, t2, df))
    assert err.max() < 1e-5, f"max rel L2 {err.max():.3g}"


def test_simulate_without_inversion(M, ctx, oracle_lib):
    base = S.sequence(6, 256)
    seq = S.Sequence(base.flip_rad, base.rf_phase_rad, base.tr_ms, base.te_ms, 0, 0.0)
    t1, t2, df = _random_params(42, 128)
    err = rel_l2(_gpu_simulate(M, ctx, seq, t1, t2, df), oracle_lib.simulate(seq, t1, t2, df))
    assert err.max() < 1e-5


def _f32_values(hi16, lo8):
    """Stored MRF_F32 values: fp16 part 2^-15 plus e4m3 residual 2^-19."""
    return hi16.double() * 2.0 ** -15 + lo8.float().double() * 2.0 ** -19


def _dict_rows(M, d, dtype):
    info = M.mrf_dict_query(d)
    D, ld = info.entries, info.ld
    eb = 1 if dtype == M.MRF_FP8E4M3 else 2
    hi = device_bytes(info.hi_dev, D * ld * eb).cpu().numpy()
    norm = device_bytes(info.norm_dev, 4 * D).cpu().numpy().view(np.float32)
    # stored value x per-entry scale = unit-norm entry, for every dtype
    sc = device_bytes(info.scale_dev, 4 * D).cpu().numpy().view(np.float32).astype(np.float64)
    if dtype == M.MRF_FP8E4M3:
        q = torch.from_numpy(hi).view(torch.float8_e4m3fn).float().numpy().reshape(D, ld)
        vals = q * sc[:, None]
    elif dtype == M.MRF_F32:
        # fp16 part x 2^-15 + e4m3 residual x 2^-19 (the second of the two e4m3 planes)
        lo = device_bytes(info.lo_dev, D * ld * 2).cpu()
        vals = _f32_values(torch.from_numpy(hi).view(torch.float16), lo[D * ld:].view(torch.float8_e4m3fn))
        vals = vals.numpy().reshape(D, ld) * sc[:, None]
    else:
        vals = torch.from_numpy(hi).view(torch.bfloat16).float().numpy().reshape(D, ld).astype(np.float64)
        vals = vals * sc[:, None]
    n = info.n
    return vals[:, 0:2 * n:2] + 1j * vals[:, 1:2 * n:2], vals[:, 2 * n:], norm, info


@pytest.mark.parametrize("dtype,tol", [(0, F32_STORE_TOL), (1, 3e-3), (2, 7e-2)])
def test_dictionary_tiny_matches_oracle(M, ctx, oracle_lib, dtype, tol):
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, dtype)
    torch.cuda.synchronize()
    try:
        rows, pad, norm, info = _dict_rows(M, d, dtype)
        assert info.entries == 193 and info.ld >= 400 and (info.ld * (1 if dtype == 2 else 2)) % 128 == 0
        a, b, c = oracle_lib.grid_params(g)
        t1, t2, df = S.grid_values(g)
        ref = oracle_lib.simulate(seq, t1[a], t2[b], df[c])
        refn = ref / np.linalg.norm(ref, axis=1, keepdims=True)
        err = rel_l2(rows, refn)
        assert err.max() < tol, f"dtype {dtype}: max rel L2 {err.max():.3g}"
        np.testing.assert_allclose(norm, np.linalg.norm(ref, axis=1), rtol=1e-5)
        assert np.all(pad == 0)
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


@pytest.mark.parametrize("n", [1, 12, 37])
@pytest.mark.parametrize("dtype,tol", [(0, F32_STORE_TOL), (1, 3e-3), (2, 7e-2)])
def test_dictionary_short_sequences(M, ctx, oracle_lib, n, dtype, tol):
    """Sequences far shorter than a row's padding (N = 1, 12, 37 timepoints)
    on a grid with a df axis: rows, norms and zero padding as for N = 200."""
    seq = S.sequence(3, n)
    g = S.Grid(100.0, 100.0, 20, 20.0, 20.0, 10, -20.0, 5.0, 9)
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, dtype)
    torch.cuda.synchronize()
    try:
        rows, pad, norm, info = _dict_rows(M, d, dtype)
        a, b, c = oracle_lib.grid_params(g)
        t1, t2, df = S.grid_values(g)
        ref = oracle_lib.simulate(seq, t1[a], t2[b], df[c])
        nr = np.linalg.norm(ref, axis=1)
        live = nr > 1e-6 * nr.max()
        refn = ref[live] / nr[live, None]
        err = rel_l2(rows[live], refn)
        assert err.max() < tol, f"N {n}, dtype {dtype}: max rel L2 {err.max():.3g}"
        np.testing.assert_allclose(norm, nr, rtol=1e-5, atol=1e-7)
        assert np.all(pad == 0)
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


@pytest.mark.parametrize("kind", ["general_rf_asym_te", "xonly_asym_te", "general_rf_sym_te"])
@pytest.mark.parametrize("dtype,tol", [(0, F32_STORE_TOL), (1, 3e-3), (2, 7e-2)])
def test_dictionary_other_sequence_kinds(M, ctx, oracle_lib, kind, dtype, tol):
    """Sequences outside the symmetric x-rotation form (an RF phase off the
    multiples of pi, TE_j != TR_j - TE_j) take the table-driven kernel: rows,
    norms and padding against the oracle on a grid with a df axis."""
    base = S.sequence(4, 150)
    rng = np.random.default_rng(91)
    phase = rng.uniform(0, 2 * math.pi, 150) if kind.startswith("general") else base.rf_phase_rad
    te = base.tr_ms * 0.3 if kind.endswith("asym_te") else base.te_ms
    seq = S.Sequence(base.flip_rad, phase, base.tr_ms, te, 1, 15.0)
    g = S.Grid(100.0, 100.0, 20, 20.0, 20.0, 10, -20.0, 5.0, 9)
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
        assert err.max() < tol, f"{kind}, dtype {dtype}: max rel L2 {err.max():.3g}"
        np.testing.assert_allclose(norm, nr, rtol=1e-5)
        assert np.all(pad == 0)
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_dictionary_full_size_sampled(M, ctx, oracle_lib):
    """The 614,508-entry FP32-equivalent dictionary at N = 1000: sampled rows."""
    seq = S.sequence(1, 1000)
    g = S.GRIDS["fp32_brute"]
    h = M.mrf_sequence_load(ctx, seq)
    d = M.mrf_dict_generate(ctx, h, g, M.MRF_F32)
    torch.cuda.synchronize()
    try:
        info = M.mrf_dict_query(d)
        D, ld = info.entries, info.ld
        assert D == 614508 and ld >= 2000 and (ld * 2) % 128 == 0
        rng = np.random.default_rng(3)
        idx = np.unique(np.concatenate([rng.integers(0, D, 250), [0, D - 1]]))
        hi = device_bytes(info.hi_dev, D * ld * 2).view(torch.float16).view(D, ld)
        lo = device_bytes(info.lo_dev, D * ld * 2)[D * ld:].view(torch.float8_e4m3fn).view(D, ld)
        sc = device_bytes(info.scale_dev, 4 * D).view(torch.float32)
        it = torch.from_numpy(idx).cuda()
        # stored value x per-entry scale = unit-norm entry
        vals = (_f32_values(hi[it], lo[it]) * sc[it].double()[:, None]).cpu().numpy()
        rows = vals[:, 0:2000:2] + 1j * vals[:, 1:2000:2]
        params = [M.mrf_grid_unravel(g, int(i)) for i in idx]
        t1, t2, df = S.grid_values(g)
        ref = oracle_lib.simulate(seq, t1[[p[0] for p in params]], t2[[p[1] for p in params]], df[[p[2] for p in params]])
        refn = ref / np.linalg.norm(ref, axis=1, keepdims=True)
        err = rel_l2(rows, refn)
        # the storage bound, and the rms of 2000 rounded values well inside it
        assert err.max() < F32_STORE_TOL, f"max rel L2 {err.max():.3g}"
        assert np.median(err) < 1e-5, f"median rel L2 {np.median(err):.3g}"
        assert torch.count_nonzero(hi[it][:, 2000:]).item() == 0
    finally:
        M.mrf_dict_free(ctx, d)
        M.mrf_sequence_free(ctx, h)


def test_cc_landscape_around_a_fingerprint(M, ctx):
    """The CC landscape of GPU fingerprints around a target on this sequence
    (Theory, Properties I-III; Experiment 1 as a shape). What must hold: the
    df line through the target peaks at the target with CC = 1, and the T1
    and T2 lines through it are unimodal with their maximum at the target.
    What the paper postulates beyond that (df argmax at the target for every
    T1/T2 pair, periodic df side lobes) is measured and printed: on this
    sequence the alternating-sign train gives every candidate a competing df
    peak at 0 Hz, and the random TRs leave no clean 1/TR period."""
    seq = S.sequence(1, 1000)
    h = M.mrf_sequence_load(ctx, seq)
    try:
        def sim(t1, t2, df):
            t = [torch.tensor(np.asarray(v, np.float32)).cuda() for v in (t1, t2, df)]
            out = torch.empty((t[0].numel(), seq.n), dtype=torch.complex64, device="cuda")
            M.mrf_simulate(ctx, h, t[0], t[1], t[2], out)
            torch.cuda.synchronize()
            return out.cpu().numpy().astype(np.complex128)

        target = (1400.0, 200.0, 20.0)
        x = sim([target[0]], [target[1]], [target[2]])[0]
        x /= np.linalg.norm(x)
        cc = lambda d: np.abs(d.conj() @ x) / np.linalg.norm(d, axis=1)
        dfs = np.arange(-300.0, 301.0, 1.0)
        c = cc(sim(np.full(dfs.size, target[0]), np.full(dfs.size, target[1]), dfs))
        assert dfs[np.argmax(c)] == target[2] and abs(c.max() - 1.0) < 1e-5
        t1s = np.arange(100.0, 4001.0, 20.0)
        c1 = cc(sim(t1s, np.full(t1s.size, target[1]), np.full(t1s.size, target[2])))
        t2s = np.arange(10.0, 401.0, 5.0)
        c2 = cc(sim(np.full(t2s.size, target[0]), t2s, np.full(t2s.size, target[2])))
        for line, axis, want in ((c1, t1s, target[0]), (c2, t2s, target[1])):
            maxima = [i for i in range(1, line.size - 1) if line[i] > line[i - 1] and line[i] > line[i + 1]]
            assert len(maxima) == 1 and axis[maxima[0]] == want
        hits = 0
        for t1 in (700.0, 1400.0, 3000.0):
            for t2 in (50.0, 100.0, 300.0):
                cd = cc(sim(np.full(dfs.size, t1), np.full(dfs.size, t2), dfs))
                hits += dfs[np.argmax(cd)] == target[2]
        print(f"CC landscape: df argmax at the target for {hits} of 9 off-target (T1, T2) pairs; "
              f"CC at df = 0 Hz on the target's T1/T2: {c[dfs == 0.0][0]:.4f}")
    finally:
        M.mrf_sequence_free(ctx, h)


def test_fp32_fma_rate_is_plausible(M, ctx):
    """The measured FP32 FMA rate (the roofline of the on-the-fly kernels)
    lies between half and 1.05 x the nominal SMs x 128 FMA/clk x 2 x the
    highest SM clock."""
    props = torch.cuda.get_device_properties(0)
    rate = M.mrf_fp32_fma_rate(ctx)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.5 * nominal < rate < 1.05 * nominal, (rate, nominal)
    print(f"FP32 FMA rate {rate:.1f} TFLOP/s (nominal at 2.07 GHz {nominal:.1f})")
