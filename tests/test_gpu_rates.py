"""The measured rooflines the benchmark divides by: the FP32 FMA rate
(mrf_fp32_fma_rate) and the dense tensor-core rate of the matcher's MMA
shape (mrf_mma_rate), whose e4m3 form issues twice the bf16 flops per MMA."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu


def test_mma_rates(M, ctx):
    bf16 = M.mrf_mma_rate(ctx, M.MRF_BF16)
    fp8 = M.mrf_mma_rate(ctx, M.MRF_FP8E4M3)
    assert 500.0 < bf16 < 5000.0
    assert 1.6 < fp8 / bf16 < 2.4
    M.mrf_stream_sync(ctx)   # no wait timed out
    t = C.c_double()
    assert M.lib().mrf_mma_rate(ctx, M.MRF_F32, C.byref(t)) == M.MRF_E_INVALID


def test_fp32_fma_rate(M, ctx):
    assert 20.0 < M.mrf_fp32_fma_rate(ctx) < 200.0
