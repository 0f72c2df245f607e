"""Shared test inputs: seeded phantoms whose clean signals come from the FP64 oracle."""
import numpy as np

import mrf_synth as S


def ongrid_voxels(orc, seq, grid, v, snr, seed):
    """Voxels on random valid grid points (M0, phase, noise from mrf_synth)."""
    ph = S.phantom_ongrid(seed, v, grid)
    clean = orc.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    g_re, g_im = S.noise_draws(seed, v, seq.n)
    return ph, S.compose_voxels(clean, ph["m0"], ph["phase"], g_re, g_im, snr)


def offgrid_voxels(orc, seq, v, snr, seed, **ranges):
    """Off-grid voxels: log-uniform T1/T2 (T2 < T1), uniform df (mrf_synth recipe)."""
    ph = S.phantom_offgrid(seed, v, **ranges)
    clean = orc.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    g_re, g_im = S.noise_draws(seed, v, seq.n)
    return ph, S.compose_voxels(clean, ph["m0"], ph["phase"], g_re, g_im, snr)


def rel_l2(a, b, axis=-1):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b, axis=axis) / np.linalg.norm(b, axis=axis)


# Relative L2 bound on a stored MRF_F32 dictionary row against the FP64
# oracle: each value is held as fp16 plus an e4m3 copy of the fp16 residual
# (residual <= 2^-11 of the value, e4m3 unit roundoff 2^-4), i.e. to at most
# 2^-15 relative, on top of the FP32 simulation's 1e-5.
F32_STORE_TOL = 2.0 ** -15 + 1e-5
