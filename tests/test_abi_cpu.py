"""C-ABI library checks that need no GPU: it builds, loads, exports every
symbol include/mrf.h declares, and its host-side grid logic agrees with the
oracle. No compute call is made."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import mrf_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(mrf_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def M():
    import paper_1506_05393_gb300 as M
    M.lib()
    return M


def test_library_exports_every_declared_symbol(M):
    path = M.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mrf_[a-z0-9_]+)", out))
    declared = set(_declared_functions())
    assert declared, "no declarations parsed"
    assert declared <= exported, f"missing: {sorted(declared - exported)}"
    assert set(M.EXPORTS) <= declared


def test_version(M):
    assert "sm_103a" in M.mrf_version()


@pytest.mark.parametrize("name", list(S.GRIDS))
def test_grid_count_matches_oracle(M, oracle_lib, name):
    assert M.mrf_grid_count(S.GRIDS[name]) == oracle_lib.grid_count(S.GRIDS[name])


def test_grid_unravel_matches_oracle(M, oracle_lib):
    g = S.Grid(100.0, 50.0, 9, 40.0, 30.0, 7, -5.0, 2.5, 5)
    a, b, c = oracle_lib.grid_params(g)
    for i in range(0, a.shape[0], 5):
        assert M.mrf_grid_unravel(g, i) == (a[i], b[i], c[i])
    with pytest.raises(M.MrfError):
        M.mrf_grid_unravel(g, a.shape[0])


def test_invalid_grids_rejected(M):
    bad = [S.Grid(100.0, 0.0, 5, 10.0, 5.0, 3, 0.0, 1.0, 1),
           S.Grid(100.0, 10.0, 0, 10.0, 5.0, 3, 0.0, 1.0, 1),
           S.Grid(-1.0, 10.0, 5, 10.0, 5.0, 3, 0.0, 1.0, 1),
           S.Grid(100.0, 10.0, 5, 10.0, 5.0, 3, 0.0, 1.0, 1, 2)]
    for g in bad:
        assert M.lib().mrf_grid_count(C.byref(M.grid_desc(g))) == M.MRF_E_INVALID


def test_zoom_opts_default_is_experiment_2(M):
    o = M.mrf_zoom_opts_default()
    assert o.t1_init_ms == 1000.0 and o.t2_init_ms == 100.0
    assert o.n_s2 == 2 and list(o.s2_t1_ms[:2]) == [200.0, 100.0]
    assert o.n_s4 == 8
    assert list(o.s4_param[:8]) == [0, 1, 0, 0, 0, 1, 1, 1]
    assert list(o.s4_ms[:8]) == [100.0, 100.0, 50.0, 20.0, 10.0, 50.0, 20.0, 10.0]
    assert abs(o.s1a_step_frac - 6 / 7) < 1e-15 and o.s1b_step_frac == 0.05 and o.s3_half_frac == 0.5


def test_no_device_fails_loudly(M):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(M.MrfError):
        M.mrf_ctx_create(0)


def test_null_arguments_rejected(M):
    L = M.lib()
    assert L.mrf_sequence_load(None, None, None) == M.MRF_E_INVALID
    assert L.mrf_match_bruteforce(None, None, None, 0, None, None, None) == M.MRF_E_INVALID
    assert L.mrf_zoom_search(None, None, None, None, None, 0, None, None) == M.MRF_E_INVALID
    assert "NULL" in M.last_error()
    assert L.mrf_match_bruteforce_grid(None, None, None, None, 0, None, 0, None, None) == M.MRF_E_INVALID
    assert "NULL" in M.last_error()


def test_result_struct_layout(M):
    assert M.RESULT_DTYPE.itemsize == 56
    assert M.RESULT_DTYPE.fields["index"][1] == 0
    assert M.RESULT_DTYPE.fields["min_margin"][1] == 48


def test_bounds_checked_variant_compiles_and_is_kept_apart(tmp_path):
    """The bounds-checked variant (MRF_BUILD_VARIANT=check) builds into its own
    folder, and the translation units with device index checks compile with
    -DMRF_CHECK for sm_103a (nvcc cross-compiles without a GPU)."""
    code = ("import paper_1506_05393_gb300._build as b; print(b.VARIANT, b.LIB)")
    env = dict(os.environ, MRF_BUILD_VARIANT="check")
    out = subprocess.run(["python", "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, check=True)
    variant, lib = out.stdout.split()
    assert variant == "check" and os.path.basename(os.path.dirname(lib)) == "_build_check"
    bad = subprocess.run(["python", "-c", code], env=dict(os.environ, MRF_BUILD_VARIANT="fast"), cwd=ROOT,
                         capture_output=True, text=True)
    assert bad.returncode != 0 and "MRF_BUILD_VARIANT" in bad.stderr
    from paper_1506_05393_gb300 import _build
    csrc = os.path.join(ROOT, "paper_1506_05393_gb300", "csrc")
    for name in ("bloch.cu", "match.cu"):
        r = subprocess.run([_build._nvcc(), *_build.ARCH, "-O1", "-std=c++17", "--expt-relaxed-constexpr",
                            "-DMRF_CHECK", "-I", os.path.join(ROOT, "include"), "-c", os.path.join(csrc, name),
                            "-o", str(tmp_path / (name + ".o"))], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
