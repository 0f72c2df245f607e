"""Pins of the FP64 oracle against facts that do not come from the oracle.

Simulator (Appendix, Eq. A1/A2): closed forms for pure T1 recovery, pure T2
decay with precession, magnitude conservation, the textbook balanced-SSFP
steady state, exact df periodicity for a constant TR (Property II), and the
general RF-phase rotation against Rodrigues' formula.
CC (Eq. 1): a hand example, self-correlation, scale invariance, the bound.
Grid: closed-form entry counts.
Brute force: exact recovery of noise-free on-grid voxels (Experiment 2) and an
independent exhaustive top-k with noise.
ZOOM: a hand-derived trace on an analytic score (tests/golden), recovery of
on-grid voxels, local optimality, and equality with brute force when omega
equals the df resolution (Experiment 2).
"""
import math
import os

import numpy as np
import pytest

import mrf_synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _seq(n, flip, tr, te, inversion=0, delay=0.0, phase=None):
    flip = np.broadcast_to(np.asarray(flip, float), (n,)).copy()
    tr = np.broadcast_to(np.asarray(tr, float), (n,)).copy()
    te = np.broadcast_to(np.asarray(te, float), (n,)).copy()
    ph = np.zeros(n) if phase is None else np.broadcast_to(np.asarray(phase, float), (n,)).copy()
    return S.Sequence(flip, ph, tr, te, inversion, delay)


# ------------------------------------------------ finite RF pulses (Appendix)

def _bloch_pulse_rk4(m, alpha, phi, tau, df, steps=4000):
    """Integrate the rotating-frame Bloch equation (Eq. A1 without relaxation)
    over one RF pulse of duration tau ms: dM/dt = W x M with the RF field of
    phase phi turning M about (cos phi, sin phi, 0) by -alpha over tau (the
    hard-pulse sense), and off-resonance turning it counterclockwise about z
    at 2 pi df / 1000 rad/ms (the sense of R_off), both at once (RK4)."""
    w = np.array([-alpha / tau * math.cos(phi), -alpha / tau * math.sin(phi), 2.0 * math.pi * df / 1000.0])
    f = lambda v: np.cross(w, v)
    h = tau / steps
    v = np.array(m, float)
    for _ in range(steps):
        k1 = f(v)
        k2 = f(v + 0.5 * h * k1)
        k3 = f(v + 0.5 * h * k2)
        k4 = f(v + h * k3)
        v = v + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return v


def _one_pulse(oracle_lib, m, alpha, phi, tau, df):
    """The oracle's state right after one pulse: n = 1, TE = 0 (the free
    evolution before the sample is the identity), no inversion."""
    seq = S.with_pulses(_seq(1, alpha, 10.0, 0.0, phase=phi), tau)
    _, st = oracle_lib.simulate_state(seq, 1e9, 1e9, df, m_init=m)
    return st[0]


@pytest.mark.parametrize("alpha,phi,tau,df", [(0.7, 0.0, 1.0, 40.0), (-0.7, 0.0, 1.0, 40.0), (0.3, 1.2, 2.0, -25.0),
                                              (1.4, math.pi / 2, 0.5, 300.0), (0.0, 0.0, 1.5, 30.0),
                                              (-0.2, math.pi, 3.0, -400.0)])
def test_finite_pulse_against_the_bloch_equation(oracle_lib, alpha, phi, tau, df):
    """The Appendix's off-resonant RF rotation R_z(phi) R_y(beta) R_x(alpha')
    R_y(-beta) R_z(-phi) equals the Bloch equation integrated through the
    pulse with the RF and off-resonance fields together (signed flip angles,
    alpha = 0, far off resonance), and keeps |M|."""
    rng = np.random.default_rng(int(1000 * abs(alpha) + abs(df)))
    m = rng.normal(size=3)
    m /= np.linalg.norm(m)
    got = _one_pulse(oracle_lib, m, alpha, phi, tau, df)
    want = _bloch_pulse_rk4(m, alpha, phi, tau, df)
    np.testing.assert_allclose(got, want, atol=1e-10)
    assert abs(np.linalg.norm(got) - 1.0) < 1e-13


def test_finite_pulse_without_rf_is_free_precession(oracle_lib):
    """alpha = 0: the pulse interval is precession alone, a counterclockwise
    z rotation by 2 pi df tau / 1000."""
    m = np.array([0.6, -0.3, 0.74])
    got = _one_pulse(oracle_lib, m, 0.0, 0.4, 2.5, 37.0)
    th = 2 * math.pi * 37.0 * 2.5 / 1000.0
    want = np.array([math.cos(th) * m[0] - math.sin(th) * m[1], math.sin(th) * m[0] + math.cos(th) * m[1], m[2]])
    np.testing.assert_allclose(got, want, atol=1e-15)


def test_finite_pulse_limits_are_the_hard_pulse(oracle_lib):
    """tau = 0 is the hard pulse exactly; tau -> 0 converges to it; on
    resonance (df = 0) the effective field lies along the RF axis, so any tau
    gives the hard pulse (alternating signs, 0/90/180 degree phases)."""
    base = S.sequence_paper(4, 120)
    alt = S.sequence(5, 120)
    for seq in (base, alt):
        hard = oracle_lib.simulate(seq, [900.0, 1500.0], [80.0, 40.0], [12.0, -30.0])
        zero = oracle_lib.simulate(S.with_pulses(seq, 0.0), [900.0, 1500.0], [80.0, 40.0], [12.0, -30.0])
        assert np.array_equal(hard, zero)
        tiny = oracle_lib.simulate(S.with_pulses(seq, 1e-9), [900.0, 1500.0], [80.0, 40.0], [12.0, -30.0])
        np.testing.assert_allclose(tiny, hard, atol=1e-9)
        on = oracle_lib.simulate(S.with_pulses(seq, 2.0), [900.0, 1500.0], [80.0, 40.0], [0.0, 0.0])
        np.testing.assert_allclose(on, oracle_lib.simulate(seq, [900.0, 1500.0], [80.0, 40.0], [0.0, 0.0]),
                                   atol=1e-13)
        off = oracle_lib.simulate(S.with_pulses(seq, 2.0), [900.0], [80.0], [30.0])
        assert np.abs(off - hard[:1]).max() > 1e-3          # a 2 ms pulse 30 Hz off resonance matters


# ----------------------------------------------------------------- simulator

def test_pure_t1_recovery_after_inversion(oracle_lib):
    """Zero flip angles after an ideal inversion: Mz(t) = 1 - 2 exp(-t/T1), no
    transverse signal, sampled TE_j after pulse j."""
    rng = np.random.default_rng(5)
    n = 60
    tr = rng.uniform(5, 15, n)
    te = tr * rng.uniform(0.1, 0.9, n)
    seq = _seq(n, 0.0, tr, te, inversion=1, delay=20.0)
    T1 = 837.0
    sig, st = oracle_lib.simulate_state(seq, T1, 95.0, 13.0)
    t = 20.0 + np.concatenate([[0.0], np.cumsum(tr)[:-1]]) + te
    np.testing.assert_allclose(st[:, 2], 1.0 - 2.0 * np.exp(-t / T1), rtol=0, atol=1e-13)
    assert np.max(np.abs(sig)) < 1e-15   # sin(pi) rounding only


def test_pure_t2_decay_and_precession(oracle_lib):
    """One pulse of +90 degrees from equilibrium, then zero flips: the hard
    pulse R_x(-alpha) puts M on +y, so s(t) = i exp(-t/T2) exp(+i 2 pi df t)
    (counterclockwise R_off), and Mz(t) = 1 - exp(-t/T1)."""
    rng = np.random.default_rng(6)
    n = 40
    tr = rng.uniform(8, 14, n)
    te = tr * rng.uniform(0.2, 0.8, n)
    flip = np.zeros(n)
    flip[0] = math.pi / 2
    seq = _seq(n, flip, tr, te)
    T1, T2, df = 1200.0, 80.0, 17.5
    sig, st = oracle_lib.simulate_state(seq, T1, T2, df)
    t = np.concatenate([[0.0], np.cumsum(tr)[:-1]]) + te   # time since the pulse
    expect = 1j * np.exp(-t / T2) * np.exp(1j * 2 * np.pi * df * t / 1000.0)
    np.testing.assert_allclose(sig, expect, rtol=0, atol=1e-13)
    np.testing.assert_allclose(st[:, 2], 1.0 - np.exp(-t / T1), rtol=0, atol=1e-13)


def test_magnitude_conserved_without_relaxation(oracle_lib):
    seq = S.sequence(3, 300)
    seq = S.Sequence(seq.flip_rad, np.random.default_rng(1).uniform(0, 2 * np.pi, 300),
                     seq.tr_ms, seq.te_ms, 1, 20.0)
    _, st = oracle_lib.simulate_state(seq, math.inf, math.inf, 23.7)
    np.testing.assert_allclose(np.linalg.norm(st, axis=1), 1.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("alpha_deg,T1,T2", [(30.0, 800.0, 60.0), (60.0, 1500.0, 200.0), (10.0, 300.0, 250.0)])
def test_bssfp_steady_state(oracle_lib, alpha_deg, T1, T2):
    """Alternating +-alpha, constant TR, TE = TR/2, on resonance: the signal
    magnitude converges to the textbook balanced-SSFP steady state
    sin(a)(1-E1)sqrt(E2) / (1 - (E1-E2)cos(a) - E1 E2)."""
    n, TR = 4000, 10.0
    a = math.radians(alpha_deg)
    flip = a * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    seq = _seq(n, flip, TR, TR / 2)
    sig, _ = oracle_lib.simulate_state(seq, T1, T2, 0.0)
    E1, E2 = math.exp(-TR / T1), math.exp(-TR / T2)
    ss = math.sin(a) * (1 - E1) * math.sqrt(E2) / (1 - (E1 - E2) * math.cos(a) - E1 * E2)
    np.testing.assert_allclose(np.abs(sig[-10:]), ss, rtol=1e-10)


def test_df_period_is_one_over_tr(oracle_lib):
    """Property II made exact: with a constant TR, df and df + 1000/TR Hz give
    fingerprints that differ by a constant phase, so CC = 1."""
    rng = np.random.default_rng(7)
    n, TR = 250, 12.5
    seq = _seq(n, rng.uniform(-1, 1, n), TR, TR / 2, inversion=1, delay=20.0)
    for df in (-30.0, 0.0, 12.3):
        s0 = oracle_lib.simulate(seq, 900.0, 70.0, df)[0]
        s1 = oracle_lib.simulate(seq, 900.0, 70.0, df + 1000.0 / TR)[0]
        assert abs(oracle_lib.cc(s0, s1) - 1.0) < 1e-12
        np.testing.assert_allclose(s1, -s0, atol=1e-12)  # TE = TR/2 -> phase pi
        s2 = oracle_lib.simulate(seq, 900.0, 70.0, df + 0.37 * 1000.0 / TR)[0]
        assert oracle_lib.cc(s0, s2) < 0.999


def test_rf_phase_is_rotation_about_tilted_axis(oracle_lib):
    """R_z(phi) R_x(-alpha) R_z(-phi) is a rotation by -alpha about the axis
    (cos phi, sin phi, 0): compare with Rodrigues' formula."""
    rng = np.random.default_rng(8)
    for _ in range(20):
        alpha, phi = rng.uniform(-3, 3), rng.uniform(-4, 4)
        m = rng.normal(size=3)
        seq = _seq(1, alpha, 0.0, 0.0, phase=phi)
        _, st = oracle_lib.simulate_state(seq, 1e3, 1e2, 0.0, m_init=m)
        k = np.array([math.cos(phi), math.sin(phi), 0.0])
        th = -alpha
        rod = (m * math.cos(th) + np.cross(k, m) * math.sin(th) + k * np.dot(k, m) * (1 - math.cos(th)))
        np.testing.assert_allclose(st[0], rod, atol=1e-13)


# ----------------------------------------------------------------- CC (Eq. 1)

def test_cc_hand_values(oracle_lib):
    assert oracle_lib.cc([1, 1j], [1, 1]) == pytest.approx(math.sqrt(2) / 2, abs=1e-15)
    assert oracle_lib.cc([1, 1], [1, -1]) == pytest.approx(0.0, abs=1e-15)
    assert oracle_lib.cc([1j, 0], [1, 0]) == pytest.approx(1.0, abs=1e-15)
    assert oracle_lib.cc([3 + 4j, 0], [0, 2]) == pytest.approx(0.0, abs=1e-15)


def test_cc_invariants(oracle_lib):
    rng = np.random.default_rng(9)
    for _ in range(10):
        x = rng.normal(size=64) + 1j * rng.normal(size=64)
        d = rng.normal(size=64) + 1j * rng.normal(size=64)
        assert oracle_lib.cc(x, x) == pytest.approx(1.0, abs=1e-14)
        c = complex(*rng.normal(size=2))
        assert oracle_lib.cc(c * x, d) == pytest.approx(oracle_lib.cc(x, d), abs=1e-14)
        assert 0.0 <= oracle_lib.cc(x, d) <= 1.0


# ----------------------------------------------------------------- grid

def _closed_form_count(g):
    t1, _, _ = S.grid_values(g)
    # number of T2 values strictly below T1: ceil((T1 - t2_min) / t2_step), clipped
    nb = np.clip(np.ceil((t1 - g.t2_min) / g.t2_step - 1e-9), 0, g.n_t2).astype(np.int64)
    return int(nb.sum()) * g.n_df


@pytest.mark.parametrize("name", list(S.GRIDS))
def test_grid_counts(oracle_lib, name):
    g = S.GRIDS[name]
    assert oracle_lib.grid_count(g) == _closed_form_count(g)


def test_grid_order_and_index(oracle_lib):
    g = S.GRIDS["tiny"]
    a, b, c = oracle_lib.grid_params(g)
    ea, eb, ec = S.grid_valid_params(g)
    assert (a == ea).all() and (b == eb).all() and (c == ec).all()
    g2 = S.Grid(100.0, 50.0, 7, 40.0, 30.0, 6, -5.0, 2.5, 5)
    a, b, c = oracle_lib.grid_params(g2)
    for i in range(0, a.shape[0], 7):
        assert oracle_lib.grid_index(g2, a[i], b[i], c[i]) == i
    assert oracle_lib.grid_index(g2, 0, 5, 0) == -1   # T2 = 190 >= T1 = 100


# ----------------------------------------------------------------- brute force

def _tiny_voxels(oracle_lib, v, snr, seed=100):
    g = S.GRIDS["tiny"]
    seq = S.sequence(0, 200)
    ph = S.phantom_ongrid(seed, v, g)
    clean = oracle_lib.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    g_re, g_im = S.noise_draws(seed, v, seq.n)
    x = S.compose_voxels(clean, ph["m0"], ph["phase"], g_re, g_im, snr)
    return seq, g, ph, x


def test_bruteforce_recovers_noise_free_on_grid(oracle_lib):
    """Experiment 2: targets on grid points are found exactly; CC = 1 and M0,
    phase are the applied scale (Theory: proton density from the scale)."""
    seq, g, ph, x = _tiny_voxels(oracle_lib, 64, None)
    r = oracle_lib.bruteforce(seq, g, x, k=2)
    assert (r["idx"][:, 0] == ph["index"]).all()
    np.testing.assert_allclose(r["cc"][:, 0], 1.0, atol=1e-12)
    assert (r["cc"][:, 1] < 1.0 - 1e-6).all()
    np.testing.assert_allclose(r["m0"], ph["m0"], rtol=1e-12)
    np.testing.assert_allclose(np.angle(np.exp(1j * (r["phase"] - ph["phase"]))), 0.0, atol=1e-12)


def test_bruteforce_topk_matches_exhaustive_numpy(oracle_lib):
    seq, g, ph, x = _tiny_voxels(oracle_lib, 32, 30.0)
    k = 5
    r = oracle_lib.bruteforce(seq, g, x, k=k)
    t1, t2, df = S.grid_values(g)
    a, b, c = S.grid_valid_params(g)
    D = oracle_lib.simulate(seq, t1[a], t2[b], df[c])
    ip = x @ D.conj().T
    cc = np.abs(ip) / (np.linalg.norm(x, axis=1)[:, None] * np.linalg.norm(D, axis=1)[None, :])
    order = np.lexsort((np.broadcast_to(np.arange(D.shape[0]), cc.shape), -cc), axis=1)[:, :k]
    assert (r["idx"] == order).all()
    np.testing.assert_allclose(r["cc"], np.take_along_axis(cc, order, 1), atol=1e-13)
    best = order[:, 0]
    m0 = np.abs(ip[np.arange(32), best]) / np.linalg.norm(D[best], axis=1) ** 2
    np.testing.assert_allclose(r["m0"], m0, rtol=1e-12)


# ----------------------------------------------------------------- ZOOM

def _read_trace():
    rows = []
    with open(os.path.join(GOLDEN, "zoom_quadratic_trace.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows, np.int32)


def test_zoom_hand_trace(oracle_lib):
    g = S.Grid(0.0, 1.0, 41, 0.0, 1.0, 41, 0.0, 1.0, 21, 0)
    f = lambda a, b, c: -(a - 27) ** 2 - 2 * (b - 13) ** 2 - 3 * (c - 11) ** 2
    o = oracle_lib.default_zoom_opts(t1_init_ms=20.0, t2_init_ms=20.0,
                                     s2=[(8.0, 8.0), (4.0, 4.0)],
                                     s4=[(0, 4.0), (1, 4.0), (0, 2.0), (0, 1.0), (1, 2.0), (1, 1.0)])
    r = oracle_lib.zoom_generic(g, f, 7.0, o)
    expect = _read_trace()
    assert r["trace"].shape == expect.shape
    assert (r["trace"] == expect).all()
    assert r["abc"] == (27, 13, 11) and r["cc"] == 0.0
    assert r["evaluated"] == 76 and r["min_margin"] == 0.0


def test_zoom_skips_invalid_points(oracle_lib):
    """Points with T2 >= T1 or outside the grid score -inf and are never evaluated."""
    g = S.Grid(0.0, 1.0, 30, 0.0, 1.0, 30, 0.0, 1.0, 5, 1)
    seen = []

    def f(a, b, c):
        seen.append((a, b, c))
        return -abs(a - 12) - abs(b - 11) - abs(c - 2)

    r = oracle_lib.zoom_generic(g, f, 3.0, oracle_lib.default_zoom_opts(t1_init_ms=5.0, t2_init_ms=9.0,
                                                                         s2=[(4.0, 4.0)], s4=[(0, 2.0), (1, 2.0)]))
    assert all(0 <= b < a < 30 and 0 <= c < 5 for a, b, c in seen)
    assert r["abc"] == (12, 11, 2)
    assert r["evaluated"] == len(seen)


def test_zoom_recovers_noise_free_on_grid(oracle_lib):
    seq, g, ph, x = _tiny_voxels(oracle_lib, 64, None)
    z = oracle_lib.zoom(seq, g, x)
    assert (z["abc"][:, 0] == ph["a"]).all() and (z["abc"][:, 1] == ph["b"]).all()
    np.testing.assert_allclose(z["cc"], 1.0, atol=1e-12)
    np.testing.assert_allclose(z["m0"], ph["m0"], rtol=1e-12)


def test_zoom_final_point_is_local_optimum(oracle_lib):
    """Local-optimality certificate at the finest step, checked with Eq. 1
    evaluated directly (not through the ZOOM code)."""
    seq = S.sequence(1, 300)
    g = S.Grid(300.0, 20.0, 60, 20.0, 5.0, 50, -20.0, 1.0, 41)
    p = S.phantom_offgrid(11, 12, t1_range=(400, 1400), t2_range=(30, 200), df_range=(-15, 15))
    clean = oracle_lib.simulate(seq, p["t1"], p["t2"], p["df"])
    x = S.compose_voxels(clean, p["m0"], p["phase"], *S.noise_draws(11, 12, seq.n), 25.0)
    z = oracle_lib.zoom(seq, g, x)
    t1, t2, df = S.grid_values(g)
    for v in range(12):
        a, b, c = z["abc"][v]
        d0 = oracle_lib.simulate(seq, t1[a], t2[b], df[c])[0]
        c0 = oracle_lib.cc(x[v], d0)
        assert c0 == pytest.approx(z["cc"][v], abs=1e-12)
        for da in (-1, 0, 1):
            for db in (-1, 0, 1):
                aa, bb = a + da, b + db
                if (da, db) == (0, 0) or not (0 <= aa < g.n_t1 and 0 <= bb < g.n_t2) or t2[bb] >= t1[aa]:
                    continue
                dn = oracle_lib.simulate(seq, t1[aa], t2[bb], df[c])[0]
                assert oracle_lib.cc(x[v], dn) <= c0


def test_zoom_with_omega_at_resolution_is_brute_force_in_df(oracle_lib):
    """Experiment 2: with omega equal to the df resolution the df search is a
    full scan, i.e. brute force over df."""
    seq = S.sequence(2, 200)
    g = S.Grid(900.0, 1.0, 1, 80.0, 1.0, 1, -30.0, 1.0, 61)
    p = S.phantom_offgrid(12, 6, t1_range=(899, 901), t2_range=(79, 81), df_range=(-28, 28))
    clean = oracle_lib.simulate(seq, p["t1"], p["t2"], p["df"])
    x = S.compose_voxels(clean, p["m0"], p["phase"], *S.noise_draws(12, 6, seq.n), 5.0)
    z = oracle_lib.zoom(seq, g, x, oracle_lib.default_zoom_opts(omega_hz=1.0, t1_init_ms=900, t2_init_ms=80))
    bf = oracle_lib.bruteforce(seq, g, x, k=1)
    assert (z["abc"][:, 2] == bf["idx"][:, 0]).all()
    np.testing.assert_allclose(z["cc"], bf["cc"][:, 0], atol=1e-14)


def test_zoom_centre_is_running_maximum(oracle_lib):
    """The accepted centre value never decreases along the trace."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    x = oracle_lib.simulate(seq, 733.0, 71.0, 0.0)[0]
    x = x + 0.01 * np.random.default_rng(3).normal(size=x.shape)
    t1, t2, df = S.grid_values(g)
    cache = {}

    def score(a, b, c):
        key = (a, b, c)
        if key not in cache:
            cache[key] = oracle_lib.cc(x, oracle_lib.simulate(seq, t1[a], t2[b], df[c])[0])
        return cache[key]

    r = oracle_lib.zoom_generic(g, score, oracle_lib.default_omega(seq))
    # moves and scans only ever accept a strictly better point, so the final
    # centre holds the maximum of everything evaluated
    assert r["cc"] == r["trace_cc"].max()
    z = oracle_lib.zoom(seq, g, x[None, :])
    assert tuple(z["abc"][0]) == r["abc"]
    assert z["evaluated"][0] == r["evaluated"]


def test_zoom_neighbour_ties_follow_scan_order(oracle_lib):
    """Two neighbours tie for best: the move goes to the first one in the
    fixed scan order (T1 offset outer, -1 before +1)."""
    g = S.Grid(0.0, 1.0, 41, 0.0, 1.0, 41, 0.0, 1.0, 1, 0)
    f = lambda a, b, c: -float(min((a - 16) ** 2, (a - 24) ** 2)) - float((b - 20) ** 2)
    o = oracle_lib.default_zoom_opts(t1_init_ms=20.0, t2_init_ms=20.0, s2=[(4.0, 4.0)], s4=[])
    r = oracle_lib.zoom_generic(g, f, 1.0, o)
    assert r["abc"] == (16, 20, 0)
    assert r["min_margin"] == 0.0


def test_bruteforce_exact_ties_go_to_smaller_index(oracle_lib):
    """T1 values so large that exp(-t/T1) rounds to 1 give bitwise identical
    fingerprints, hence exactly tied CC: the smaller linear index ranks first."""
    seq = S.sequence(4, 64)
    g = S.Grid(1e300, 1e290, 3, 50.0, 10.0, 2, -5.0, 5.0, 3)
    x = oracle_lib.simulate(seq, 1e300, 60.0, 0.0)
    r = oracle_lib.bruteforce(seq, g, x, k=4)
    # entries (a, b=1, c=1) for a = 0, 1, 2 are identical -> indices 4, 10, 16
    assert list(r["idx"][0, :3]) == [4, 10, 16]
    assert r["cc"][0, 0] == r["cc"][0, 1] == r["cc"][0, 2]


# ------------------------------------------------------- windowed refinement

def test_refine_l1_score_closed_form(oracle_lib):
    """Score -(|a-a*| + |b-b*| + |c-c*|): the best of the 26 neighbours steps
    every unsettled coordinate one towards the target, so the climb takes
    max |delta| moves, ends at the target, and (away from the grid's edges)
    evaluates 1 + 26 (moves + 1) points; integer scores give a margin of 1."""
    g = S.Grid(0.0, 1.0, 40, 0.0, 1.0, 40, 0.0, 1.0, 30, 0)
    target = (25, 14, 9)
    f = lambda a, b, c: -(abs(a - target[0]) + abs(b - target[1]) + abs(c - target[2]))
    for start in [(10, 20, 3), (25, 14, 9), (30, 5, 20), (24, 15, 9)]:
        r = oracle_lib.refine_generic(g, f, start)
        moves = max(abs(s - t) for s, t in zip(start, target))
        assert r["abc"] == target
        assert r["cc"] == 0.0
        assert r["evaluated"] == 1 + 26 * (moves + 1)
        assert r["min_margin"] == 1.0


def test_refine_ties_follow_neighbour_order(oracle_lib):
    """Two neighbours tie for best: the first in the order (T1 offset outer,
    then T2, then df, -1 before +1) wins; (+1, -1, 0) comes before (+1, 0, -1)."""
    g = S.Grid(0.0, 1.0, 9, 0.0, 1.0, 9, 0.0, 1.0, 9, 0)
    top = {(5, 3, 4): 1.0, (5, 4, 3): 1.0}
    f = lambda a, b, c: top.get((a, b, c), 0.0) - (0.5 if (a, b, c) not in top and (a, b, c) != (4, 4, 4) else 0.0)
    r = oracle_lib.refine_generic(g, f, (4, 4, 4))
    assert r["abc"] == (5, 3, 4) and r["cc"] == 1.0
    assert r["min_margin"] == 0.0


def test_refine_skips_invalid_points_and_stops_at_max_moves(oracle_lib):
    g = S.Grid(0.0, 1.0, 12, 0.0, 1.0, 12, 0.0, 1.0, 4, 1)
    seen = []

    def f(a, b, c):
        seen.append((a, b, c))
        return -abs(a - 3) - abs(b - 2) - abs(c - 0)

    r = oracle_lib.refine_generic(g, f, (8, 6, 3))
    assert all(0 <= b < a < 12 and 0 <= c < 4 for a, b, c in seen)
    assert r["abc"] == (3, 2, 0) and r["evaluated"] == len(seen)
    with pytest.raises(RuntimeError):
        oracle_lib.refine_generic(g, f, (8, 6, 3), max_moves=2)


def test_refine_keeps_brute_force_optimum_and_reaches_local_optima(oracle_lib):
    """From the exhaustive optimum the climb does not move (the global maximum
    is a local one). From perturbed starts it ends at a point whose FP64 CC is
    at least that of each of its 26 neighbours (checked here with numpy)."""
    seq = S.sequence(4, 120)
    g = S.Grid(200.0, 40.0, 30, 20.0, 15.0, 20, -12.0, 3.0, 9)
    ph = S.phantom_offgrid(44, 12, t1_range=(400.0, 1300.0), t2_range=(50.0, 250.0), df_range=(-8.0, 8.0))
    clean = oracle_lib.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    x = S.compose_voxels(clean, ph["m0"], ph["phase"], *S.noise_draws(44, 12, seq.n), 25.0)
    bf = oracle_lib.bruteforce(seq, g, x, k=1)
    a, b, c = oracle_lib.grid_params(g)
    best = np.stack([a[bf["idx"][:, 0]], b[bf["idx"][:, 0]], c[bf["idx"][:, 0]]], 1)
    r0 = oracle_lib.refine(seq, g, x, best)
    assert (r0["abc"] == best).all()
    np.testing.assert_allclose(r0["cc"], bf["cc"][:, 0], rtol=0, atol=1e-14)
    rng = np.random.default_rng(9)
    start = np.clip(best + rng.integers(-4, 5, best.shape), 0, [g.n_t1 - 1, g.n_t2 - 1, g.n_df - 1])
    t1, t2, df = S.grid_values(g)
    start[:, 1] = np.minimum(start[:, 1], np.searchsorted(t2, t1[start[:, 0]]) - 1)
    r = oracle_lib.refine(seq, g, x, start)
    d0 = oracle_lib.simulate(seq, t1[start[:, 0]], t2[start[:, 1]], df[start[:, 2]])
    cc0 = np.abs(np.sum(d0.conj() * x, 1)) / (np.linalg.norm(d0, axis=1) * np.linalg.norm(x, axis=1))
    assert (r["cc"] >= cc0 - 1e-12).all()
    for v in range(len(x)):
        ca, cb, cc0 = r["abc"][v]
        pts = [(ca + i, cb + j, cc0 + k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]
        pts = [p for p in pts if 0 <= p[0] < g.n_t1 and 0 <= p[1] < g.n_t2 and 0 <= p[2] < g.n_df
               and t2[p[1]] < t1[p[0]]]
        pts = np.array(pts)
        d = oracle_lib.simulate(seq, t1[pts[:, 0]], t2[pts[:, 1]], df[pts[:, 2]])
        cc = np.abs(d.conj() @ x[v]) / (np.linalg.norm(d, axis=1) * np.linalg.norm(x[v]))
        assert cc.max() <= r["cc"][v] + 1e-12
        assert len(pts) == 27 or r["evaluated"][v] >= len(pts)


# ---------------------------------------------------------- temporal smoothing

def test_smoothing_closed_forms(oracle_lib):
    """Gaussian weights exp(-k^2 / 2 sigma^2), renormalised where the window
    leaves the timecourse: constants are unchanged, an interior linear ramp is
    unchanged (symmetric weights), an impulse returns the normalised weights,
    and width 1 is the identity."""
    n = 40
    c = np.full((1, n), 0.3 - 0.7j)
    for w in (3, 5):
        np.testing.assert_allclose(oracle_lib.smooth(c, w), c, rtol=0, atol=1e-15)
    ramp = (np.arange(n) * (0.25 + 0.5j))[None, :]
    out = oracle_lib.smooth(ramp, 5, 1.3)
    np.testing.assert_allclose(out[0, 2:-2], ramp[0, 2:-2], rtol=0, atol=1e-13)
    imp = np.zeros((1, n), complex)
    imp[0, 20] = 1.0
    for w, s in ((3, 1.0), (5, 1.0), (5, 0.7)):
        h = (w - 1) // 2
        wts = np.exp(-np.arange(-h, h + 1) ** 2 / (2 * s * s))
        out = oracle_lib.smooth(imp, w, s)[0]
        # sample 20 + k receives weight w_{-k} of the impulse over the full window sum
        np.testing.assert_allclose(out[20 - h: 21 + h].real, wts[::-1] / wts.sum(), rtol=1e-14)
        assert np.abs(np.delete(out, np.arange(20 - h, 21 + h))).max() == 0.0
    # the first sample's window is cut to samples 0..h, renormalised there
    x = np.arange(1, n + 1, dtype=float)[None, :] + 0j
    wts = np.exp(-np.arange(0, 3) ** 2 / 2.0)
    np.testing.assert_allclose(oracle_lib.smooth(x, 5)[0, 0].real, (wts * x[0, :3].real).sum() / wts.sum(), rtol=1e-14)
    rng = np.random.default_rng(3)
    z = rng.normal(size=(2, n)) + 1j * rng.normal(size=(2, n))
    np.testing.assert_array_equal(oracle_lib.smooth(z, 1), z)


def test_smoothed_bruteforce_recovers_on_grid_voxels(oracle_lib):
    """Smoothing is linear and applied alike to both sides, so a noise-free
    on-grid fingerprint, smoothed, still matches its own smoothed entry with
    CC = 1 and the applied scale as M0."""
    seq, g, ph, x = _tiny_voxels(oracle_lib, 24, None, seed=300)
    for w in (3, 5):
        xs = oracle_lib.smooth(x, w)
        r = oracle_lib.bruteforce(seq, g, xs, k=1, smooth=(w, 1.0))
        a, b, c = oracle_lib.grid_params(g)
        assert (a[r["idx"][:, 0]] == ph["a"]).all() and (b[r["idx"][:, 0]] == ph["b"]).all()
        np.testing.assert_allclose(r["cc"][:, 0], 1.0, atol=1e-12)
        np.testing.assert_allclose(r["m0"], ph["m0"], rtol=1e-12)
    # smoothing the dictionary alone changes the scores: the plain entry no longer matches exactly
    r1 = oracle_lib.bruteforce(seq, g, x, k=1, smooth=(5, 1.0))
    assert (r1["cc"][:, 0] < 1.0 - 1e-6).all()


# ---------------------------------------------------------------------------
# Spatial-neighbour prior (Methods, Experiment 3)

def _box_by_enumeration(g, abc_p, half):
    """The index box of the axis values within the half-widths of the
    preceding voxel's values, found by scanning each axis (no step formula)."""
    axes = [(g.t1_min, g.t1_step, g.n_t1), (g.t2_min, g.t2_step, g.n_t2), (g.df_min, g.df_step, g.n_df)]
    box = []
    for (mn, st, n), p, h in zip(axes, abc_p, half):
        inside = [i for i in range(n) if abs((mn + i * st) - (mn + p * st)) <= h + 1e-9]
        box.append((min(inside), max(inside)))
    return box


def test_prior_box_by_hand(oracle_lib):
    """The index box of T1p +- 100 ms on a 20 ms axis is 5 steps each way,
    cut by the axis ends; the paper's windows (3000, 800, 150) cover most of
    this grid."""
    g = S.GRIDS["fp32_brute"]   # T1 step 20 ms (196), T2 step 5 ms (79), df step 2 Hz (41)
    assert oracle_lib.prior_box(g, (10, 40, 20), (100.0, 50.0, 6.0)) == [(5, 15), (30, 50), (17, 23)]
    assert oracle_lib.prior_box(g, (2, 77, 0), (100.0, 50.0, 6.0)) == [(0, 7), (67, 78), (0, 3)]
    assert oracle_lib.prior_box(g, (2, 77, 0), (3000.0, 800.0, 150.0)) == [(0, 152), (0, 78), (0, 40)]
    for p in ((0, 0, 0), (195, 78, 40), (97, 12, 33)):
        for half in ((100.0, 50.0, 6.0), (55.0, 7.5, 1.0), (3000.0, 800.0, 150.0)):
            assert oracle_lib.prior_box(g, p, half) == _box_by_enumeration(g, p, half)


def _uniform_slice(oracle_lib, seq, t1, t2, df, v, seed):
    """v noise-free voxels of one (T1, T2, df), each with its own M0 and phase."""
    rng = np.random.default_rng(seed)
    clean = oracle_lib.simulate(seq, np.full(v, t1), np.full(v, t2), np.full(v, df))
    return clean * (rng.uniform(0.5, 1.0, v) * np.exp(1j * rng.uniform(0, 2 * np.pi, v)))[:, None]


def test_prior_chain_started_at_the_optimum_by_hand(oracle_lib):
    """A 3 x 3 slice of one on-grid tissue (noise-free), on the tiny grid (T1
    100-2000/100 ms, T2 20-200/20 ms, df 0): voxel 0 is searched plainly and
    finds the point (a, b) = (13, 4), i.e. 1400 / 100 ms; every later voxel
    starts at its predecessor's result, which is its own optimum (CC 1), so no
    decision moves and its evaluation count is that of the schedule's
    decisions around (13, 4), counted by hand: step 1 one df point; step 2 at
    (2, 10) steps only (11, 4) and (15, 4) exist, at (1, 5) the five points
    with b = 4 or 9; step 4 T1 at 1 step 2, T2 at 5 steps 1 (b = 9), T1 at 1
    step 2, T2 at 3 steps 2, T2 at 1 step 2 (T1 at 20 and 10 ms snap to the
    same 1-step level and are dropped, as is T2 at 10 ms); step 5 eight:
    1 + 2 + 5 + 2 + 1 + 2 + 2 + 2 + 8 = 25."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    x = _uniform_slice(oracle_lib, seq, 1400.0, 100.0, 0.0, 9, 11)
    r = oracle_lib.zoom_prior(seq, g, x)
    assert [tuple(v) for v in r["abc"]] == [(13, 4, 0)] * 9
    np.testing.assert_allclose(r["cc"], 1.0, atol=1e-12)
    assert list(r["evaluated"][1:]) == [25] * 8
    assert r["evaluated"][0] > 25          # the first voxel walks from the default start
    for v in range(1, 9):
        assert tuple(r["box"][v]) == (0, 19, 0, 9, 0, 0)   # the paper's windows cover this grid


def test_prior_chain_follows_the_preceding_voxel(oracle_lib):
    """Voxels alternate between two tissues, (1400, 100) ms and (600, 40) ms,
    on the tiny grid with narrow windows (T1p +- 300 ms, T2p +- 40 ms): each
    voxel's box is the enumerated box around its predecessor's result, every
    result lies in its box, and a (600, 40) voxel after a (1400, 100) one
    cannot reach its own point. Cut into chains of 3, the first voxel of each
    chain is searched on the whole grid and finds its own point, and the
    chain's first voxels equal the single chain's."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["tiny"]
    xa = _uniform_slice(oracle_lib, seq, 1400.0, 100.0, 0.0, 5, 12)
    xb = _uniform_slice(oracle_lib, seq, 600.0, 40.0, 0.0, 4, 13)
    x = np.stack([xa[0], xb[0], xa[1], xb[1], xa[2], xb[2], xa[3], xb[3], xa[4]])
    half = (300.0, 40.0, 0.0)
    r = oracle_lib.zoom_prior(seq, g, x, half=half)
    for v in range(1, 9):
        box = _box_by_enumeration(g, r["abc"][v - 1], half)
        assert tuple(r["box"][v]) == (box[0][0], box[0][1], box[1][0], box[1][1], box[2][0], box[2][1])
        for k in range(3):
            assert box[k][0] <= r["abc"][v][k] <= box[k][1]
    assert tuple(r["abc"][0]) == (13, 4, 0)
    assert tuple(r["abc"][1]) != (5, 1, 0)       # (600, 40) lies outside the box around (1400, 100)
    assert abs(int(r["abc"][1][0]) - 13) <= 3
    r3 = oracle_lib.zoom_prior(seq, g, x, chain=3, half=half)
    for v in (0, 3, 6):
        assert tuple(r3["box"][v]) == (0, 19, 0, 9, 0, 0)
    assert [tuple(r3["abc"][v]) for v in (0, 3, 6)] == [(13, 4, 0), (5, 1, 0), (13, 4, 0)]
    assert tuple(r3["abc"][4]) != (13, 4, 0) and abs(int(r3["abc"][4][0]) - 5) <= 3   # bounded by voxel 3
    for k in ("abc", "evaluated", "cc"):
        assert np.array_equal(r3[k][:3], r[k][:3]), k


def test_prior_covering_the_grid_changes_nothing(oracle_lib):
    """With windows wider than every axis and the start left at the options'
    start, the sub-grid is the grid: the prior search returns exactly the
    plain search's results."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["fp32_brute"]
    ph = S.phantom_piecewise(5, 4, 4)
    clean = oracle_lib.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    g_re, g_im = S.noise_draws(5, 16, seq.n)
    x = S.compose_voxels(clean, ph["m0"], ph["phase"], g_re, g_im, 30.0)
    plain = oracle_lib.zoom(seq, g, x)
    pri = oracle_lib.zoom_prior(seq, g, x, half=(1e6, 1e6, 1e6), start_from_prior=False)
    for k in ("abc", "evaluated"):
        assert np.array_equal(plain[k], pri[k]), k
    assert np.array_equal(plain["cc"], pri["cc"])


def test_prior_results_lie_in_their_boxes(oracle_lib):
    """Narrow windows (T1p +- 200 ms, T2p +- 30 ms, dfp +- 6 Hz) on a noisy
    piecewise-smooth 4 x 4 slice: every result lies in the box around its
    predecessor's result, and starts from it, so it equals the plain search
    on that box's sub-grid started at the predecessor's (T1, T2)."""
    seq = S.sequence(0, 200)
    g = S.GRIDS["fp32_brute"]
    ph = S.phantom_piecewise(6, 4, 4)
    clean = oracle_lib.simulate(seq, ph["t1"], ph["t2"], ph["df"])
    g_re, g_im = S.noise_draws(6, 16, seq.n)
    x = S.compose_voxels(clean, ph["m0"], ph["phase"], g_re, g_im, 30.0)
    half = (200.0, 30.0, 6.0)
    pri = oracle_lib.zoom_prior(seq, g, x, half=half)
    for v in range(1, 16):
        box = _box_by_enumeration(g, pri["abc"][v - 1], half)
        assert list(pri["box"][v]) == [box[0][0], box[0][1], box[1][0], box[1][1], box[2][0], box[2][1]]
        for k in range(3):
            assert box[k][0] <= pri["abc"][v][k] <= box[k][1]
    v = 7
    (a0, a1), (b0, b1), (c0, c1) = _box_by_enumeration(g, pri["abc"][v - 1], half)
    sub = S.Grid(g.t1_min + a0 * g.t1_step, g.t1_step, a1 - a0 + 1, g.t2_min + b0 * g.t2_step, g.t2_step, b1 - b0 + 1,
                 g.df_min + c0 * g.df_step, g.df_step, c1 - c0 + 1)
    p = pri["abc"][v - 1]
    o = oracle_lib.default_zoom_opts(t1_init_ms=g.t1_min + p[0] * g.t1_step, t2_init_ms=g.t2_min + p[1] * g.t2_step)
    r = oracle_lib.zoom(seq, sub, x[v:v + 1], o)
    assert list(r["abc"][0] + np.array([a0, b0, c0])) == list(pri["abc"][v])
