/*
 * mrf_oracle.c -- plain FP64 CPU oracle for MRF dictionary generating and
 * searching (DGS), written from Z. Wang, "MRF-ZOOM: A Fast Dictionary
 * Searching Algorithm for Magnetic Resonance Fingerprinting".
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the GPU library links, includes or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do. It shares no code with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - Bloch propagation, Appendix Eq. A2 (M <- R_off R_relax R_RF M) with the
 *     hard-pulse RF form R_RF = R_z(phi) R_x(-alpha) R_z(-phi) stated at the
 *     end of the Appendix, and the longitudinal recovery term of Eq. A1; for
 *     pulses of finite duration tau the Appendix's off-resonant form
 *     R_RF = R_z(phi) R_y(beta) R_x(alpha') R_y(-beta) R_z(-phi).
 *   - Complex correlation coefficient, Eq. 1 (Theory).
 *   - Brute-force DGS: argmax of Eq. 1 over every grid entry (Theory, "the
 *     original DGS"; Experiment 2).
 *   - MRF-ZOOM: the df search of Theory (steps 1-4) with the constants of
 *     Experiment 2 step 1, the 2D ZOOM of Fig. 2, the df refinement of step 3,
 *     the interleaved 1D ZOOMs of Fig. 1 / step 4 and the final 2D ZOOM of
 *     step 5.
 *   - Windowed refinement: the windowed brute-force check around a ZOOM
 *     answer (Results, Experiment 2), repeated as a hill climb on the grid.
 *   - Temporal smoothing of fingerprints and dictionary entries (Methods,
 *     Experiment 4), and brute force against a smoothed dictionary.
 *
 * Precision: IEEE double throughout, libm exp/sin/cos, no FMA contraction
 * (built with -ffp-contract=off). OpenMP parallelises over independent
 * dictionary entries or voxels only; every per-entry and per-voxel result is
 * computed in a fixed order, so results do not depend on the thread count.
 *
 * Parity status: simulator, CC, grid enumeration, brute force and the ZOOM
 * stage machine are pinned by tests (closed forms, invariants, exhaustive
 * search, hand-derived traces on analytic score functions). ZOOM on the
 * finest (2.4e9-entry) grid has no exhaustive reference: "parity unpinned"
 * there beyond local-optimality and windowed brute-force checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Descriptors (laid out like the ctypes structures in oracle/__init__.py).   */

typedef struct {
    int32_t n;             /* timepoints */
    const double *flip;    /* alpha_j in rad, signed */
    const double *phase;   /* RF phase phi_j in rad, NULL means all zero */
    const double *tr;      /* TR_j in ms */
    const double *te;      /* TE_j in ms, 0 <= TE_j <= TR_j */
    int32_t inversion;     /* 1: ideal 180 degree pulse, then inv_delay */
    double inv_delay;      /* ms */
    const double *pulse;   /* RF pulse duration tau_j in ms, NULL means all hard (0) */
} or_seq;

typedef struct {
    double t1_min, t1_step; int32_t n_t1;
    double t2_min, t2_step; int32_t n_t2;
    double df_min, df_step; int32_t n_df;
    int32_t require_t2_lt_t1;
} or_grid;

#define OR_MAX_LEVELS 16
typedef struct {
    double omega_hz;        /* <= 0: 1000 / min_j TR_j (Property II, ~1/TR) */
    double t1_init_ms;      /* starting T1 of the df search */
    double t2_init_ms;      /* starting T2 of the df search */
    double s1a_step_frac;   /* coarse df scan step as a fraction of omega */
    double s1b_half_frac;   /* half-width of the first df window, x omega */
    double s1b_step_frac;   /* step inside that window, x omega */
    double s3_half_frac;    /* half-width of the finest df window, x omega */
    int32_t n_s2;           /* 2D ZOOM levels before the df refinement */
    double s2_t1_ms[OR_MAX_LEVELS];
    double s2_t2_ms[OR_MAX_LEVELS];
    int32_t n_s4;           /* interleaved 1D ZOOMs */
    int32_t s4_param[OR_MAX_LEVELS];   /* 0: T1, 1: T2 */
    double s4_ms[OR_MAX_LEVELS];
} or_zoom_opts;

/* ------------------------------------------------------------------------- */
/* Appendix: rotations (counterclockwise), relaxation, RF.                    */

static void rot_x(double th, double M[3])
{
    double c = cos(th), s = sin(th);
    double y = M[1], z = M[2];
    M[1] = c * y - s * z;
    M[2] = s * y + c * z;
}

static void rot_z(double th, double M[3])
{
    double c = cos(th), s = sin(th);
    double x = M[0], y = M[1];
    M[0] = c * x - s * y;
    M[1] = s * x + c * y;
}

static void rot_y(double th, double M[3])
{
    double c = cos(th), s = sin(th);
    double x = M[0], z = M[2];
    M[0] = c * x + s * z;
    M[2] = -s * x + c * z;
}

/* Hard pulse: R_RF = R_z(phi) R_x(-alpha) R_z(-phi), applied right to left. */
static void rf_pulse(double alpha, double phi, double M[3])
{
    rot_z(-phi, M);
    rot_x(-alpha, M);
    rot_z(phi, M);
}

/* Pulse of duration tau ms off resonance by df Hz (Appendix): R_RF =
 * R_z(phi) R_y(beta) R_x(alpha') R_y(-beta) R_z(-phi) with beta the angle
 * between the x axis and the effective field, tan(beta) = tau dw / alpha,
 * and alpha' = -tau sqrt(dw^2 + (alpha / tau)^2) the rotation about it over
 * the pulse, dw = 2 pi df / 1000 rad/ms. beta is taken as atan2(tau dw,
 * alpha), which is the printed arctangent for alpha > 0 and keeps the signed
 * (alternating) flip angles and alpha = 0 on the same effective field; tau = 0
 * is the hard pulse. No relaxation acts during the pulse (R_RF has none). */
static void rf_pulse_finite(double alpha, double phi, double tau, double df, double M[3])
{
    if (!(tau > 0.0)) { rf_pulse(alpha, phi, M); return; }
    double tdw = tau * 2.0 * M_PI * df / 1000.0;
    double beta = atan2(tdw, alpha);
    double ap = -sqrt(alpha * alpha + tdw * tdw);
    rot_z(-phi, M);
    rot_y(-beta, M);
    rot_x(ap, M);
    rot_y(beta, M);
    rot_z(phi, M);
}

/* Free evolution over tau ms: R_relax (with the (M0 - Mz)/T1 recovery of
 * Eq. A1, M0 = 1), then R_off = R_z(2 pi df tau / 1000), df in Hz. */
static void free_evolve(double tau, double T1, double T2, double df, double M[3])
{
    double E1 = exp(-tau / T1);
    double E2 = exp(-tau / T2);
    M[0] = E2 * M[0];
    M[1] = E2 * M[1];
    M[2] = E1 * M[2] + (1.0 - E1);
    rot_z(2.0 * M_PI * df * tau / 1000.0, M);
}

/* One fingerprint. Start state (0,0,1) unless m_init is given. For each j:
 * RF pulse (hard, or of duration tau_j), evolve TE_j, sample s_j = Mx + i My,
 * evolve TR_j - TE_j. The inversion is an ideal hard pulse.
 * sig: n interleaved (re, im). state (optional): n x 3 state at each sample. */
static void simulate_one(const or_seq *s, double T1, double T2, double df,
                         const double *m_init, double *sig, double *state)
{
    double M[3] = {0.0, 0.0, 1.0};
    if (m_init) { M[0] = m_init[0]; M[1] = m_init[1]; M[2] = m_init[2]; }
    if (s->inversion) {
        rf_pulse(M_PI, 0.0, M);
        free_evolve(s->inv_delay, T1, T2, df, M);
    }
    for (int32_t j = 0; j < s->n; ++j) {
        rf_pulse_finite(s->flip[j], s->phase ? s->phase[j] : 0.0, s->pulse ? s->pulse[j] : 0.0, df, M);
        free_evolve(s->te[j], T1, T2, df, M);
        if (sig) { sig[2 * j] = M[0]; sig[2 * j + 1] = M[1]; }
        if (state) { state[3 * j] = M[0]; state[3 * j + 1] = M[1]; state[3 * j + 2] = M[2]; }
        free_evolve(s->tr[j] - s->te[j], T1, T2, df, M);
    }
}

int or_simulate_state(const or_seq *s, double T1, double T2, double df,
                      const double *m_init, double *sig, double *state)
{
    if (!s || s->n < 1) return -1;
    simulate_one(s, T1, T2, df, m_init, sig, state);
    return 0;
}

/* count fingerprints for parameter triples; out: count x n x 2 doubles. */
int or_simulate(const or_seq *s, int64_t count, const double *T1, const double *T2,
                const double *df, double *out)
{
    if (!s || s->n < 1 || count < 0) return -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t e = 0; e < count; ++e)
        simulate_one(s, T1[e], T2[e], df[e], NULL, out + (size_t)e * 2 * s->n, NULL);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1: CC = |sum_j x_j conj(d_j)| / (||x|| ||d||); 0 when a norm is 0.     */

static void inner(int32_t n, const double *x, const double *d, double *re, double *im)
{
    double r = 0.0, i = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        /* x conj(d) = (xr + i xi)(dr - i di) */
        r += x[2 * j] * d[2 * j] + x[2 * j + 1] * d[2 * j + 1];
        i += x[2 * j + 1] * d[2 * j] - x[2 * j] * d[2 * j + 1];
    }
    *re = r; *im = i;
}

static double norm2(int32_t n, const double *x)
{
    double acc = 0.0;
    for (int32_t j = 0; j < n; ++j) acc += x[2 * j] * x[2 * j] + x[2 * j + 1] * x[2 * j + 1];
    return acc;
}

double or_cc(int32_t n, const double *x, const double *d)
{
    double re, im;
    inner(n, x, d, &re, &im);
    double nx = sqrt(norm2(n, x)), nd = sqrt(norm2(n, d));
    if (nx == 0.0 || nd == 0.0) return 0.0;
    return sqrt(re * re + im * im) / (nx * nd);
}

/* ------------------------------------------------------------------------- */
/* Grid: value i of an axis is min + i * step; valid iff T2 < T1 (if asked). */

static double t1_of(const or_grid *g, int32_t a) { return g->t1_min + (double)a * g->t1_step; }
static double t2_of(const or_grid *g, int32_t b) { return g->t2_min + (double)b * g->t2_step; }
static double df_of(const or_grid *g, int32_t c) { return g->df_min + (double)c * g->df_step; }

static int valid_ab(const or_grid *g, int32_t a, int32_t b)
{
    if (a < 0 || a >= g->n_t1 || b < 0 || b >= g->n_t2) return 0;
    return g->require_t2_lt_t1 ? (t2_of(g, b) < t1_of(g, a)) : 1;
}

static int grid_ok(const or_grid *g)
{
    return g && g->n_t1 >= 1 && g->n_t2 >= 1 && g->n_df >= 1 &&
           g->t1_step > 0 && g->t2_step > 0 && g->df_step > 0;
}

/* valid T2 count for each T1 index (the valid set of b is a prefix 0..k-1
 * because T2 increases with b). */
static int32_t nb_valid(const or_grid *g, int32_t a)
{
    int32_t k = 0;
    for (int32_t b = 0; b < g->n_t2; ++b) if (valid_ab(g, a, b)) k = b + 1;
    return k;
}

int64_t or_grid_count(const or_grid *g)
{
    if (!grid_ok(g)) return -1;
    int64_t total = 0;
    for (int32_t a = 0; a < g->n_t1; ++a)
        for (int32_t b = 0; b < g->n_t2; ++b)
            if (valid_ab(g, a, b)) total += g->n_df;
    return total;
}

/* Linear index of valid entry (a, b, c): T1 outermost, T2, df innermost. */
int64_t or_grid_index(const or_grid *g, int32_t a, int32_t b, int32_t c)
{
    if (!grid_ok(g) || !valid_ab(g, a, b) || c < 0 || c >= g->n_df) return -1;
    int64_t idx = 0;
    for (int32_t aa = 0; aa < a; ++aa)
        for (int32_t bb = 0; bb < g->n_t2; ++bb)
            if (valid_ab(g, aa, bb)) idx += g->n_df;
    for (int32_t bb = 0; bb < b; ++bb)
        if (valid_ab(g, a, bb)) idx += g->n_df;
    return idx + c;
}

/* Enumerate all valid entries in linear order (small grids). */
int64_t or_grid_params(const or_grid *g, int64_t cap, int32_t *a_out, int32_t *b_out, int32_t *c_out)
{
    if (!grid_ok(g)) return -1;
    int64_t k = 0;
    for (int32_t a = 0; a < g->n_t1; ++a)
        for (int32_t b = 0; b < g->n_t2; ++b) {
            if (!valid_ab(g, a, b)) continue;
            for (int32_t c = 0; c < g->n_df; ++c, ++k)
                if (k < cap) { a_out[k] = a; b_out[k] = b; c_out[k] = c; }
        }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Temporal smoothing (Methods, Experiment 4: "3 points and 5 points moving
 * Gaussian smoothing" of the fingerprints and of the dictionary). Each sample
 * becomes the weighted mean of the samples within h = (width - 1) / 2 of it,
 * weights exp(-k^2 / (2 sigma^2)), renormalised over the samples that exist
 * at the ends of the timecourse; Re and Im alike. width = 1: the identity.
 * x and out: n interleaved complex samples, distinct arrays.              */

static void smooth_one(int32_t n, const double *x, int32_t width, double sigma, double *out)
{
    const int32_t h = (width - 1) / 2;
    for (int32_t j = 0; j < n; ++j) {
        double wr = 0.0, sr = 0.0, si = 0.0;
        for (int32_t k = -h; k <= h; ++k) {
            const int32_t i = j + k;
            if (i < 0 || i >= n) continue;
            const double w = exp(-(double)(k * k) / (2.0 * sigma * sigma));
            wr += w;
            sr += w * x[2 * i];
            si += w * x[2 * i + 1];
        }
        out[2 * j] = sr / wr;
        out[2 * j + 1] = si / wr;
    }
}

int or_smooth(int32_t n, int64_t V, const double *x, int32_t width, double sigma, double *out)
{
    if (n < 1 || V < 0 || width < 1 || (width & 1) == 0 || !(sigma > 0.0)) return -1;
    for (int64_t v = 0; v < V; ++v) smooth_one(n, x + (size_t)v * 2 * n, width, sigma, out + (size_t)v * 2 * n);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Brute-force DGS: for every voxel, the top-k entries by Eq. 1 (descending
 * CC, ties to the smaller linear index), plus M0 = |<x,d>| / ||d||^2 and
 * phase = arg <x,d> of the best entry (Theory: proton density from scale). */

typedef struct { double cc; int64_t idx; } or_cand;

static int cand_before(double cc, int64_t idx, const or_cand *o)
{
    return cc > o->cc || (cc == o->cc && idx < o->idx);
}

static void topk_insert(or_cand *list, int32_t k, double cc, int64_t idx)
{
    if (!cand_before(cc, idx, &list[k - 1])) return;
    int32_t p = k - 1;
    while (p > 0 && cand_before(cc, idx, &list[p - 1])) { list[p] = list[p - 1]; --p; }
    list[p].cc = cc; list[p].idx = idx;
}

/* Brute force against a dictionary whose entries are smoothed (width, sigma)
 * before their norm and CC are taken; width = 1 is the plain dictionary. The
 * fingerprints x are used as given (smooth them with or_smooth to smooth both
 * sides). */
static int bruteforce_impl(const or_seq *s, const or_grid *g, const double *x, int64_t V, int32_t k,
                           int32_t width, double sigma, int64_t *top_idx, double *top_cc, double *m0, double *phase)
{
    if (!s || s->n < 1 || !grid_ok(g) || V < 0 || k < 1) return -1;
    if (width < 1 || (width & 1) == 0 || !(sigma > 0.0)) return -1;
    if (V == 0) return 0;
    const int32_t n = s->n;
    double *xn = (double *)malloc(sizeof(double) * (size_t)V);
    int64_t *a_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(g->n_t1 + 1));
    if (!xn || !a_off) { free(xn); free(a_off); return -2; }
    for (int64_t v = 0; v < V; ++v) xn[v] = sqrt(norm2(n, x + (size_t)v * 2 * n));
    a_off[0] = 0;
    for (int32_t a = 0; a < g->n_t1; ++a) a_off[a + 1] = a_off[a] + (int64_t)nb_valid(g, a) * g->n_df;

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    or_cand *all = (or_cand *)malloc(sizeof(or_cand) * (size_t)nthreads * (size_t)V * (size_t)k);
    if (!all) { free(xn); free(a_off); return -2; }
    for (size_t i = 0; i < (size_t)nthreads * (size_t)V * (size_t)k; ++i) { all[i].cc = -1.0; all[i].idx = INT64_MAX; }
    int err = 0;

    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        or_cand *mine = all + (size_t)tid * (size_t)V * (size_t)k;
        double *d = (double *)malloc(sizeof(double) * 4 * (size_t)n);
        if (!d) {
            #pragma omp atomic write
            err = 1;
        } else {
            double *raw = d + 2 * (size_t)n;
            #pragma omp for schedule(dynamic, 1)
            for (int32_t a = 0; a < g->n_t1; ++a) {
                int64_t idx = a_off[a];
                int32_t nb = nb_valid(g, a);
                for (int32_t b = 0; b < nb; ++b)
                    for (int32_t c = 0; c < g->n_df; ++c, ++idx) {
                        if (width == 1) {
                            simulate_one(s, t1_of(g, a), t2_of(g, b), df_of(g, c), NULL, d, NULL);
                        } else {
                            simulate_one(s, t1_of(g, a), t2_of(g, b), df_of(g, c), NULL, raw, NULL);
                            smooth_one(n, raw, width, sigma, d);
                        }
                        double nd = sqrt(norm2(n, d));
                        for (int64_t v = 0; v < V; ++v) {
                            double re, im, cc = 0.0;
                            inner(n, x + (size_t)v * 2 * n, d, &re, &im);
                            if (nd > 0.0 && xn[v] > 0.0) cc = sqrt(re * re + im * im) / (xn[v] * nd);
                            topk_insert(mine + (size_t)v * k, k, cc, idx);
                        }
                    }
            }
            free(d);
        }
    }
    if (err) { free(all); free(xn); free(a_off); return -2; }

    /* merge the per-thread lists, then M0 and phase of each voxel's best */
    double *d = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    for (int64_t v = 0; v < V; ++v) {
        or_cand *dst = all + (size_t)v * k;   /* thread 0's list */
        for (int t = 1; t < nthreads; ++t) {
            or_cand *src = all + ((size_t)t * (size_t)V + (size_t)v) * (size_t)k;
            for (int32_t i = 0; i < k; ++i) topk_insert(dst, k, src[i].cc, src[i].idx);
        }
        for (int32_t i = 0; i < k; ++i) {
            top_idx[(size_t)v * k + i] = dst[i].idx == INT64_MAX ? -1 : dst[i].idx;
            top_cc[(size_t)v * k + i] = dst[i].cc;
        }
        if (d && dst[0].idx != INT64_MAX && (m0 || phase)) {
            /* recover (a, b, c) of the best linear index */
            int64_t best = dst[0].idx;
            int32_t a = 0;
            while (a + 1 <= g->n_t1 && a_off[a + 1] <= best) ++a;
            int64_t rem = best - a_off[a];
            int32_t b = (int32_t)(rem / g->n_df), c = (int32_t)(rem % g->n_df);
            if (width == 1) {
                simulate_one(s, t1_of(g, a), t2_of(g, b), df_of(g, c), NULL, d, NULL);
            } else {
                simulate_one(s, t1_of(g, a), t2_of(g, b), df_of(g, c), NULL, d + 2 * (size_t)n, NULL);
                smooth_one(n, d + 2 * (size_t)n, width, sigma, d);
            }
            double re, im;
            inner(n, x + (size_t)v * 2 * n, d, &re, &im);
            double dd = norm2(n, d);
            if (m0) m0[v] = dd > 0.0 ? sqrt(re * re + im * im) / dd : 0.0;
            if (phase) phase[v] = atan2(im, re);
        }
    }
    free(d); free(all); free(xn); free(a_off);
    return 0;
}

int or_bruteforce(const or_seq *s, const or_grid *g, const double *x, int64_t V, int32_t k,
                  int64_t *top_idx, double *top_cc, double *m0, double *phase)
{
    return bruteforce_impl(s, g, x, V, k, 1, 1.0, top_idx, top_cc, m0, phase);
}

int or_bruteforce_smooth(const or_seq *s, const or_grid *g, const double *x, int64_t V, int32_t k, int32_t width,
                         double sigma, int64_t *top_idx, double *top_cc, double *m0, double *phase)
{
    return bruteforce_impl(s, g, x, V, k, width, sigma, top_idx, top_cc, m0, phase);
}

/* ------------------------------------------------------------------------- */
/* MRF-ZOOM stage machine, written against a score callback so that the    */
/* control flow can be checked on analytic functions.                        */

typedef double (*or_score_fn)(void *ctx, int32_t a, int32_t b, int32_t c);

typedef struct {
    const or_grid *g;
    or_score_fn fn;
    void *ctx;
    int32_t evaluated;
    double min_margin;
    int32_t trace_cap, trace_n;
    int32_t *trace;       /* trace_cap x 4: stage, a, b, c */
    double *trace_cc;     /* trace_cap */
    int32_t stage;
    int32_t guard_hit;
} zoom_state;

/* CC of a grid point, -inf when out of range or invalid (never evaluated). */
static double zscore(zoom_state *z, int32_t a, int32_t b, int32_t c)
{
    const or_grid *g = z->g;
    if (c < 0 || c >= g->n_df || !valid_ab(g, a, b)) return -INFINITY;
    double v = z->fn(z->ctx, a, b, c);
    z->evaluated++;
    if (z->trace && z->trace_n < z->trace_cap) {
        int32_t *t = z->trace + 4 * z->trace_n;
        t[0] = z->stage; t[1] = a; t[2] = b; t[3] = c;
        z->trace_cc[z->trace_n] = v;
    }
    z->trace_n++;
    return v;
}

/* margin bookkeeping: gap between the two largest finite values of a decision set */
typedef struct { double top1, top2; } gap2;
static void gap_reset(gap2 *m) { m->top1 = -INFINITY; m->top2 = -INFINITY; }
static void gap_add(gap2 *m, double v)
{
    if (!isfinite(v)) return;
    if (v > m->top1) { m->top2 = m->top1; m->top1 = v; }
    else if (v > m->top2) m->top2 = v;
}
static void gap_close(zoom_state *z, const gap2 *m)
{
    if (isfinite(m->top2)) {
        double gp = m->top1 - m->top2;
        if (gp < z->min_margin) z->min_margin = gp;
    }
}

/* round-half-up snap of a physical step to whole grid steps, at least 1 */
static int32_t snap_steps(double h_phys, double step)
{
    int32_t h = (int32_t)floor(h_phys / step + 0.5);
    return h < 1 ? 1 : h;
}

#define ZOOM_MAX_MOVES (1 << 20)

/* 2D ZOOM (Fig. 2): compare the centre with its 4 edge and 4 corner
 * neighbours at (h1, h2); move to the best neighbour if it is strictly
 * better, repeat until the centre wins. Eager evaluation, fixed order. */
static void move2d(zoom_state *z, int32_t *a, int32_t *b, int32_t c, double *centre, int32_t h1, int32_t h2)
{
    static const int32_t off[8][2] = {{-1, -1}, {-1, 0}, {-1, 1}, {0, -1}, {0, 1}, {1, -1}, {1, 0}, {1, 1}};
    for (int32_t it = 0; it < ZOOM_MAX_MOVES; ++it) {
        gap2 m; gap_reset(&m); gap_add(&m, *centre);
        double best = -INFINITY; int32_t ba = *a, bb = *b;
        for (int k = 0; k < 8; ++k) {
            int32_t na = *a + off[k][0] * h1, nb = *b + off[k][1] * h2;
            double v = zscore(z, na, nb, c);
            gap_add(&m, v);
            if (v > best) { best = v; ba = na; bb = nb; }
        }
        gap_close(z, &m);
        if (best > *centre) { *a = ba; *b = bb; *centre = best; }
        else return;
    }
    z->guard_hit = 1;
}

/* 1D ZOOM (Fig. 1): compare the centre with the left and right ends at
 * half-width h along one parameter (0: T1, 1: T2). */
static void move1d(zoom_state *z, int32_t *a, int32_t *b, int32_t c, double *centre, int param, int32_t h)
{
    for (int32_t it = 0; it < ZOOM_MAX_MOVES; ++it) {
        gap2 m; gap_reset(&m); gap_add(&m, *centre);
        double best = -INFINITY; int32_t ba = *a, bb = *b;
        for (int s = -1; s <= 1; s += 2) {
            int32_t na = *a + (param == 0 ? s * h : 0), nb = *b + (param == 1 ? s * h : 0);
            double v = zscore(z, na, nb, c);
            gap_add(&m, v);
            if (v > best) { best = v; ba = na; bb = nb; }
        }
        gap_close(z, &m);
        if (best > *centre) { *a = ba; *b = bb; *centre = best; }
        else return;
    }
    z->guard_hit = 1;
}

/* The full schedule (Experiment 2, steps 1-5). Returns 0, or -1 when the
 * grid has no valid starting point. */
static int zoom_run(zoom_state *z, const or_zoom_opts *o, double omega,
                    int32_t *ra, int32_t *rb, int32_t *rc, double *rcc)
{
    const or_grid *g = z->g;
    /* starting (T1, T2): nearest grid point, clipped, moved to a valid point */
    int32_t a = (int32_t)floor((o->t1_init_ms - g->t1_min) / g->t1_step + 0.5);
    int32_t b = (int32_t)floor((o->t2_init_ms - g->t2_min) / g->t2_step + 0.5);
    if (a < 0) a = 0;
    if (a > g->n_t1 - 1) a = g->n_t1 - 1;
    if (b < 0) b = 0;
    if (b > g->n_t2 - 1) b = g->n_t2 - 1;
    while (b > 0 && !valid_ab(g, a, b)) --b;
    while (a < g->n_t1 - 1 && !valid_ab(g, a, b)) ++a;
    if (!valid_ab(g, a, b)) return -1;

    /* Step 1a: coarse df scan over the whole range with a step below omega. */
    z->stage = 1;
    gap2 m; gap_reset(&m);
    int32_t hA = snap_steps(o->s1a_step_frac * omega, g->df_step);
    double best = -INFINITY; int32_t c = 0;
    for (int32_t cc = 0; cc < g->n_df; cc += hA) {
        double v = zscore(z, a, b, cc);
        gap_add(&m, v);
        if (v > best) { best = v; c = cc; }
    }
    gap_close(z, &m);

    /* Step 1b: window of +-(s1b_half x omega) around it, step s1b_step x omega. */
    z->stage = 2;
    {
        int32_t W = (int32_t)floor(o->s1b_half_frac * omega / g->df_step + 0.5);
        int32_t hB = snap_steps(o->s1b_step_frac * omega, g->df_step);
        int32_t K = W / hB, c0 = c;
        gap_reset(&m); gap_add(&m, best);
        for (int32_t k = -K; k <= K; ++k) {
            if (k == 0) continue;
            int32_t cc = c0 + k * hB;
            if (cc < 0 || cc >= g->n_df) continue;
            double v = zscore(z, a, b, cc);
            gap_add(&m, v);
            if (v > best) { best = v; c = cc; }
        }
        gap_close(z, &m);
    }

    /* Step 1c: probes at every integer multiple of omega from the optimum. */
    z->stage = 3;
    {
        int32_t hC = snap_steps(omega, g->df_step), c0 = c;
        gap_reset(&m); gap_add(&m, best);
        for (int32_t cc = c0 - (c0 / hC) * hC; cc < g->n_df; cc += hC) {
            if (cc == c0) continue;
            double v = zscore(z, a, b, cc);
            gap_add(&m, v);
            if (v > best) { best = v; c = cc; }
        }
        gap_close(z, &m);
    }

    /* Step 2: 2D ZOOM at the coarse resolutions. */
    z->stage = 4;
    int32_t ph1 = -1, ph2 = -1;
    for (int32_t l = 0; l < o->n_s2; ++l) {
        int32_t h1 = snap_steps(o->s2_t1_ms[l], g->t1_step), h2 = snap_steps(o->s2_t2_ms[l], g->t2_step);
        if (h1 == ph1 && h2 == ph2) continue;
        ph1 = h1; ph2 = h2;
        move2d(z, &a, &b, c, &best, h1, h2);
    }

    /* Step 3: finest-step df scan over +-(s3_half x omega). */
    z->stage = 5;
    {
        int32_t W = (int32_t)floor(o->s3_half_frac * omega / g->df_step + 0.5), c0 = c;
        gap_reset(&m); gap_add(&m, best);
        for (int32_t cc = c0 - W; cc <= c0 + W; ++cc) {
            if (cc == c0 || cc < 0 || cc >= g->n_df) continue;
            double v = zscore(z, a, b, cc);
            gap_add(&m, v);
            if (v > best) { best = v; c = cc; }
        }
        gap_close(z, &m);
    }

    /* Step 4: interleaved 1D ZOOMs; consecutive duplicates after snapping are dropped. */
    z->stage = 6;
    int pp = -1; int32_t ph = -1;
    for (int32_t l = 0; l < o->n_s4; ++l) {
        int param = o->s4_param[l];
        int32_t h = snap_steps(o->s4_ms[l], param == 0 ? g->t1_step : g->t2_step);
        if (param == pp && h == ph) continue;
        pp = param; ph = h;
        move1d(z, &a, &b, c, &best, param, h);
    }

    /* Step 5: final 2D ZOOM at the finest resolution. */
    z->stage = 7;
    move2d(z, &a, &b, c, &best, 1, 1);

    *ra = a; *rb = b; *rc = c; *rcc = best;
    return 0;
}

/* ZOOM on an arbitrary score function (test hook). trace may be NULL. */
int or_zoom_generic(const or_grid *g, const or_zoom_opts *o, double omega, or_score_fn fn, void *ctx,
                    int32_t *abc, double *cc, int32_t *evaluated, double *min_margin,
                    int32_t trace_cap, int32_t *trace_n, int32_t *trace, double *trace_cc)
{
    if (!grid_ok(g) || !o || !fn || !(omega > 0.0)) return -1;
    zoom_state z;
    memset(&z, 0, sizeof z);
    z.g = g; z.fn = fn; z.ctx = ctx; z.min_margin = INFINITY;
    z.trace_cap = trace ? trace_cap : 0; z.trace = trace; z.trace_cc = trace_cc;
    int rc = zoom_run(&z, o, omega, &abc[0], &abc[1], &abc[2], cc);
    if (evaluated) *evaluated = z.evaluated;
    if (min_margin) *min_margin = z.min_margin;
    if (trace_n) *trace_n = z.trace_n;
    if (z.guard_hit) return -3;
    return rc;
}

typedef struct {
    const or_seq *s;
    const or_grid *g;
    const double *x;      /* n interleaved */
    double xnorm;
    double *d;            /* scratch, n interleaved */
} cc_ctx;

static double score_cc(void *vctx, int32_t a, int32_t b, int32_t c)
{
    cc_ctx *k = (cc_ctx *)vctx;
    simulate_one(k->s, t1_of(k->g, a), t2_of(k->g, b), df_of(k->g, c), NULL, k->d, NULL);
    double re, im;
    inner(k->s->n, k->x, k->d, &re, &im);
    double nd = sqrt(norm2(k->s->n, k->d));
    if (nd == 0.0 || k->xnorm == 0.0) return 0.0;
    return sqrt(re * re + im * im) / (k->xnorm * nd);
}

double or_default_omega(const or_seq *s)
{
    double mn = INFINITY;
    for (int32_t j = 0; j < s->n; ++j) if (s->tr[j] < mn) mn = s->tr[j];
    return 1000.0 / mn;
}

/* MRF-ZOOM for V voxels (x: V x n interleaved). Outputs per voxel: grid
 * indices (a, b, c), CC, M0, phase, candidates evaluated, smallest decision
 * margin. Voxels are independent; OpenMP over voxels. */
int or_zoom(const or_seq *s, const or_grid *g, const or_zoom_opts *o, const double *x, int64_t V,
            int32_t *abc, double *cc, double *m0, double *phase, int32_t *evaluated, double *min_margin)
{
    if (!s || s->n < 1 || !grid_ok(g) || !o || V < 0) return -1;
    double omega = o->omega_hz > 0.0 ? o->omega_hz : or_default_omega(s);
    const int32_t n = s->n;
    int err = 0;
    #pragma omp parallel
    {
        double *d = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        if (!d) {
            #pragma omp atomic write
            err = -2;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t v = 0; v < V; ++v) {
                cc_ctx k = {s, g, x + (size_t)v * 2 * n, sqrt(norm2(n, x + (size_t)v * 2 * n)), d};
                zoom_state z;
                memset(&z, 0, sizeof z);
                z.g = g; z.fn = score_cc; z.ctx = &k; z.min_margin = INFINITY;
                int32_t *r = abc + 3 * v;
                int rc = zoom_run(&z, o, omega, &r[0], &r[1], &r[2], &cc[v]);
                if (rc != 0 || z.guard_hit) {
                    #pragma omp atomic write
                    err = rc != 0 ? rc : -3;
                    continue;
                }
                evaluated[v] = z.evaluated;
                min_margin[v] = z.min_margin;
                simulate_one(s, t1_of(g, r[0]), t2_of(g, r[1]), df_of(g, r[2]), NULL, d, NULL);
                double re, im;
                inner(n, k.x, d, &re, &im);
                double dd = norm2(n, d);
                if (m0) m0[v] = dd > 0.0 ? sqrt(re * re + im * im) / dd : 0.0;
                if (phase) phase[v] = atan2(im, re);
            }
            free(d);
        }
    }
    return err;
}

/* ------------------------------------------------------------------------- */
/* Windowed refinement. Results (Experiment 2) checks ZOOM answers with a
 * brute-force search in a small window around them; applied repeatedly it is
 * a hill climb on the full grid: compare the centre with the 26 points of its
 * 3 x 3 x 3 neighbourhood (T1 offset outer, then T2, then df; -1 before +1),
 * move to the best of them when it is strictly better than the centre (the
 * first in that order on ties), and stop when the centre wins. The starting
 * centre is evaluated too. Points off the grid or with T2 >= T1 (when the
 * grid requires T2 < T1) are never evaluated. min_margin: the smallest gap
 * between the two largest finite values of a decision set.                 */

static int refine_run(const or_grid *g, or_score_fn fn, void *ctx, int32_t max_moves, int32_t *a, int32_t *b,
                      int32_t *c, double *centre, int32_t *evaluated, double *min_margin)
{
    if (*c < 0 || *c >= g->n_df || !valid_ab(g, *a, *b)) return -1;
    double cv = fn(ctx, *a, *b, *c);
    ++*evaluated;
    int32_t it;
    for (it = 0; it < max_moves; ++it) {
        double t1 = cv, t2 = -INFINITY, best = -INFINITY;
        int32_t ba = *a, bb = *b, bc = *c;
        for (int da = -1; da <= 1; ++da)
            for (int db = -1; db <= 1; ++db)
                for (int dc = -1; dc <= 1; ++dc) {
                    if (da == 0 && db == 0 && dc == 0) continue;
                    const int32_t na = *a + da, nb = *b + db, nc = *c + dc;
                    if (nc < 0 || nc >= g->n_df || !valid_ab(g, na, nb)) continue;
                    const double v = fn(ctx, na, nb, nc);
                    ++*evaluated;
                    if (v > t1) { t2 = t1; t1 = v; } else if (v > t2) t2 = v;
                    if (v > best) { best = v; ba = na; bb = nb; bc = nc; }
                }
        if (isfinite(t2) && t1 - t2 < *min_margin) *min_margin = t1 - t2;
        if (!(best > cv)) break;
        *a = ba; *b = bb; *c = bc; cv = best;
    }
    *centre = cv;
    return it < max_moves ? 0 : -3;
}

/* Refinement on an arbitrary score function (test hook). abc: in/out. */
int or_refine_generic(const or_grid *g, int32_t max_moves, or_score_fn fn, void *ctx, int32_t *abc, double *cc,
                      int32_t *evaluated, double *min_margin)
{
    if (!grid_ok(g) || !fn || max_moves < 0) return -1;
    int32_t ev = 0;
    double mm = INFINITY;
    int rc = refine_run(g, fn, ctx, max_moves, &abc[0], &abc[1], &abc[2], cc, &ev, &mm);
    if (evaluated) *evaluated = ev;
    if (min_margin) *min_margin = mm;
    return rc;
}

/* Refinement for V voxels (x: V x n interleaved) from the starting points in
 * abc (V x 3, in/out). Outputs per voxel: CC, M0, phase of the final point,
 * candidates evaluated, smallest decision margin (+inf when no decision had
 * two finite values). OpenMP over voxels. */
int or_refine(const or_seq *s, const or_grid *g, const double *x, int64_t V, int32_t max_moves, int32_t *abc,
              double *cc, double *m0, double *phase, int32_t *evaluated, double *min_margin)
{
    if (!s || s->n < 1 || !grid_ok(g) || V < 0 || max_moves < 0) return -1;
    const int32_t n = s->n;
    int err = 0;
    #pragma omp parallel
    {
        double *d = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        if (!d) {
            #pragma omp atomic write
            err = -2;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t v = 0; v < V; ++v) {
                cc_ctx k = {s, g, x + (size_t)v * 2 * n, sqrt(norm2(n, x + (size_t)v * 2 * n)), d};
                int32_t *r = abc + 3 * v;
                int32_t ev = 0;
                double mm = INFINITY;
                int rc = refine_run(g, score_cc, &k, max_moves, &r[0], &r[1], &r[2], &cc[v], &ev, &mm);
                if (rc != 0) {
                    #pragma omp atomic write
                    err = rc;
                    continue;
                }
                evaluated[v] = ev;
                min_margin[v] = mm;
                simulate_one(s, t1_of(g, r[0]), t2_of(g, r[1]), df_of(g, r[2]), NULL, d, NULL);
                double re, im;
                inner(n, k.x, d, &re, &im);
                double dd = norm2(n, d);
                if (m0) m0[v] = dd > 0.0 ? sqrt(re * re + im * im) / dd : 0.0;
                if (phase) phase[v] = atan2(im, re);
            }
            free(d);
        }
    }
    return err;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
