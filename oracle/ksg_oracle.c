/*
 * ksg_oracle.c -- CPU oracle for the KSG conditional-mutual-information path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the GPU library computes.  Only the tests, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it follows (the paper is the IDTxl software paper, arXiv 1807.10459):
 *   - Summary, paragraph 6: the nonlinear estimator of Kraskov, Stoegbauer and
 *     Grassberger (2004) for (conditional) mutual information.  The paper
 *     prints no formula; the estimator used here is KSG "algorithm 1" in its
 *     conditional form (a reading, listed in the design notes):
 *         I(X;Y|Z) = psi(k) + (1/N) sum_i [ psi(n_z+1) - psi(n_xz+1) - psi(n_yz+1) ]
 *     with eps_i the k-th smallest joint max-norm distance over j != i and
 *     n_S the number of j != i whose max-norm distance in subspace S is
 *     strictly smaller than eps_i.  Result in nats.
 *   - Summary, paragraph 4: surrogate null distributions gate the greedy
 *     parent selection and stop it.  Surrogates permute the rows of X
 *     (a reading); the gate is the maximum statistic over candidates.
 *
 * Arithmetic: distances are fp32 (|a-b| in round-to-nearest, then max), the
 * digamma values and all sums are computed in long double / double.  Build
 * without -ffast-math and with -ffp-contract=off.
 *
 * Parity status of each function (what pins it) is stated in its comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Digamma at positive integers.                                             */
/* Definition: psi(1) = -gamma (Euler-Mascheroni), psi(n+1) = psi(n) + 1/n.  */
/* Pinned by: scipy.special.digamma at integers; psi(1) = -gamma.            */
/* ------------------------------------------------------------------------ */
static const long double ORC_EULER_GAMMA = 0.577215664901532860606512090082402431L;

/* out[0] is set to NaN (psi has a pole at 0); out[n] = psi(n) for 1 <= n <= n_max. */
int orc_psi_table(int64_t n_max, double *out)
{
    if (n_max < 1 || out == NULL) return -1;
    long double acc = -ORC_EULER_GAMMA;
    out[0] = NAN;
    for (int64_t n = 1; n <= n_max; ++n) {
        out[n] = (double)acc;
        acc += 1.0L / (long double)n;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Max-norm distances between samples i and j in a block of columns.       */
/* Columns are stored one after another with leading dimension ld:          */
/* value of dimension d at sample t is col[d*ld + t].  dim == 0 gives 0.     */
/* ------------------------------------------------------------------------ */
static float orc_maxnorm(const float *col, int dim, int64_t ld, int64_t i, int64_t j)
{
    float m = 0.0f;
    for (int d = 0; d < dim; ++d) {
        float a = col[(int64_t)d * ld + i];
        float b = col[(int64_t)d * ld + j];
        float v = fabsf(a - b);
        if (v > m) m = v;
    }
    return m;
}

static float orc_max2(float a, float b) { return a > b ? a : b; }

/* ------------------------------------------------------------------------ */
/* KSG neighbour statistics of one estimate.                                 */
/*   eps[i]  = k-th smallest of { max(dX,dY,dZ)(i,j) : j != i }              */
/*   nxz[i]  = #{ j != i : max(dX,dZ)(i,j) < eps[i] }                        */
/*   nyz[i]  = #{ j != i : max(dY,dZ)(i,j) < eps[i] }                        */
/*   nz[i]   = #{ j != i : dZ(i,j)        < eps[i] }   (dz == 0: dZ = 0)     */
/* Pinned by: the hand-worked N=6 example, an independent numpy brute force, */
/* the X<->Y swap, sample-reordering and power-of-two scaling invariants.    */
/* Returns 0, or -1 on bad arguments.                                        */
/* ------------------------------------------------------------------------ */
/* Statistics of one query i; best[] is scratch for k floats. */
static void orc_ksg_query(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                          int64_t n, int64_t ld, int k, int64_t i, float *best, float *eps,
                          int32_t *nxz, int32_t *nyz, int32_t *nz)
{
    /* pass 1: the k smallest joint distances, kept sorted ascending */
    for (int m = 0; m < k; ++m) best[m] = INFINITY;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        float d = orc_max2(orc_maxnorm(x, dx, ld, i, j),
                           orc_max2(orc_maxnorm(y, dy, ld, i, j), orc_maxnorm(z, dz, ld, i, j)));
        if (d < best[k - 1]) {
            int m = k - 1;
            while (m > 0 && best[m - 1] > d) {
                best[m] = best[m - 1];
                --m;
            }
            best[m] = d;
        }
    }
    float e = best[k - 1];
    *eps = e;
    /* pass 2: strict-radius counts in the three subspaces */
    int32_t cxz = 0, cyz = 0, cz = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        float ddx = orc_maxnorm(x, dx, ld, i, j);
        float ddy = orc_maxnorm(y, dy, ld, i, j);
        float ddz = orc_maxnorm(z, dz, ld, i, j);
        if (orc_max2(ddx, ddz) < e) ++cxz;
        if (orc_max2(ddy, ddz) < e) ++cyz;
        if (ddz < e) ++cz;
    }
    *nxz = cxz;
    *nyz = cyz;
    *nz = cz;
}

static int orc_args_ok(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                       int64_t n, int64_t ld, int k)
{
    if (n < 2 || k < 1 || k > n - 1 || dx < 1 || dy < 1 || dz < 0 || ld < n) return 0;
    if (!x || !y || (dz > 0 && !z)) return 0;
    return 1;
}

int orc_ksg_counts(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                   int64_t n, int64_t ld, int k, float *eps, int32_t *nxz, int32_t *nyz,
                   int32_t *nz)
{
    if (!orc_args_ok(x, dx, y, dy, z, dz, n, ld, k) || !eps || !nxz || !nyz || !nz) return -1;
#pragma omp parallel
    {
        float *best = (float *)malloc(sizeof(float) * (size_t)k);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            orc_ksg_query(x, dx, y, dy, z, dz, n, ld, k, i, best, &eps[i], &nxz[i], &nyz[i],
                          &nz[i]);
        free(best);
    }
    return 0;
}

/* The same statistics for the m queries listed in idx (outputs indexed 0..m-1). */
int orc_ksg_counts_at(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                      int64_t n, int64_t ld, int k, const int64_t *idx, int64_t m, float *eps,
                      int32_t *nxz, int32_t *nyz, int32_t *nz)
{
    if (!orc_args_ok(x, dx, y, dy, z, dz, n, ld, k) || !idx || m < 0 || !eps || !nxz || !nyz ||
        !nz)
        return -1;
    for (int64_t q = 0; q < m; ++q)
        if (idx[q] < 0 || idx[q] >= n) return -1;
#pragma omp parallel
    {
        float *best = (float *)malloc(sizeof(float) * (size_t)k);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < m; ++q)
            orc_ksg_query(x, dx, y, dy, z, dz, n, ld, k, idx[q], best, &eps[q], &nxz[q], &nyz[q],
                          &nz[q]);
        free(best);
    }
    return 0;
}

/* The estimate from its counts: psi(k) + mean_i[psi(nz+1) - psi(nxz+1) - psi(nyz+1)].
 * psi is the table from orc_psi_table covering index n (counts are <= n-1). */
double orc_cmi_from_counts(const int32_t *nxz, const int32_t *nyz, const int32_t *nz, int64_t n,
                           int k, const double *psi)
{
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i)
        sum += psi[nz[i] + 1] - psi[nxz[i] + 1] - psi[nyz[i] + 1];
    return psi[k] + sum / (double)n;
}

/* One KSG CMI estimate I(X;Y|Z) in nats.  Optional outputs may be NULL.
 * Returns 0 or -1. */
int orc_cmi_ksg(const float *x, int dx, const float *y, int dy, const float *z, int dz, int64_t n,
                int64_t ld, int k, double *cmi, float *eps_out, int32_t *counts_out)
{
    if (n < 2 || !cmi) return -1;
    float *eps = eps_out ? eps_out : (float *)malloc(sizeof(float) * (size_t)n);
    int32_t *cnt = counts_out ? counts_out : (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)n);
    double *psi = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    int rc = orc_ksg_counts(x, dx, y, dy, z, dz, n, ld, k, eps, cnt, cnt + n, cnt + 2 * n);
    if (rc == 0) {
        orc_psi_table(n, psi);
        *cmi = orc_cmi_from_counts(cnt, cnt + n, cnt + 2 * n, n, k, psi);
    }
    free(psi);
    if (!eps_out) free(eps);
    if (!counts_out) free(cnt);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Surrogate permutations (a reading: the paper only says "surrogates").     */
/*                                                                           */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by      */
/* 0x9E3779B97F4A7C15 and each output is the state passed through the mixer  */
/*   z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB; */
/*   z ^= z>>31.                                                             */
/* Pinned by: the generator's published output sequence for seed 1234567.    */
/*                                                                           */
/* The permutation of [0,n) keyed by (seed, stream) is the Fisher-Yates      */
/* (Durstenfeld) shuffle of the identity driven by SplitMix64 started from   */
/* the state seed ^ mix(stream): for i = n-1 down to 1, draw r and swap      */
/* a[i] with a[j], j = floor(r * (i+1) / 2^64) (the high word of the 128-bit */
/* product).  pi = a.                                                        */
/* Pinned by: bijection on many n, chi-square uniformity of positions.       */
/* ------------------------------------------------------------------------ */
static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n outputs of SplitMix64 from the given initial state. */
void orc_splitmix64(uint64_t state, int n, uint64_t *out)
{
    for (int t = 0; t < n; ++t) {
        state += 0x9E3779B97F4A7C15ULL;
        out[t] = orc_mix64(state);
    }
}

/* out[i] = pi(i) for 0 <= i < n. */
int orc_perm(uint64_t seed, uint64_t stream, int64_t n, int64_t *out)
{
    if (n < 1 || !out) return -1;
    uint64_t state = seed ^ orc_mix64(stream);
    for (int64_t i = 0; i < n; ++i) out[i] = i;
    for (int64_t i = n - 1; i >= 1; --i) {
        state += 0x9E3779B97F4A7C15ULL;
        uint64_t r = orc_mix64(state);
        int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
        int64_t t = out[i];
        out[i] = out[j];
        out[j] = t;
    }
    return 0;
}

/* Surrogate columns: xs[d*ld + i] = x[d*ld + pi(i)] for every X dimension. */
static void orc_permute_rows(const float *x, int dx, int64_t n, int64_t ld, const int64_t *pi,
                             float *xs)
{
    for (int d = 0; d < dx; ++d)
        for (int64_t i = 0; i < n; ++i) xs[(int64_t)d * ld + i] = x[(int64_t)d * ld + pi[i]];
}

/* One estimate plus n_surr surrogates: out[0] = I(X;Y|Z), out[1+s] = the
 * estimate with X's rows permuted by the permutation keyed (seed, stream = s).
 * Returns 0 or -1. */
int orc_cmi_surrogates(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                       int64_t n, int64_t ld, int k, int n_surr, uint64_t seed, double *out)
{
    if (n_surr < 0 || !out) return -1;
    if (orc_cmi_ksg(x, dx, y, dy, z, dz, n, ld, k, &out[0], NULL, NULL) != 0) return -1;
    float *xs = (float *)malloc(sizeof(float) * (size_t)dx * (size_t)ld);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int rc = 0;
    for (int s = 0; s < n_surr && rc == 0; ++s) {
        orc_perm(seed, (uint64_t)s, n, pi);
        orc_permute_rows(x, dx, n, ld, pi, xs);
        rc = orc_cmi_ksg(xs, dx, y, dy, z, dz, n, ld, k, &out[1 + s], NULL, NULL);
    }
    free(xs);
    free(pi);
    return rc;
}

/* Replication-level surrogates (a reading of the surrogates the Summary     */
/* mentions, for data made of n_reps replications of len = n / n_reps        */
/* consecutive samples): surrogate s moves whole replications of X,          */
/* X_s[r*len + t] = X[pi_s(r)*len + t], pi_s the permutation of [0, n_reps)  */
/* keyed (seed, stream = s) as above; Y and Z stay.                          */
/* Pinned by: with n_reps = n (one sample per replication) it is the         */
/* sample-level orc_cmi_surrogates exactly.                                  */
int orc_cmi_surrogates_reps(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                            int64_t n, int64_t ld, int k, int n_surr, uint64_t seed, int64_t n_reps,
                            double *out)
{
    if (n_surr < 0 || !out || n_reps < 1 || n % n_reps != 0) return -1;
    if (orc_cmi_ksg(x, dx, y, dy, z, dz, n, ld, k, &out[0], NULL, NULL) != 0) return -1;
    const int64_t len = n / n_reps;
    float *xs = (float *)malloc(sizeof(float) * (size_t)dx * (size_t)ld);
    int64_t *pr = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_reps);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int rc = 0;
    for (int s = 0; s < n_surr && rc == 0; ++s) {
        orc_perm(seed, (uint64_t)s, n_reps, pr);
        for (int64_t i = 0; i < n; ++i) pi[i] = pr[i / len] * len + i % len;
        orc_permute_rows(x, dx, n, ld, pi, xs);
        rc = orc_cmi_ksg(xs, dx, y, dy, z, dz, n, ld, k, &out[1 + s], NULL, NULL);
    }
    free(xs);
    free(pr);
    free(pi);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Greedy parent selection for one target with max-statistic gating         */
/* (Summary, paragraph 4: parents are added by maximising a CMI criterion;   */
/* surrogate tests gate each addition and stop the loop; paragraph 3: the    */
/* test must control errors from testing many sources).  Readings:          */
/*   - samples t in [L, T), L = max(max_lag, n_past); N = T - L;            */
/*   - Y[i] = series[target][L+i]; target past = lags 1..n_past of target;  */
/*   - candidates (p, lag), p in [0,n_proc), lag in [min_lag, max_lag],      */
/*     without the target-past variables; candidate id                       */
/*     c = p*(max_lag-min_lag+1) + (lag-min_lag);                           */
/*   - T_obs = max_c I(X_c;Y|Z), ties to the lowest c;                      */
/*   - T_s = max_c I(X_c o pi_{step,c,s}; Y|Z), stream = step<<48|c<<24|s;  */
/*   - p = #{s : T_s >= T_obs} / S; significant iff p < alpha.              */
/* Pinned by: a strongly coupled VAR recovers its true parents; tiny cases   */
/* checked against a brute-force gate in the tests.                          */
/* ------------------------------------------------------------------------ */
static void orc_gather_lag(const float *series, int64_t T, int p, int lag, int64_t L, float *col)
{
    int64_t n = T - L;
    for (int64_t i = 0; i < n; ++i) col[i] = series[(int64_t)p * T + L + i - lag];
}

/* Per-step record written by orc_select_target. */
typedef struct {
    int32_t cand;     /* candidate id of the step's maximiser (-1: no candidate) */
    int32_t significant;
    double stat;      /* T_obs */
    double pval;
} orc_step;

/* est_out (nullable): [n_cand_total][1+n_surr] estimates of the FIRST step,
 * indexed by candidate id (rows of excluded candidates are left untouched). */
int orc_select_target(const float *series, int n_proc, int64_t T, int target, int n_past,
                      int min_lag, int max_lag, int k, int n_surr, double alpha, uint64_t seed,
                      int max_parents, orc_step *steps, int *n_steps, int32_t *parents,
                      int *n_parents, double *est_out)
{
    if (!series || n_proc < 1 || target < 0 || target >= n_proc || n_past < 0 || min_lag < 1 ||
        max_lag < min_lag || k < 1 || n_surr < 1 || max_parents < 0 || !steps || !n_steps ||
        !parents || !n_parents)
        return -1;
    int n_lags = max_lag - min_lag + 1;
    int n_cand_total = n_proc * n_lags;
    int64_t L = max_lag > n_past ? max_lag : n_past;
    if (T - L < (int64_t)k + 1) return -1;
    int64_t n = T - L;

    int *alive = (int *)calloc((size_t)n_cand_total, sizeof(int));
    for (int p = 0; p < n_proc; ++p)
        for (int lag = min_lag; lag <= max_lag; ++lag)
            alive[p * n_lags + (lag - min_lag)] = !(p == target && lag <= n_past);

    int dz_max = n_past + max_parents;
    float *y = (float *)malloc(sizeof(float) * (size_t)n);
    float *z = (float *)malloc(sizeof(float) * (size_t)n * (size_t)(dz_max > 0 ? dz_max : 1));
    float *xc = (float *)malloc(sizeof(float) * (size_t)n);
    float *xs = (float *)malloc(sizeof(float) * (size_t)n);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *est = (double *)malloc(sizeof(double) * (size_t)n_cand_total * (size_t)(1 + n_surr));
    orc_gather_lag(series, T, target, 0, L, y);
    int dz = 0;
    for (int lag = 1; lag <= n_past; ++lag) orc_gather_lag(series, T, target, lag, L, z + (int64_t)dz++ * n);

    int np = 0, ns = 0, rc = 0;
    for (int step = 0; step <= max_parents && rc == 0; ++step) {
        int any = 0;
        for (int c = 0; c < n_cand_total; ++c) any |= alive[c];
        if (!any || step == max_parents) break;
        for (int c = 0; c < n_cand_total && rc == 0; ++c) {
            if (!alive[c]) continue;
            int p = c / n_lags, lag = min_lag + c % n_lags;
            orc_gather_lag(series, T, p, lag, L, xc);
            double *row = est + (int64_t)c * (1 + n_surr);
            rc |= orc_cmi_ksg(xc, 1, y, 1, z, dz, n, n, k, &row[0], NULL, NULL);
            for (int s = 0; s < n_surr && rc == 0; ++s) {
                uint64_t stream = ((uint64_t)step << 48) | ((uint64_t)c << 24) | (uint64_t)s;
                orc_perm(seed, stream, n, pi);
                orc_permute_rows(xc, 1, n, n, pi, xs);
                rc |= orc_cmi_ksg(xs, 1, y, 1, z, dz, n, n, k, &row[1 + s], NULL, NULL);
            }
        }
        if (rc) break;
        if (step == 0 && est_out)
            for (int c = 0; c < n_cand_total; ++c)
                if (alive[c])
                    memcpy(est_out + (int64_t)c * (1 + n_surr), est + (int64_t)c * (1 + n_surr),
                           sizeof(double) * (size_t)(1 + n_surr));
        /* maximum statistic */
        int best = -1;
        double t_obs = -INFINITY;
        for (int c = 0; c < n_cand_total; ++c)
            if (alive[c] && est[(int64_t)c * (1 + n_surr)] > t_obs) {
                t_obs = est[(int64_t)c * (1 + n_surr)];
                best = c;
            }
        int count = 0;
        for (int s = 0; s < n_surr; ++s) {
            double t_s = -INFINITY;
            for (int c = 0; c < n_cand_total; ++c)
                if (alive[c] && est[(int64_t)c * (1 + n_surr) + 1 + s] > t_s)
                    t_s = est[(int64_t)c * (1 + n_surr) + 1 + s];
            if (t_s >= t_obs) ++count;
        }
        double pval = (double)count / (double)n_surr;
        int sig = pval < alpha;
        steps[ns].cand = best;
        steps[ns].significant = sig;
        steps[ns].stat = t_obs;
        steps[ns].pval = pval;
        ++ns;
        if (!sig) break;
        parents[np++] = best;
        alive[best] = 0;
        orc_gather_lag(series, T, best / n_lags, min_lag + best % n_lags, L, z + (int64_t)dz++ * n);
    }
    *n_steps = ns;
    *n_parents = np;
    free(alive);
    free(y);
    free(z);
    free(xc);
    free(xs);
    free(pi);
    free(est);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Non-uniform target past (the Summary says the greedy conditioning builds  */
/* a non-uniform embedding; how the target's own past is chosen is a         */
/* reading): the past is selected first by the same greedy max-statistic    */
/* loop restricted to the target's own variables (target, lag), lag in      */
/* [min_lag, max_lag], with Z = the past lags chosen so far (step s uses     */
/* stream (0xD000+s)<<48 | c<<24 | i); then the sources are selected with Z  */
/* starting from that past (candidates: every variable not in the past;     */
/* step s uses stream s<<48 | c<<24 | i).  Samples t in [max_lag, T).        */
/* Pinned by: source selection from the past (target, 1..n_past) reproduces */
/* orc_select_target(n_past) exactly (an independent implementation of the  */
/* same loop); the past of an AR(2) target is its lags 1 and 2.             */
/* ------------------------------------------------------------------------ */
static int orc_greedy(const float *series, int n_proc, int64_t T, int target, int min_lag,
                      int max_lag, const int32_t *init_ids, int n_init, const char *allowed,
                      uint64_t step_base, int k, int n_surr, double alpha, uint64_t seed,
                      int max_sel, orc_step *steps, int *n_steps, int32_t *sel, int *n_sel)
{
    const int n_lags = max_lag - min_lag + 1, n_all = n_proc * n_lags;
    const int64_t L = max_lag, n = T - L;
    char *open_c = (char *)malloc((size_t)n_all);
    for (int c = 0; c < n_all; ++c) open_c[c] = allowed[c];
    for (int i = 0; i < n_init; ++i) open_c[init_ids[i]] = 0;
    float *y = (float *)malloc(sizeof(float) * (size_t)n);
    float *z = (float *)malloc(sizeof(float) * (size_t)n * (size_t)(n_init + max_sel + 1));
    float *x = (float *)malloc(sizeof(float) * (size_t)n);
    float *xp = (float *)malloc(sizeof(float) * (size_t)n);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *row = (double *)malloc(sizeof(double) * (size_t)n_all * (size_t)(1 + n_surr));
    orc_gather_lag(series, T, target, 0, L, y);
    int dz = 0;
    for (int i = 0; i < n_init; ++i)
        orc_gather_lag(series, T, init_ids[i] / n_lags, min_lag + init_ids[i] % n_lags, L,
                       z + (int64_t)dz++ * n);
    int rc = 0, ns = 0, nsel = 0;
    while (rc == 0 && nsel < max_sel) {
        int left = 0;
        for (int c = 0; c < n_all; ++c) left += open_c[c];
        if (!left) break;
        const uint64_t step = step_base + (uint64_t)ns;
        for (int c = 0; c < n_all && rc == 0; ++c) {
            if (!open_c[c]) continue;
            orc_gather_lag(series, T, c / n_lags, min_lag + c % n_lags, L, x);
            double *r = row + (int64_t)c * (1 + n_surr);
            rc |= orc_cmi_ksg(x, 1, y, 1, z, dz, n, n, k, &r[0], NULL, NULL);
            for (int i = 0; i < n_surr && rc == 0; ++i) {
                orc_perm(seed, (step << 48) | ((uint64_t)c << 24) | (uint64_t)i, n, pi);
                orc_permute_rows(x, 1, n, n, pi, xp);
                rc |= orc_cmi_ksg(xp, 1, y, 1, z, dz, n, n, k, &r[1 + i], NULL, NULL);
            }
        }
        if (rc) break;
        int best = -1;
        for (int c = 0; c < n_all; ++c)
            if (open_c[c] && (best < 0 || row[(int64_t)c * (1 + n_surr)] > row[(int64_t)best * (1 + n_surr)]))
                best = c;
        const double t_obs = row[(int64_t)best * (1 + n_surr)];
        int count = 0;
        for (int i = 0; i < n_surr; ++i) {
            double t_i = -INFINITY;
            for (int c = 0; c < n_all; ++c)
                if (open_c[c] && row[(int64_t)c * (1 + n_surr) + 1 + i] > t_i)
                    t_i = row[(int64_t)c * (1 + n_surr) + 1 + i];
            count += t_i >= t_obs;
        }
        steps[ns].cand = best;
        steps[ns].stat = t_obs;
        steps[ns].pval = (double)count / (double)n_surr;
        steps[ns].significant = steps[ns].pval < alpha;
        if (!steps[ns++].significant) break;
        sel[nsel++] = best;
        open_c[best] = 0;
        orc_gather_lag(series, T, best / n_lags, min_lag + best % n_lags, L, z + (int64_t)dz++ * n);
    }
    *n_steps = ns;
    *n_sel = nsel;
    free(open_c);
    free(y);
    free(z);
    free(x);
    free(xp);
    free(pi);
    free(row);
    return rc;
}

/* The target's past: ids of (target, lag) in selection order. */
int orc_select_past(const float *series, int n_proc, int64_t T, int target, int min_lag,
                    int max_lag, int k, int n_surr, double alpha, uint64_t seed, int max_past,
                    orc_step *steps, int *n_steps, int32_t *past, int *n_past)
{
    if (!series || n_proc < 1 || target < 0 || target >= n_proc || min_lag < 1 ||
        max_lag < min_lag || k < 1 || n_surr < 1 || max_past < 0 || !steps || !n_steps ||
        !past || !n_past || T - max_lag < (int64_t)k + 1)
        return -1;
    const int n_lags = max_lag - min_lag + 1;
    char *allowed = (char *)calloc((size_t)(n_proc * n_lags), 1);
    for (int c = target * n_lags; c < (target + 1) * n_lags; ++c) allowed[c] = 1;
    int rc = orc_greedy(series, n_proc, T, target, min_lag, max_lag, NULL, 0, allowed, 0xD000,
                        k, n_surr, alpha, seed, max_past, steps, n_steps, past, n_past);
    free(allowed);
    return rc;
}

/* Sources given a past (candidate ids, in order; the past is Z's first columns). */
int orc_select_sources(const float *series, int n_proc, int64_t T, int target,
                       const int32_t *past, int n_past_ids, int min_lag, int max_lag, int k,
                       int n_surr, double alpha, uint64_t seed, int max_parents, orc_step *steps,
                       int *n_steps, int32_t *parents, int *n_parents)
{
    if (!series || n_proc < 1 || target < 0 || target >= n_proc || min_lag < 1 ||
        max_lag < min_lag || k < 1 || n_surr < 1 || max_parents < 0 || n_past_ids < 0 ||
        (n_past_ids > 0 && !past) || !steps || !n_steps || !parents || !n_parents ||
        T - max_lag < (int64_t)k + 1)
        return -1;
    const int n_all = n_proc * (max_lag - min_lag + 1);
    for (int i = 0; i < n_past_ids; ++i)
        if (past[i] < 0 || past[i] >= n_all) return -1;
    char *allowed = (char *)malloc((size_t)n_all);
    memset(allowed, 1, (size_t)n_all);
    int rc = orc_greedy(series, n_proc, T, target, min_lag, max_lag, past, n_past_ids, allowed, 0,
                        k, n_surr, alpha, seed, max_parents, steps, n_steps, parents, n_parents);
    free(allowed);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Tests after the greedy selection (Summary, paragraph 3: the errors of     */
/* testing many sources must be controlled; the paper describes no test).    */
/* Readings, for a target, its past Z0 (lags 1..n_past) and a selected       */
/* parent list P = (c_0, ..., c_{m-1}) of candidate ids:                     */
/*   - leave-one-out statistic of parent i:                                  */
/*       T_i = I(X_{c_i}; Y | Z0, X_{c_j} for j != i, in list order),        */
/*     its surrogate s permutes X_{c_i} with stream tag | c_i<<24 | s;       */
/*   - pruning (minimum statistic): T_min = min_i T_i (ties: lowest i),      */
/*     p = #{s : min_i T_i,s >= T_min} / S; if p >= alpha the parent at the  */
/*     minimum is removed and the test repeats on the rest (round r uses     */
/*     tag 0x9000+r in the top 16 bits); it stops at the first significant   */
/*     round or when no parent is left;                                      */
/*   - omnibus: T = I(X_P; Y | Z0) with X_P all selected parents jointly;    */
/*     surrogate s permutes the rows of X_P (one permutation for all its     */
/*     columns), stream 0xA000<<48 | 0xFFFFFF<<24 | s; p = #{s : T_s >= T}/S;*/
/*   - sequential maximum statistic: parents in decreasing order of T_i      */
/*     (ties: lowest i first), tag 0xB000; the r-th is tested against the    */
/*     surrogate maxima over itself and the parents after it,                */
/*     p_r = #{s : max_{j at or after r} T_j,s >= T_(r)} / S; parents are    */
/*     significant down to the first p_r >= alpha, none after it.            */
/* Pinned by: an independent noise source added to true parents is pruned   */
/* and the true parents kept; the omnibus test of true parents is            */
/* significant and of independent noise is not; with one parent the three   */
/* statistics equal the greedy step's estimate of that candidate; a test     */
/* rebuilds every round, statistic and decision from orc_cmi_ksg and the     */
/* shuffle by the rules above.                                               */
/* ------------------------------------------------------------------------ */
#define ORC_TAG_PRUNE 0x9000u
#define ORC_TAG_OMNIBUS 0xA000u
#define ORC_TAG_SEQMAX 0xB000u

static int orc_post_args_ok(const float *series, int n_proc, int64_t T, int target, int n_past,
                            int min_lag, int max_lag, const int32_t *parents, int m, int k,
                            int n_surr)
{
    if (!series || n_proc < 1 || target < 0 || target >= n_proc || n_past < 0 || min_lag < 1 ||
        max_lag < min_lag || k < 1 || n_surr < 1 || m < 1 || !parents)
        return 0;
    int n_lags = max_lag - min_lag + 1;
    for (int i = 0; i < m; ++i)
        if (parents[i] < 0 || parents[i] >= n_proc * n_lags) return 0;
    int64_t L = max_lag > n_past ? max_lag : n_past;
    return T - L >= (int64_t)k + 1;
}

/* est[i*(1+S) + 0] = T_i, est[i*(1+S) + 1 + s] = its surrogate s. */
static int orc_loo_estimates(const float *series, int n_proc, int64_t T, int target, int n_past,
                             int min_lag, int max_lag, const int32_t *parents, int m, int k,
                             int n_surr, uint64_t seed, uint64_t tag, double *est)
{
    (void)n_proc;
    int n_lags = max_lag - min_lag + 1;
    int64_t L = max_lag > n_past ? max_lag : n_past;
    int64_t n = T - L;
    int dz = n_past + m - 1;
    float *y = (float *)malloc(sizeof(float) * (size_t)n);
    float *z = (float *)malloc(sizeof(float) * (size_t)n * (size_t)(dz > 0 ? dz : 1));
    float *xc = (float *)malloc(sizeof(float) * (size_t)n);
    float *xs = (float *)malloc(sizeof(float) * (size_t)n);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    orc_gather_lag(series, T, target, 0, L, y);
    int rc = 0;
    for (int i = 0; i < m && rc == 0; ++i) {
        int d = 0;
        for (int lag = 1; lag <= n_past; ++lag) orc_gather_lag(series, T, target, lag, L, z + (int64_t)d++ * n);
        for (int j = 0; j < m; ++j)
            if (j != i)
                orc_gather_lag(series, T, parents[j] / n_lags, min_lag + parents[j] % n_lags, L,
                               z + (int64_t)d++ * n);
        int c = parents[i];
        orc_gather_lag(series, T, c / n_lags, min_lag + c % n_lags, L, xc);
        double *row = est + (int64_t)i * (1 + n_surr);
        rc |= orc_cmi_ksg(xc, 1, y, 1, z, dz, n, n, k, &row[0], NULL, NULL);
        for (int s = 0; s < n_surr && rc == 0; ++s) {
            uint64_t stream = (tag << 48) | ((uint64_t)c << 24) | (uint64_t)s;
            orc_perm(seed, stream, n, pi);
            orc_permute_rows(xc, 1, n, n, pi, xs);
            rc |= orc_cmi_ksg(xs, 1, y, 1, z, dz, n, n, k, &row[1 + s], NULL, NULL);
        }
    }
    free(y);
    free(z);
    free(xc);
    free(xs);
    free(pi);
    return rc;
}

/* Pruning.  kept[0..n_kept) = surviving parents in their original order;
 * rounds[r] = (cand removed or kept at the minimum, significant, T_min, p). */
int orc_prune(const float *series, int n_proc, int64_t T, int target, int n_past, int min_lag,
              int max_lag, const int32_t *parents, int n_parents, int k, int n_surr, double alpha,
              uint64_t seed, int32_t *kept, int *n_kept, orc_step *rounds, int *n_rounds)
{
    if (!orc_post_args_ok(series, n_proc, T, target, n_past, min_lag, max_lag, parents, n_parents,
                          k, n_surr) ||
        !kept || !n_kept || !rounds || !n_rounds)
        return -1;
    int m = n_parents;
    memcpy(kept, parents, sizeof(int32_t) * (size_t)m);
    double *est = (double *)malloc(sizeof(double) * (size_t)m * (size_t)(1 + n_surr));
    int r = 0, rc = 0;
    while (m > 0) {
        rc = orc_loo_estimates(series, n_proc, T, target, n_past, min_lag, max_lag, kept, m, k,
                               n_surr, seed, ORC_TAG_PRUNE + (uint64_t)r, est);
        if (rc) break;
        int at = 0;
        for (int i = 1; i < m; ++i)
            if (est[(int64_t)i * (1 + n_surr)] < est[(int64_t)at * (1 + n_surr)]) at = i;
        double t_min = est[(int64_t)at * (1 + n_surr)];
        int count = 0;
        for (int s = 0; s < n_surr; ++s) {
            double mn = INFINITY;
            for (int i = 0; i < m; ++i) {
                double v = est[(int64_t)i * (1 + n_surr) + 1 + s];
                if (v < mn) mn = v;
            }
            if (mn >= t_min) ++count;
        }
        double pval = (double)count / (double)n_surr;
        int sig = pval < alpha;
        rounds[r].cand = kept[at];
        rounds[r].significant = sig;
        rounds[r].stat = t_min;
        rounds[r].pval = pval;
        ++r;
        if (sig) break;
        for (int i = at; i + 1 < m; ++i) kept[i] = kept[i + 1];
        --m;
    }
    free(est);
    *n_kept = m;
    *n_rounds = r;
    return rc;
}

/* Omnibus test of the whole parent set. */
int orc_omnibus(const float *series, int n_proc, int64_t T, int target, int n_past, int min_lag,
                int max_lag, const int32_t *parents, int n_parents, int k, int n_surr,
                double alpha, uint64_t seed, double *stat, double *pval, int *significant)
{
    if (!orc_post_args_ok(series, n_proc, T, target, n_past, min_lag, max_lag, parents, n_parents,
                          k, n_surr) ||
        !stat || !pval || !significant)
        return -1;
    int n_lags = max_lag - min_lag + 1;
    int64_t L = max_lag > n_past ? max_lag : n_past;
    int64_t n = T - L;
    int m = n_parents;
    float *y = (float *)malloc(sizeof(float) * (size_t)n);
    float *z = (float *)malloc(sizeof(float) * (size_t)n * (size_t)(n_past > 0 ? n_past : 1));
    float *x = (float *)malloc(sizeof(float) * (size_t)n * (size_t)m);
    float *xs = (float *)malloc(sizeof(float) * (size_t)n * (size_t)m);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    double *est = (double *)malloc(sizeof(double) * (size_t)(1 + n_surr));
    orc_gather_lag(series, T, target, 0, L, y);
    for (int lag = 1; lag <= n_past; ++lag) orc_gather_lag(series, T, target, lag, L, z + (int64_t)(lag - 1) * n);
    for (int i = 0; i < m; ++i)
        orc_gather_lag(series, T, parents[i] / n_lags, min_lag + parents[i] % n_lags, L,
                       x + (int64_t)i * n);
    int rc = orc_cmi_ksg(x, m, y, 1, z, n_past, n, n, k, &est[0], NULL, NULL);
    for (int s = 0; s < n_surr && rc == 0; ++s) {
        uint64_t stream = ((uint64_t)ORC_TAG_OMNIBUS << 48) | ((uint64_t)0xFFFFFFu << 24) | (uint64_t)s;
        orc_perm(seed, stream, n, pi);
        orc_permute_rows(x, m, n, n, pi, xs);
        rc = orc_cmi_ksg(xs, m, y, 1, z, n_past, n, n, k, &est[1 + s], NULL, NULL);
    }
    if (rc == 0) {
        int count = 0;
        for (int s = 0; s < n_surr; ++s)
            if (est[1 + s] >= est[0]) ++count;
        *stat = est[0];
        *pval = (double)count / (double)n_surr;
        *significant = *pval < alpha;
    }
    free(y);
    free(z);
    free(x);
    free(xs);
    free(pi);
    free(est);
    return rc;
}

/* Sequential maximum statistic: stats[i] = T_i, pvals[i], significant[i],
 * all indexed like parents. */
int orc_seqmax(const float *series, int n_proc, int64_t T, int target, int n_past, int min_lag,
               int max_lag, const int32_t *parents, int n_parents, int k, int n_surr, double alpha,
               uint64_t seed, double *stats, double *pvals, int32_t *significant)
{
    if (!orc_post_args_ok(series, n_proc, T, target, n_past, min_lag, max_lag, parents, n_parents,
                          k, n_surr) ||
        !stats || !pvals || !significant)
        return -1;
    int m = n_parents;
    double *est = (double *)malloc(sizeof(double) * (size_t)m * (size_t)(1 + n_surr));
    int *order = (int *)malloc(sizeof(int) * (size_t)m);
    int rc = orc_loo_estimates(series, n_proc, T, target, n_past, min_lag, max_lag, parents, m, k,
                               n_surr, seed, ORC_TAG_SEQMAX, est);
    if (rc == 0) {
        /* decreasing T_i, ties to the lower index: insertion sort of indices */
        for (int i = 0; i < m; ++i) {
            int j = i;
            while (j > 0 && est[(int64_t)i * (1 + n_surr)] > est[(int64_t)order[j - 1] * (1 + n_surr)]) {
                order[j] = order[j - 1];
                --j;
            }
            order[j] = i;
        }
        int still = 1;
        for (int r = 0; r < m; ++r) {
            int c = order[r];
            double t = est[(int64_t)c * (1 + n_surr)];
            int count = 0;
            for (int s = 0; s < n_surr; ++s) {
                double mx = -INFINITY;
                for (int q = r; q < m; ++q) {
                    double v = est[(int64_t)order[q] * (1 + n_surr) + 1 + s];
                    if (v > mx) mx = v;
                }
                if (mx >= t) ++count;
            }
            stats[c] = t;
            pvals[c] = (double)count / (double)n_surr;
            still = still && pvals[c] < alpha;
            significant[c] = still;
        }
    }
    free(est);
    free(order);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Bivariate transfer entropy (Summary, paragraph 5 lists bivariate TE among */
/* the network inference algorithms; the test is a reading): every source    */
/* variable c = (p, lag), p != target, lag in [min_lag, max_lag], on its own:*/
/*   T(c) = I(X_c; Y | target lags 1..n_past), surrogate s permutes X_c with */
/*   stream 0xC000<<48 | c<<24 | s; p(c) = #{s : T_s(c) >= T(c)} / S.        */
/* est [n_cand_total][1+S] and pvals [n_cand_total]; rows of the target's    */
/* own variables are left untouched.                                         */
/* Pinned by: the drivers of a driven system are significant and independent*/
/* sources are not; T(c) equals the greedy step's first estimate of c.       */
/* ------------------------------------------------------------------------ */
#define ORC_TAG_BIVAR 0xC000u

int orc_bivariate_te(const float *series, int n_proc, int64_t T, int target, int n_past,
                     int min_lag, int max_lag, int k, int n_surr, uint64_t seed, double *est,
                     double *pvals)
{
    if (!series || n_proc < 1 || target < 0 || target >= n_proc || n_past < 0 || min_lag < 1 ||
        max_lag < min_lag || k < 1 || n_surr < 1 || !est || !pvals)
        return -1;
    int n_lags = max_lag - min_lag + 1;
    int64_t L = max_lag > n_past ? max_lag : n_past;
    if (T - L < (int64_t)k + 1) return -1;
    int64_t n = T - L;
    float *y = (float *)malloc(sizeof(float) * (size_t)n);
    float *z = (float *)malloc(sizeof(float) * (size_t)n * (size_t)(n_past > 0 ? n_past : 1));
    float *xc = (float *)malloc(sizeof(float) * (size_t)n);
    float *xs = (float *)malloc(sizeof(float) * (size_t)n);
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    orc_gather_lag(series, T, target, 0, L, y);
    for (int lag = 1; lag <= n_past; ++lag) orc_gather_lag(series, T, target, lag, L, z + (int64_t)(lag - 1) * n);
    int rc = 0;
    for (int c = 0; c < n_proc * n_lags && rc == 0; ++c) {
        int p = c / n_lags, lag = min_lag + c % n_lags;
        if (p == target) continue;
        orc_gather_lag(series, T, p, lag, L, xc);
        double *row = est + (int64_t)c * (1 + n_surr);
        rc |= orc_cmi_ksg(xc, 1, y, 1, z, n_past, n, n, k, &row[0], NULL, NULL);
        int count = 0;
        for (int s = 0; s < n_surr && rc == 0; ++s) {
            uint64_t stream = ((uint64_t)ORC_TAG_BIVAR << 48) | ((uint64_t)c << 24) | (uint64_t)s;
            orc_perm(seed, stream, n, pi);
            orc_permute_rows(xc, 1, n, n, pi, xs);
            rc |= orc_cmi_ksg(xs, 1, y, 1, z, n_past, n, n, k, &row[1 + s], NULL, NULL);
            if (row[1 + s] >= row[0]) ++count;
        }
        pvals[c] = (double)count / (double)n_surr;
    }
    free(y);
    free(z);
    free(xc);
    free(xs);
    free(pi);
    return rc;
}

/* Number of threads the OpenMP runtime will use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------ */
/* Learned screen: a 3-layer perceptron F -> H -> H -> 1 with ReLU, used to   */
/* predict a candidate's largest surrogate estimate (no counterpart in the    */
/* paper; the network and its training are the build's own addition).        */
/* Parameters, flat: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.             */
/* The forward pass uses the weights rounded to bfloat16 (round to nearest,  */
/* ties to even, from the format: keep the top 16 bits of the fp32 pattern    */
/* after adding 0x7FFF plus the lowest kept bit); biases stay fp32.  This     */
/* oracle computes in double.  Inputs are normalised x' = (x - mean) * scale. */
/* Pinned by: finite differences of the loss; bfloat16 rounding against a    */
/* library conversion.                                                        */
/* ------------------------------------------------------------------------ */
float orc_bf16_round(float v)
{
    uint32_t u;
    memcpy(&u, &v, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return v; /* inf / nan unchanged */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

static int orc_mlp_nparams(int f, int h) { return h * f + h + h * h + h + h + 1; }

/* Weights as the forward pass sees them: matrices rounded to bf16 (when bf16 is
 * set), biases kept. */
static double orc_w(float v, int bf16) { return (double)(bf16 ? orc_bf16_round(v) : v); }

static void orc_mlp_effective(const float *p, int f, int h, double *q, int bf16)
{
    int o = 0;
    for (int i = 0; i < h * f; ++i, ++o) q[o] = orc_w(p[o], bf16);
    for (int i = 0; i < h; ++i, ++o) q[o] = (double)p[o];
    for (int i = 0; i < h * h; ++i, ++o) q[o] = orc_w(p[o], bf16);
    for (int i = 0; i < h; ++i, ++o) q[o] = (double)p[o];
    for (int i = 0; i < h; ++i, ++o) q[o] = orc_w(p[o], bf16);
    q[o] = (double)p[o];
}

/* y[n] = network(normalised x[n][f]); bf16 selects bf16-rounded weight matrices. */
int orc_mlp_forward(const float *p, int f, int h, const float *mean, const float *scale,
                    const float *x, int64_t n, int bf16, double *y)
{
    if (!p || !x || !y || f < 1 || h < 1 || n < 0) return -1;
    int np = orc_mlp_nparams(f, h);
    double *q = (double *)malloc(sizeof(double) * (size_t)np);
    double *a1 = (double *)malloc(sizeof(double) * (size_t)h);
    double *a2 = (double *)malloc(sizeof(double) * (size_t)h);
    double *xn = (double *)malloc(sizeof(double) * (size_t)f);
    orc_mlp_effective(p, f, h, q, bf16);
    const double *W1 = q, *b1 = q + h * f, *W2 = b1 + h, *b2 = W2 + h * h, *w3 = b2 + h,
                 *b3 = w3 + h;
    for (int64_t s = 0; s < n; ++s) {
        for (int i = 0; i < f; ++i)
            xn[i] = ((double)x[s * f + i] - (double)mean[i]) * (double)scale[i];
        for (int j = 0; j < h; ++j) {
            double acc = b1[j];
            for (int i = 0; i < f; ++i) acc += W1[j * f + i] * xn[i];
            a1[j] = acc > 0.0 ? acc : 0.0;
        }
        for (int j = 0; j < h; ++j) {
            double acc = b2[j];
            for (int i = 0; i < h; ++i) acc += W2[j * h + i] * a1[i];
            a2[j] = acc > 0.0 ? acc : 0.0;
        }
        double out = b3[0];
        for (int j = 0; j < h; ++j) out += w3[j] * a2[j];
        y[s] = out;
    }
    free(q);
    free(a1);
    free(a2);
    free(xn);
    return 0;
}

/* Loss over n rows and its gradient with respect to every parameter
 * (derivatives taken through the bf16-rounded weights, i.e. d L / d p evaluated
 * at the rounded values, the rounding treated as identity).  quantile == 0:
 * mean squared error L = (1/n) sum (y - t)^2; 0 < quantile < 1: mean pinball
 * loss L = (1/n) sum rho(t - y), rho(u) = u (quantile - [u < 0]), whose
 * minimiser is the conditional quantile of t. */
int orc_mlp_loss_grad(const float *p, int f, int h, const float *mean, const float *scale,
                      const float *x, const float *t, int64_t n, int bf16, double quantile,
                      double *loss, double *grad)
{
    if (!p || !x || !t || !loss || !grad || f < 1 || h < 1 || n < 1) return -1;
    int np = orc_mlp_nparams(f, h);
    double *q = (double *)malloc(sizeof(double) * (size_t)np);
    double *z1 = (double *)malloc(sizeof(double) * (size_t)h);
    double *a1 = (double *)malloc(sizeof(double) * (size_t)h);
    double *z2 = (double *)malloc(sizeof(double) * (size_t)h);
    double *a2 = (double *)malloc(sizeof(double) * (size_t)h);
    double *d2 = (double *)malloc(sizeof(double) * (size_t)h);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)h);
    double *xn = (double *)malloc(sizeof(double) * (size_t)f);
    orc_mlp_effective(p, f, h, q, bf16);
    const double *W1 = q, *b1 = q + h * f, *W2 = b1 + h, *b2 = W2 + h * h, *w3 = b2 + h,
                 *b3 = w3 + h;
    double *gW1 = grad, *gb1 = grad + h * f, *gW2 = gb1 + h, *gb2 = gW2 + h * h, *gw3 = gb2 + h,
           *gb3 = gw3 + h;
    for (int i = 0; i < np; ++i) grad[i] = 0.0;
    double l = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        for (int i = 0; i < f; ++i)
            xn[i] = ((double)x[s * f + i] - (double)mean[i]) * (double)scale[i];
        for (int j = 0; j < h; ++j) {
            double acc = b1[j];
            for (int i = 0; i < f; ++i) acc += W1[j * f + i] * xn[i];
            z1[j] = acc;
            a1[j] = acc > 0.0 ? acc : 0.0;
        }
        for (int j = 0; j < h; ++j) {
            double acc = b2[j];
            for (int i = 0; i < h; ++i) acc += W2[j * h + i] * a1[i];
            z2[j] = acc;
            a2[j] = acc > 0.0 ? acc : 0.0;
        }
        double y = b3[0];
        for (int j = 0; j < h; ++j) y += w3[j] * a2[j];
        double r = y - (double)t[s];
        double dy;
        if (quantile > 0.0) {
            double u = -r; /* t - y */
            l += u * (quantile - (u < 0.0 ? 1.0 : 0.0));
            dy = ((u < 0.0 ? 1.0 : 0.0) - quantile) / (double)n;
        } else {
            l += r * r;
            dy = 2.0 * r / (double)n;
        }
        gb3[0] += dy;
        for (int j = 0; j < h; ++j) {
            gw3[j] += dy * a2[j];
            d2[j] = z2[j] > 0.0 ? dy * w3[j] : 0.0;
        }
        for (int j = 0; j < h; ++j) {
            gb2[j] += d2[j];
            for (int i = 0; i < h; ++i) gW2[j * h + i] += d2[j] * a1[i];
        }
        for (int i = 0; i < h; ++i) {
            double acc = 0.0;
            for (int j = 0; j < h; ++j) acc += W2[j * h + i] * d2[j];
            d1[i] = z1[i] > 0.0 ? acc : 0.0;
        }
        for (int j = 0; j < h; ++j) {
            gb1[j] += d1[j];
            for (int i = 0; i < f; ++i) gW1[j * f + i] += d1[j] * xn[i];
        }
    }
    *loss = l / (double)n;
    free(q);
    free(z1);
    free(a1);
    free(z2);
    free(a2);
    free(d2);
    free(d1);
    free(xn);
    return 0;
}
