/*
 * idtx.h -- C ABI of the GB300 KSG conditional-mutual-information library.
 *
 * The library computes the hot path of greedy multivariate transfer-entropy
 * inference as described in the IDTxl paper (arXiv 1807.10459):
 *   - the Kraskov-Stoegbauer-Grassberger (KSG) nonlinear estimator of
 *     conditional mutual information (Summary, paragraph on estimators; the
 *     paper names the estimator and its GPU implementation but prints no
 *     formula -- the conditional form of KSG algorithm 1 is used);
 *   - surrogate null distributions that gate parent selection and stop it
 *     (Summary, paragraph on the greedy approach);
 *   - the greedy parent-set loop that maximises a CMI criterion over
 *     candidate (source, lag) variables (same paragraph).
 *
 * Estimator, for samples i = 0..N-1 of the joint variable (X, Y, Z):
 *   eps_i   = k-th smallest over j != i of max(|X_i-X_j|, |Y_i-Y_j|, |Z_i-Z_j|)
 *             (max norm over all dimensions, fp32);
 *   n_xz,i  = #{ j != i : max-norm distance in (X,Z) < eps_i }, likewise n_yz,i
 *             and n_z,i (dz == 0: the Z distance is 0);
 *   I(X;Y|Z) = psi(k) + (1/N) sum_i [psi(n_z,i+1) - psi(n_xz,i+1) - psi(n_yz,i+1)]
 *             in nats (digamma and sums in fp64).
 * Surrogate s of an estimate replaces X by its rows permuted by pi_s, the
 * Fisher-Yates shuffle of [0,N) driven by SplitMix64 started from the state
 * seed ^ mix64(stream) (mix64 = SplitMix64's output mixer): X_s[i] = X[pi_s(i)].
 *
 * Conventions for every call:
 *   - Return value: IDTX_OK or an error code; idtx_last_error() gives a
 *     message for the calling thread's last failure.
 *   - Column data: dimension d of a variable at sample t is p[d*ld + t]
 *     (fp32, ld >= N).  Input pointers may be device pointers or host
 *     pointers (pageable or pinned); host inputs are copied in by the
 *     library.  Output pointers may likewise be host or device memory.
 *     The caller owns every pointer it passes; the library never frees them.
 *   - Inputs must be finite: NaN or Inf anywhere in the used samples gives
 *     IDTX_EINVAL and no outputs.
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) on the context's device; every call synchronises that stream
 *     before it returns, so outputs are complete on return.
 *   - A context is not re-entrant: one call at a time per context.  The
 *     library allocates its own scratch (grown on demand) and frees it in
 *     idtx_ctx_destroy.
 *   - Device waits inside kernels are bounded (settings.timeout_ms); a wait
 *     that runs out returns IDTX_ETIMEOUT and leaves the context usable.
 */
#ifndef IDTX_H
#define IDTX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    IDTX_OK = 0,
    IDTX_EINVAL = 1,    /* bad argument, unsupported shape or non-finite input */
    IDTX_ENOMEM = 2,    /* device or host allocation failed */
    IDTX_ECUDA = 3,     /* a CUDA runtime call failed */
    IDTX_ETIMEOUT = 4,  /* a bounded device wait ran out */
    IDTX_EINTERNAL = 5  /* an internal consistency check failed */
};

/* Limits of the current kernels (larger shapes return IDTX_EINVAL). */
#define IDTX_MAX_DX 4
#define IDTX_MAX_DY 4
#define IDTX_MAX_DZ 16
#define IDTX_MAX_K 15
#define IDTX_MAX_N 2000000

typedef struct idtx_ctx idtx_ctx;

/* Execution modes (same results; only the schedule differs).
 * IDTX_MODE_BATCHED: all estimates of a call that share Y and Z (the original
 *   and its surrogates, or every candidate of a greedy step) run in one fused
 *   launch that computes their shared distances once.
 * IDTX_MODE_PLAIN: one launch per estimate, a warp per query scanning every
 *   sample, no sharing between estimates and no sample ordering (the
 *   reference point for batching); eps and counts outputs as in batched mode. */
#define IDTX_MODE_BATCHED 0
#define IDTX_MODE_PLAIN 1
/* IDTX_MODE_SCREENED (greedy calls only, no counterpart in the paper): every
 *   candidate first gets its estimate and the screen's s0 cheap surrogates; a
 *   small network (idtx_screen) predicts each candidate's largest surrogate
 *   estimate q, and only candidates with q + delta >= T_obs get the remaining
 *   surrogates.  Whenever the prediction bound holds for the skipped
 *   candidates the gate's count, and so the decision, equals batched mode's. */
#define IDTX_MODE_SCREENED 2

/* Estimation settings.  k: neighbours (1 <= k <= min(N-1, IDTX_MAX_K));
 * n_surr: surrogates per estimate (>= 0; the greedy calls need >= 1);
 * seed: surrogate seed; alpha: gate level of the greedy calls (0 < alpha < 1);
 * timeout_ms: bound on any device wait (<= 0 selects 2000 ms);
 * mode: IDTX_MODE_BATCHED (default, 0) or IDTX_MODE_PLAIN. */
typedef struct {
    int32_t k;
    int32_t n_surr;
    uint64_t seed;
    double alpha;
    int32_t timeout_ms;
    int32_t mode;
} idtx_settings;

/* Create a context bound to CUDA device `device`.  *ctx receives the handle. */
int idtx_ctx_create(idtx_ctx **ctx, int device);

/* Free the context and all its scratch memory.  NULL is accepted. */
int idtx_ctx_destroy(idtx_ctx *ctx);

/* Message for the calling thread's last error ("" if none).  The pointer is
 * valid until the thread's next call into the library. */
const char *idtx_last_error(void);

/* Library ABI version (major * 100 + minor). */
int idtx_version(void);

/* Counters of a context, for measurement (no counterpart in the paper: they
 * report what the library did).  kernel_launches counts every kernel the
 * library enqueued; the fused_* fields cover the fused estimator kernel
 * only: its launches, its device time (CUDA events recorded on the caller's
 * stream around each launch, only while profiling is enabled), and its
 * algorithmic lane operations: for every (query, reference sample, group of
 * jobs sharing Y and Z) that the kernel scans, 2(dy+dz')+1 operations in the
 * neighbour pass and 2dz'+1 in the count pass (one subtraction and one
 * max-abs per dimension plus the bound compare; dz' = max(dz, 1)); for
 * every scanned pair that passes the pass's shared bound, 2dx+1 per job in
 * the neighbour pass and 2dy + (2dx+7) per job in the count pass.
 * scanned_a / scanned_b count the (query, reference, group) triples scanned
 * by the neighbour / count pass, passed_a / passed_b those that passed the
 * pass's shared bound; exhaustive_pairs what scanning every reference tile in
 * both passes would have been (tiles whose bounding box is provably out of
 * reach are skipped; results are identical either way).  wait_cycles /
 * warp_cycles: SM clock cycles the kernel's warps spent waiting for staged
 * reference tiles, and in total (summed over warps). */
typedef struct {
    int64_t kernel_launches;
    int64_t fused_launches;
    double fused_ms;
    double fused_lane_ops;
    double scanned_a, passed_a, scanned_b, passed_b;
    double exhaustive_pairs;
    double wait_cycles, warp_cycles;
    int64_t graph_launches;  /* calls served by replaying a captured graph */
    /* List kernel (see idtx_ctx_set_kernel): launches, list entries walked in
     * the neighbour pass (list A) and the count pass (list B) per (query,
     * group of 32 jobs), samples scanned by full-scan fallbacks, fallbacks
     * taken (a (query, group) whose lists did not cover some job), and
     * timed trials run by the kernel choice.  fused_lane_ops of a list
     * launch counts 2dx+2 per list A entry and 2dx+4 per list B entry for
     * every job of the (query, group) whose warp walked the entry shared,
     * 2dx+4 per (job, entry) pair of the count walk's repacked phases, 2dx+2
     * per pair of a neighbour walk's lane-split tail, and 2(dx+dy+dz')+2 / +6 per
     * sample that a full-scan fallback of the two passes scans for the one
     * job it recomputes (brute_samples = fallbacks x (N-1)). */
    int64_t list_launches;
    double list_walk_a, list_walk_b, brute_samples, fallbacks;
    int64_t tune_trials;
    int32_t list_cap_a, list_cap_b;  /* list capacities of the last list launch */
    double list_tail_b;  /* (job, entry) pairs of the count walks' repacked phases (2dx+4 lane-ops each) */
    double list_tail_a;  /* (job, entry) pairs of the neighbour walks' lane-split tails (2dx+2 each) */
    /* List kernel: the sums of n_z and n_yz over every (query, job), and the
     * lane-operations a walk visiting exactly the list entries each job needs
     * would do, (2dx+4) sum n_z + (2dx+2) sum n_yz (the useful part of
     * fused_lane_ops). */
    double list_sum_nz, list_sum_nyz, useful_lane_ops;
} idtx_stats;

/* Measured instruction-issue rates of a device (no counterpart in the paper:
 * the denominator of the estimator kernels' roofline figure, which is
 * instruction issue on the CUDA cores -- the path has no contraction and its
 * DRAM traffic is a few percent of the HBM bandwidth).  Each rate comes from
 * a probe kernel that runs one instruction class in eight register chains
 * per thread at full occupancy, each step reading the next chain's value (so
 * nothing can be folded), with no memory traffic in its timed loop: FADD,
 * FMNMX, FADD with a compare and the predicated add that consumes it (3
 * lane-operations), IADD, and the count pass's step per (job, entry)
 * (subtract, absolute value, two compares, two adds: 6 lane-operations).
 * The assembler may pair independent FP32 operations into one instruction,
 * so a rate can exceed one lane-operation per lane and clock.
 * *_per_sm_clk: lane-operations per SM per SM clock;
 * *_per_s: lane-operations per second over the whole device; sm_clock_mhz:
 * the SM clock the probes ran at (cycle counts over event time).  Takes a few
 * tens of milliseconds; allocates and frees a few bytes of device memory. */
typedef struct {
    double fadd_per_sm_clk, fmnmx_per_sm_clk, fsetp_add_per_sm_clk, iadd_per_sm_clk;
    double count_mix_per_sm_clk;
    double fadd_per_s, fmnmx_per_s, fsetp_add_per_s, iadd_per_s, count_mix_per_s;
    double sm_clock_mhz;
    int n_sms;
} idtx_issue_rates;
int idtx_probe_issue_rates(int device, idtx_issue_rates *out);

/* Enable (1) or disable (0) event timing of the fused kernel. */
int idtx_ctx_set_profiling(idtx_ctx *ctx, int enable);

/* Enable (1) or disable (0) CUDA-graph replay of idtx_cmi_batch (off by
 * default; no counterpart in the paper: a launch-overhead measure for calls
 * repeated on the same device buffers).  When enabled, profiling is off and
 * every input is device memory, the call's device work (sample ordering,
 * tiles, permutations, gathers, the persistent fused launches,
 * finalisation) is captured once into a graph that owns its scratch
 * buffers, and a later call with identical arguments (input pointers,
 * sizes, surrogate counts, seeds, k, stream) replays it; the inputs may
 * hold new values, and out (host or device) may differ between calls (the
 * results are copied to it after the graph).  Calls with other arguments capture a new
 * graph (the old one is released); disabling releases it too.  Work
 * counters and fused-kernel timing are not collected for replayed calls.
 * Returns IDTX_EINVAL for a NULL ctx. */
int idtx_ctx_set_graphs(idtx_ctx *ctx, int enable);

/* Which kernel computes the estimates of a call (no counterpart in the paper,
 * whose GPU estimator is not described; both give bit-identical results):
 *   IDTX_KERNEL_TILE: the tile kernel scans reference tiles staged into
 *     shared memory, skipping tiles that are provably out of reach.
 *   IDTX_KERNEL_LIST: the list kernel first sorts, once per query and for
 *     all estimates of the call together (they share Y and Z), the samples
 *     by their (Y,Z) and their Z distance, keeping the nearest up to a
 *     capacity; each estimate then walks only the prefix it needs, with a
 *     full scan for a (query, estimate) whose neighbourhood the lists do not
 *     cover.  Needs dz >= 1 (dz = 0 calls use the tile kernel).
 *   IDTX_KERNEL_AUTO (default): on the first call of a shape (kernel
 *     variant, floor(log2 N)) both kernels run, timed, and the faster serves
 *     that shape from then on in this context.
 * Returns IDTX_EINVAL for a NULL ctx or an unknown value. */
#define IDTX_KERNEL_AUTO 0
#define IDTX_KERNEL_TILE 1
#define IDTX_KERNEL_LIST 2
int idtx_ctx_set_kernel(idtx_ctx *ctx, int kernel);

/* Capacities of the list kernel's per-query lists (entries; 0 restores the
 * defaults 2048 and 4096).  Smaller lists make full-scan fallbacks more
 * frequent; results do not change.  cap_a, cap_b: 0 or multiples of 32 in
 * [32, default].  Returns IDTX_EINVAL otherwise. */
int idtx_ctx_set_list_caps(idtx_ctx *ctx, int cap_a, int cap_b);

/* Bound every device wait of this context's calls (the tile kernel's staged-
 * tile and lock waits, the list kernel's tile-ring waits) by ns nanoseconds
 * instead of settings->timeout_ms; 0 restores the settings' bound.  No
 * counterpart in the paper: with a bound shorter than a tile copy the waits
 * run out, the call returns IDTX_ETIMEOUT, and the context stays usable, so
 * this exercises the time-out path without stalling the GPU.  A CTA that
 * gives up still waits for its own copies in flight (at least a second)
 * before it exits.  Returns IDTX_EINVAL for a NULL ctx or ns < 0. */
int idtx_ctx_set_wait_limit_ns(idtx_ctx *ctx, int64_t ns);

/* Read the counters accumulated since creation or the last reset. */
int idtx_ctx_get_stats(idtx_ctx *ctx, idtx_stats *out);

/* Zero the counters. */
int idtx_ctx_reset_stats(idtx_ctx *ctx);

/* One KSG estimate of I(X;Y|Z) plus settings->n_surr surrogates.
 * (KSG estimator: Summary, paragraph on estimators; surrogates: paragraph on
 * the greedy approach.)
 *   x [dx][ld], y [dy][ld], z [dz][ld] (z may be NULL when dz == 0), fp32.
 *   1 <= dx <= IDTX_MAX_DX, 1 <= dy <= IDTX_MAX_DY, 0 <= dz <= IDTX_MAX_DZ,
 *   k+1 <= n <= IDTX_MAX_N, ld >= n.
 *   cmi_out [1+n_surr] fp64: cmi_out[0] is the estimate, cmi_out[1+s] the
 *     estimate for surrogate s (permutation stream s, seed settings->seed).
 *   eps_out (nullable) [1+n_surr][n] fp32: eps_i of every estimate.
 *   counts_out (nullable) [1+n_surr][3][n] int32: n_xz, n_yz, n_z of every
 *     estimate. */
int idtx_cmi_ksg(idtx_ctx *ctx, const float *x, int dx, const float *y, int dy, const float *z,
                 int dz, int64_t n, int64_t ld, const idtx_settings *settings, double *cmi_out,
                 float *eps_out, int32_t *counts_out, void *stream);

/* idtx_cmi_ksg with replication-level surrogates (a reading of the paper's
 * surrogates for data made of n_reps replications, e.g. trials, of
 * len = n / n_reps consecutive samples): surrogate s moves whole
 * replications of X, X_s[r*len + t] = X[pi_s(r)*len + t], pi_s the
 * Fisher-Yates permutation of [0, n_reps) keyed (seed, stream s) as above; Y
 * and Z stay.  n_reps must divide n (n_reps = n gives idtx_cmi_ksg's
 * surrogates exactly).  Other arguments and outputs as idtx_cmi_ksg. */
int idtx_cmi_ksg_reps(idtx_ctx *ctx, const float *x, int dx, const float *y, int dy,
                      const float *z, int dz, int64_t n, int64_t ld, int64_t n_reps,
                      const idtx_settings *settings, double *cmi_out, float *eps_out,
                      int32_t *counts_out, void *stream);

/* One problem of a batch: its own columns, shape, surrogate count and seed. */
typedef struct {
    const float *x, *y, *z;
    int32_t dx, dy, dz;
    int32_t n_surr;
    int64_t n, ld;
    uint64_t seed;
} idtx_problem;

/* Many independent problems of uneven N and dimensions, each with its own
 * surrogates, in one pass over the GPU (Summary, paragraph on estimators:
 * parallel computing engines).  All problems use neighbour count k.
 *   out: concatenated [sum_p (1 + probs[p].n_surr)] fp64, problem by problem,
 *   each laid out as in idtx_cmi_ksg. */
int idtx_cmi_batch(idtx_ctx *ctx, const idtx_problem *probs, int n_probs, int k, double *out,
                   void *stream);

/* Result of one greedy step. */
typedef struct {
    int32_t cand;        /* candidate id of the maximiser (-1 if none) */
    int32_t significant; /* 1 if p < alpha */
    double stat;         /* T_obs = max over candidates of I(X_c;Y|Z) */
    double pval;         /* #{s : max_c I(X_c o pi_{c,s};Y|Z) >= T_obs} / n_surr */
    int32_t n_cand;      /* candidates evaluated */
    int32_t n_full;      /* candidates given more than the screen's s0 surrogates
                            (all candidates outside screened mode) */
    int32_t surr_done;   /* surrogate indices evaluated: n_surr, or fewer when a
                            screened step stopped early (pval is then a lower
                            bound that already decides: pval >= alpha) */
    int32_t reserved;
} idtx_step;

/* One step of the greedy parent selection for one target (Summary, paragraph
 * on the greedy approach).  series [n_proc][T] fp32.  Samples t in [L, T),
 * L = max(max_lag, n_past), N = T - L.  Y_t = series[target][t]; Z = the
 * target's own lags 1..n_past followed by the already selected candidates
 * `selected[0..n_selected)`.  Candidates are (p, lag), p in [0, n_proc),
 * lag in [min_lag, max_lag], with id c = p*(max_lag-min_lag+1) + lag-min_lag;
 * the target's lags <= n_past and the selected ids are excluded.  Every
 * candidate is estimated with settings->n_surr surrogates keyed by stream
 * (step_index << 48) | (c << 24) | s.  T_obs is the largest estimate (ties
 * to the lowest id), T_s the largest surrogate-s estimate over candidates;
 * significant iff #{s : T_s >= T_obs} / n_surr < alpha.
 *   result: the step's outcome.
 *   est_out (nullable): [n_proc*(max_lag-min_lag+1)][1+n_surr] fp64, rows of
 *   evaluated candidates only (others untouched). */
int idtx_mte_step(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                  int n_past, int min_lag, int max_lag, const int32_t *selected, int n_selected,
                  int step_index, const idtx_settings *settings, idtx_step *result,
                  double *est_out, void *stream);

/* The whole greedy loop for one target: repeats idtx_mte_step (step_index =
 * 0, 1, ...) adding the maximiser while the step is significant, until no
 * candidate is left or max_parents are selected.
 *   parents_out [max_parents] candidate ids in selection order, *n_parents;
 *   steps_out [max_parents+1] every executed step, *n_steps. */
int idtx_mte_select_target(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                           int n_past, int min_lag, int max_lag, const idtx_settings *settings,
                           int max_parents, int32_t *parents_out, int *n_parents,
                           idtx_step *steps_out, int *n_steps, void *stream);

/* Non-uniform target past (the paper's Summary says the greedy conditioning
 * builds a non-uniform embedding; how the target's own past is chosen is a
 * reading).  idtx_mte_select_past runs the greedy loop of idtx_mte_step over
 * the target's own variables (target, lag), lag in [min_lag, max_lag], only,
 * with Z = the past chosen so far (step s: step_index 0xD000 + s, n_past 0):
 *   past_out [max_past] candidate ids in selection order, *n_past;
 *   steps_out [max_past+1] every executed step, *n_steps.
 * idtx_mte_select_sources then selects sources with Z starting from that past
 * (past[0..n_past_ids), candidate ids, in order; step s: step_index s,
 * n_past 0): every candidate not in the past competes, as in
 * idtx_mte_select_target, whose result it reproduces exactly when past holds
 * the target's lags 1..n_past.  Samples t in [max_lag, T). */
int idtx_mte_select_past(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                         int min_lag, int max_lag, const idtx_settings *settings, int max_past,
                         int32_t *past_out, int *n_past, idtx_step *steps_out, int *n_steps,
                         void *stream);
int idtx_mte_select_sources(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                            const int32_t *past, int n_past_ids, int min_lag, int max_lag,
                            const idtx_settings *settings, int max_parents, int32_t *parents_out,
                            int *n_parents, idtx_step *steps_out, int *n_steps, void *stream);

/* Tests after the greedy selection (the paper's Summary asks that the errors
 * of testing many sources be controlled, and describes no test; these are
 * readings).  Common arguments as for idtx_mte_step; parents[0..n_parents)
 * are distinct candidate ids, none of them a target-past variable;
 * settings->mode must be IDTX_MODE_BATCHED.  The leave-one-out statistic of
 * parent i is T_i = I(X_{c_i}; Y | target lags 1..n_past, the other parents
 * in list order), its surrogate s permutes X_{c_i} with stream
 * tag << 48 | c_i << 24 | s.  Outputs may be host or device memory.
 *
 * Pruning by the minimum statistic.  Round r (tag 0x9000 + r): T_min =
 * min_i T_i (ties: lowest i), p = #{s : min_i T_i,s >= T_min} / n_surr; if
 * p >= alpha the parent at the minimum is removed and the next round tests
 * the rest; the loop stops at the first significant round or when no parent
 * is left.  kept_out [n_parents]: surviving parents in input order, *n_kept;
 * rounds_out (nullable) [n_parents]: per round, cand = the parent at the
 * minimum, significant, stat = T_min, pval; *n_rounds (nullable).
 * n_past + n_parents - 1 <= IDTX_MAX_DZ. */
int idtx_mte_prune(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                   int n_past, int min_lag, int max_lag, const int32_t *parents, int n_parents,
                   const idtx_settings *settings, int32_t *kept_out, int *n_kept,
                   idtx_step *rounds_out, int *n_rounds, void *stream);

/* Omnibus test of a parent set: T = I(X_P; Y | target lags 1..n_past) with
 * X_P the n_parents parents jointly (n_parents <= IDTX_MAX_DX); surrogate s
 * permutes the rows of X_P together, stream 0xA000 << 48 | 0xFFFFFF << 24 | s;
 * p = #{s : T_s >= T} / n_surr.  result: cand = -1, significant, stat, pval. */
int idtx_mte_omnibus(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                     int n_past, int min_lag, int max_lag, const int32_t *parents,
                     int n_parents, const idtx_settings *settings, idtx_step *result,
                     void *stream);

/* Sequential maximum statistic (tag 0xB000): parents in decreasing order of
 * T_i (ties: lower i first); the r-th is compared with the surrogate maxima
 * over itself and the parents after it, p_r = #{s : max_{j >= r} T_j,s >=
 * T_(r)} / n_surr; parents are significant down to the first p_r >= alpha.
 * stat_out, pval_out (fp64), significant_out (int32): [n_parents], indexed
 * like parents.  n_past + n_parents - 1 <= IDTX_MAX_DZ. */
int idtx_mte_seqmax(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                    int n_past, int min_lag, int max_lag, const int32_t *parents, int n_parents,
                    const idtx_settings *settings, double *stat_out, double *pval_out,
                    int32_t *significant_out, void *stream);

/* Bivariate transfer entropy of every source variable (the paper's Summary
 * lists bivariate TE among the network inference algorithms; the test is a
 * reading): for each candidate c = (p, lag) with p != target,
 * T(c) = I(X_c; Y | target lags 1..n_past), surrogate s permutes X_c with
 * stream 0xC000 << 48 | c << 24 | s, and p(c) = #{s : T_s(c) >= T(c)} / n_surr
 * (per source, no correction for the number of sources).  All sources'
 * estimates run as one batch.  pval_out [n_proc*(max_lag-min_lag+1)] fp64,
 * NaN at the target's own variables; est_out (nullable) [same][1+n_surr],
 * rows of the target's own variables untouched.  n_proc >= 2,
 * settings->mode IDTX_MODE_BATCHED. */
int idtx_bivariate_te(idtx_ctx *ctx, const float *series, int n_proc, int64_t T, int target,
                      int n_past, int min_lag, int max_lag, const idtx_settings *settings,
                      double *est_out, double *pval_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Learned screen (no counterpart in the paper).                            */
/* A perceptron F -> H -> H -> 1 with ReLU.  Parameters, flat fp32 master    */
/* values: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.  The forward pass     */
/* uses the weight matrices rounded to bfloat16 (round to nearest even) with */
/* fp32 arithmetic; biases stay fp32.  Features of candidate c, with I_c its */
/* estimate and I_c,0..s0-1 its first s0 surrogate estimates (streams of the */
/* step): x = (I_c, ln N, dx, dy, dz, k, mean_s I_c,s, std_s I_c,s (divisor   */
/* s0), max_s I_c,s, ln n_surr), normalised as (x - feat_mean) * feat_scale. */
/* The network predicts the excess of max over all n_surr surrogates of      */
/* I_c,s over the largest of the s0 cheap ones (never negative).             */
/* ------------------------------------------------------------------------ */
#define IDTX_SCREEN_F 10
#define IDTX_SCREEN_H 64
#define IDTX_SCREEN_NPARAMS                                                              \
    (IDTX_SCREEN_H * IDTX_SCREEN_F + IDTX_SCREEN_H + IDTX_SCREEN_H * IDTX_SCREEN_H +      \
     IDTX_SCREEN_H + IDTX_SCREEN_H + 1)

typedef struct {
    float params[IDTX_SCREEN_NPARAMS];
    float feat_mean[IDTX_SCREEN_F];
    float feat_scale[IDTX_SCREEN_F];
    float delta;   /* margin added to the prediction before the comparison with T_obs */
    int32_t s0;    /* cheap surrogates per candidate (1 <= s0 < n_surr) */
} idtx_screen;

/* Predictions (without delta) for n feature rows feats[n][IDTX_SCREEN_F]
 * (host or device memory); out[n] fp32 (host or device). */
int idtx_screen_predict(idtx_ctx *ctx, const idtx_screen *screen, const float *feats, int n,
                        float *out, void *stream);

/* Loss over n rows and its gradient grad[IDTX_SCREEN_NPARAMS] (host memory)
 * with respect to the master parameters, taken through the bf16-rounded
 * weights (rounding treated as the identity).  quantile == 0: mean squared
 * error; 0 < quantile < 1: mean pinball loss (t - y)(quantile - [t < y]),
 * whose minimiser is the conditional quantile of the targets. */
int idtx_screen_loss_grad(idtx_ctx *ctx, const idtx_screen *screen, const float *feats,
                          const float *targets, int n, float quantile, double *loss, float *grad,
                          void *stream);

/* Train screen->params in place on the GPU: `epochs` passes of Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the loss selected by
 * `quantile` (as in idtx_screen_loss_grad) over mini-batches of `batch` rows
 * in an order reshuffled every epoch (the Fisher-Yates shuffle of the
 * surrogates, seed `seed`, stream = epoch).  *final_loss (nullable) receives
 * the full-data loss after training.  feat_mean, feat_scale, delta and s0 are
 * left as given. */
int idtx_screen_train(idtx_ctx *ctx, idtx_screen *screen, const float *feats,
                      const float *targets, int n, int epochs, int batch, float lr, float quantile,
                      uint64_t seed, double *final_loss, void *stream);

/* Install the screen used by IDTX_MODE_SCREENED on this context (copied). */
int idtx_screen_set(idtx_ctx *ctx, const idtx_screen *screen);

/* Read a screen from the file at `path` and install it as idtx_screen_set
 * does.  File layout (little-endian, no padding): the 8 bytes "IDTXSCR1";
 * uint32 version (1), F (IDTX_SCREEN_F), H (IDTX_SCREEN_H), parameter count
 * (IDTX_SCREEN_NPARAMS); int32 s0; float32 delta; then float32 params
 * [IDTX_SCREEN_NPARAMS], feat_mean [F], feat_scale [F], and nothing after
 * them.  The library ships its trained screen in this form
 * (paper_1807_10459_gb300/screen_weights.bin).  Returns IDTX_EINVAL for a
 * file that cannot be read, has another layout, or holds non-finite values;
 * the context's screen is then unchanged. */
int idtx_screen_load(idtx_ctx *ctx, const char *path);

/* The screen's features (definition above) of n_cand candidates, computed
 * by the kernel the screened greedy step uses.  est: host or device
 * [n_cand][1 + s0] fp64, each row a candidate's estimate followed by its
 * first s0 surrogate estimates; n: samples of the estimates; dx, dy, dz, k,
 * n_surr as in the step.  feats_out: host or device [n_cand][IDTX_SCREEN_F]
 * fp32.  Synchronises `stream`.  Training data built with it has exactly
 * the features the screened step feeds the network. */
int idtx_screen_features(idtx_ctx *ctx, const double *est, int n_cand, int s0, int64_t n, int dx,
                         int dy, int dz, int k, int n_surr, float *feats_out, void *stream);

/* Allocation-free estimate (no counterpart in the paper; it exists for
 * callers that cannot allocate device memory -- code whose memory pool owns
 * the device, paths where a cudaMalloc would synchronise the device, or
 * services that must not grow their footprint after start-up).
 *
 * Same estimate and surrogates as idtx_cmi_ksg, computed by its preparation
 * kernels and its tile kernel, without a context: it runs on the current
 * CUDA device and takes all its scratch from one fixed array of
 * IDTX_NOALLOC_SCRATCH_BYTES bytes in device memory that the library
 * declares at file scope.  Every GPU that loads the library holds that array
 * until the process exits.  The per-sample eps and counts behind the
 * estimates are the same as idtx_cmi_ksg's; the estimates agree within
 * 1e-10 nats but not always bit for bit, because this entry point keeps the
 * samples in their given order (idtx_cmi_ksg sorts them along a Morton curve
 * for n > 256), so its fp64 partial sums are added in another order.  For
 * the same reason its tile kernel skips few reference tiles, and for large n
 * it is markedly slower than idtx_cmi_ksg.
 *   - x, y, z and cmi_out must be device memory; cmi_out [1+n_surr] fp64.
 *   - 0 <= settings->n_surr <= IDTX_NOALLOC_MAX_SURR; a problem whose scratch
 *     does not fit in the array returns IDTX_EINVAL with the bytes it needs.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress).  Every call copies its descriptors from host
 *     memory and synchronises `stream`, so it must not be called while a
 *     stream is being captured.
 *   - All calls share the one array, which keeps the previous call's
 *     contents: calls that overlap on the GPU (other threads, other streams)
 *     race with each other and must be serialised by the caller.
 *   - Synchronises `stream` before returning, on success and on every error
 *     after its first enqueue, so no kernel of the call is still using the
 *     array when it returns. */
#define IDTX_NOALLOC_SCRATCH_BYTES (16u << 20)
#define IDTX_NOALLOC_MAX_SURR 1000
int idtx_cmi_ksg_noalloc(const float *x, int dx, const float *y, int dy, const float *z, int dz,
                         int64_t n, int64_t ld, const idtx_settings *settings, double *cmi_out,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IDTX_H */
