// runtime.cu -- host runtime of the KSG library: contexts, scratch memory,
// argument checks, the small kernels around the fused estimator, and the C ABI
// declared in include/idtx.h.
//
// Per call, one "group" is a set of estimates ("jobs") that share Y and Z:
// the original estimate and its surrogates (idtx_cmi_ksg), one batch problem
// (idtx_cmi_batch), or every candidate of a greedy step with its surrogates
// (idtx_mte_step).  A group runs as
//   pack_shared  : Y/Z columns -> sh [n_pad][dsp] (row per sample, +inf pads)
//   shuffle      : surrogate permutations, one warp per permutation
//   gather_x     : X values of every job, permuted, -> xi [groups][n_pad][GB*DX]
//   ksg_fused    : kNN + counts + digamma partial sums (ksg_kernel.cuh)
//   finalize     : psi(k) + sum / N per job, fixed order
// and the greedy step adds the max-statistic gate kernel.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "idtx.h"
#include "ksg_common.cuh"
#include "shuffle.cuh"

namespace idtx {

// ------------------------------------------------------------------ errors
static thread_local std::string t_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

#define IDTX_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? IDTX_ENOMEM : IDTX_ECUDA,        \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

#define IDTX_TRY(expr)            \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != IDTX_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------------ device helpers
struct Col {  // value of a column at sample i: base[off + i]
    const float *base;
    int64_t off;
};

struct Job {  // one estimate: X source and permutation slot (-1: identity)
    int32_t src;
    int32_t slot;
};

// psi(n) for n in [0, n_max]: psi(0) is NaN; n < 16 by the finite harmonic sum
// psi(n) = -gamma + sum_{m<n} 1/m; n >= 16 by the asymptotic expansion
// ln n - 1/(2n) - sum_j B_2j / (2j n^2j) (Abramowitz & Stegun 6.3.18) through
// j = 5, whose first omitted term is below 1e-16 there.
__global__ void k_psi_table(double *psi, int64_t n_max)
{
    const double kEulerGamma = 0.57721566490153286060651209008240243;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= n_max;
         n += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (n == 0) {
            v = nan("");
        } else if (n < 16) {
            v = -kEulerGamma;
            for (int64_t m = 1; m < n; ++m) v += 1.0 / (double)m;
        } else {
            const double x = (double)n, r = 1.0 / x, r2 = r * r;
            v = log(x) - 0.5 * r -
                r2 * (1.0 / 12.0 -
                      r2 * (1.0 / 120.0 - r2 * (1.0 / 252.0 - r2 * (1.0 / 240.0 - r2 / 132.0))));
        }
        psi[n] = v;
    }
}

// Sample rows of sh (tiled layout, see ksg_common.cuh): sorted position j
// holds original sample order[j]; d < dzb -> z (0 beyond dz), then dyb y
// columns (0 beyond dy), then 0 up to dsp.  Positions j >= n are +inf in
// the dzb + dyb used columns.
__global__ void k_pack_shared(const Col *zc, int dz, int dzb, const Col *yc, int dy, int dyb,
                              int dsp, int64_t n, int64_t n_pad, const int32_t *order, float *sh,
                              int *err)
{
    const int64_t total = n_pad * dsp;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx / dsp;
        const int d = (int)(idx - j * dsp);
        float v = 0.0f;
        if (j >= n) {
            v = d < dzb + dyb ? INFINITY : 0.0f;
        } else {
            const int64_t t = order ? (int64_t)order[j] : j;
            if (d < dzb) {
                if (d < dz) v = zc[d].base[zc[d].off + t];
            } else if (d < dzb + dyb) {
                const int e = d - dzb;
                if (e < dy) v = yc[e].base[yc[e].off + t];
            }
            if (!isfinite(v)) atomicOr(err, kErrNonFinite);
        }
        const int64_t tile = j / kTJ, row = j - tile * kTJ;
        sh[(tile * kTileRows + row) * dsp + d] = v;
    }
}

// Rows kTJ and kTJ+1 of every sh tile: per-dimension minimum and maximum over
// the tile's real samples (one block of kTJ threads per tile).
__global__ void __launch_bounds__(kTJ) k_tile_boxes(float *sh, int dsp, int64_t n)
{
    __shared__ float s_mn[kTJ / 32], s_mx[kTJ / 32];
    const int64_t tile = blockIdx.x;
    const int r = threadIdx.x;
    const bool real = tile * kTJ + r < n;
    float *base = sh + tile * kTileRows * dsp;
    for (int d = 0; d < dsp; ++d) {
        const float v = base[r * dsp + d];
        float mn = real ? v : INFINITY, mx = real ? v : -INFINITY;
        for (int off = 16; off >= 1; off >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        }
        if ((r & 31) == 0) {
            s_mn[r >> 5] = mn;
            s_mx[r >> 5] = mx;
        }
        __syncthreads();
        if (r == 0) {
            for (int w = 1; w < kTJ / 32; ++w) {
                mn = fminf(mn, s_mn[w]);
                mx = fmaxf(mx, s_mx[w]);
            }
            base[kTJ * dsp + d] = mn;
            base[(kTJ + 1) * dsp + d] = mx;
        }
        __syncthreads();
    }
}

// Per shared column (z columns, then y columns): minimum and maximum over n
// samples; one block per column.
__global__ void k_minmax_cols(const Col *zc, int dz, const Col *yc, int dy, int64_t n, float *mm)
{
    __shared__ float s_mn[32], s_mx[32];
    const int c = blockIdx.x;
    const Col col = c < dz ? zc[c] : yc[c - dz];
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const float v = col.base[col.off + j];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    for (int off = 16; off >= 1; off >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if ((threadIdx.x & 31) == 0) {
        s_mn[threadIdx.x >> 5] = mn;
        s_mx[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mn = fminf(mn, s_mn[w]);
            mx = fmaxf(mx, s_mx[w]);
        }
        mm[2 * c] = mn;
        mm[2 * c + 1] = mx;
    }
}

// Morton (Z-order) key of every sample over its first nk shared coordinates,
// each quantised to `bits` bits between the column's minimum and maximum;
// idx[j] = j.  Only the order of the samples depends on it, never a result.
__global__ void k_morton_keys(const Col *zc, int dz, const Col *yc, int nk, int bits, int64_t n,
                              const float *mm, uint32_t *keys, int32_t *idx)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t qv[32];
        const float scale = (float)(1u << bits);
        for (int c = 0; c < nk; ++c) {
            const Col col = c < dz ? zc[c] : yc[c - dz];
            const float lo = mm[2 * c], hi = mm[2 * c + 1];
            const float t = hi > lo ? (col.base[col.off + j] - lo) / (hi - lo) : 0.0f;
            const float f = fminf(fmaxf(t * scale, 0.0f), scale - 1.0f);
            qv[c] = (uint32_t)f;
        }
        uint32_t key = 0;
        for (int b = bits - 1; b >= 0; --b)
            for (int c = 0; c < nk; ++c) key = (key << 1) | ((qv[c] >> b) & 1u);
        keys[j] = key;
        idx[j] = (int32_t)j;
    }
}

// Replication-level surrogates: slot s's permutation of the samples moves
// whole replications of len samples, pi_s(r*len + t) = blk[s][r]*len + t,
// blk[s] the permutation of the n_reps replications.  With `order`, the row
// is written composed with it: perm[s][j] = pi_s(order[j]).
__global__ void k_expand_reps(const int32_t *blk, int n_slots, int64_t n_reps, int64_t len,
                              const int32_t *order, int32_t *perm)
{
    const int64_t n = n_reps * len, total = (int64_t)n_slots * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = idx / n, j = idx - slot * n;
        const int64_t i = order ? (int64_t)order[j] : j;
        perm[idx] = (int32_t)((int64_t)blk[slot * n_reps + i / len] * len + i % len);
    }
}

constexpr int kGatherRows = kTJ % 64 == 0 ? 64 : 32;  // sample rows per CTA of k_gather_x
constexpr int kGatherThreads = 256;
constexpr int kGatherMaxWidth = 32 * 4;  // jobs per group x padded X width
constexpr int kGatherJobsPerWarp = 4;    // 32 jobs per group over 8 warps

// xi[grp][j][g*dxb + d] = X_job[d][pi_job(order[j])] (job = grp*gb + g; jobs
// past the end repeat job 0; pi the identity for slot -1), 0 for d >= dx,
// +inf for j >= n.  With `composed`, the permutation rows already hold
// pi(order[j]) at j (k_shuffle_smem, k_expand_reps), so a warp reads 32
// consecutive entries of a row.  A CTA fills kGatherRows consecutive rows of
// one group: warp w takes the jobs g = w, w + 8, ..., lane l the rows
// j0 + l + 32 h; all of a warp's permutation loads are issued before the
// first is used; the values are staged in shared memory (gather_smem bytes)
// and the rows, contiguous in xi, are written out in sequence.  Permutation
// entries and xi are touched once: loaded and stored as streaming, so that L1
// keeps the X columns the random reads hit.  Grid: n_groups * (n_pad /
// kGatherRows) CTAs.
__global__ void __launch_bounds__(kGatherThreads)
    k_gather_x(const Col *xc, int dx, int dxb, const Job *jobs, int n_jobs,
               const int32_t *perm, int64_t n, int64_t n_pad, int gb, const int32_t *order,
               bool composed, float *xi, int *err)
{
    constexpr int kWarps = kGatherThreads / 32, kHalves = kGatherRows / 32;
    extern __shared__ float s_x[];  // [kGatherRows][xw + 1]
    const int xw = gb * dxb, ld = xw + 1;
    const int64_t tiles = n_pad / kGatherRows;
    const int64_t grp = blockIdx.x / tiles;
    const int64_t j0 = (blockIdx.x - grp * tiles) * kGatherRows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool in[kHalves];
    int64_t t0[kHalves], at[kHalves];
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
        const int64_t j = j0 + h * 32 + lane;
        in[h] = j < n;
        t0[h] = in[h] ? (order ? (int64_t)order[j] : j) : 0;
        at[h] = composed ? j : t0[h];  // the row's position in a permutation row
    }
    Job jb[kGatherJobsPerWarp];
#pragma unroll
    for (int u = 0; u < kGatherJobsPerWarp; ++u) {
        int64_t job = grp * gb + warp + u * kWarps;
        if (job >= n_jobs) job = 0;
        jb[u] = jobs[job];
    }
    int64_t t[kGatherJobsPerWarp][kHalves];
#pragma unroll
    for (int u = 0; u < kGatherJobsPerWarp; ++u)
#pragma unroll
        for (int h = 0; h < kHalves; ++h) {
            const bool use = warp + u * kWarps < gb && in[h] && jb[u].slot >= 0;
            t[u][h] = use ? (int64_t)__ldcs(perm + (int64_t)jb[u].slot * n + at[h]) : t0[h];
        }
#pragma unroll
    for (int u = 0; u < kGatherJobsPerWarp; ++u) {
        const int g = warp + u * kWarps;
        if (g >= gb) break;
        for (int d = 0; d < dxb; ++d) {
            const bool real = d < dx;
            const Col c = real ? xc[(int64_t)jb[u].src * dx + d] : Col{nullptr, 0};
#pragma unroll
            for (int h = 0; h < kHalves; ++h) {
                float v = in[h] ? 0.0f : INFINITY;
                if (in[h] && real) {
                    v = c.base[c.off + t[u][h]];
                    if (!isfinite(v)) atomicOr(err, kErrNonFinite);
                }
                s_x[(h * 32 + lane) * ld + g * dxb + d] = v;
            }
        }
    }
    __syncthreads();
    float *out = xi + (grp * n_pad + j0) * xw;
    for (int e = threadIdx.x; e < kGatherRows * xw; e += kGatherThreads) {
        const int r = e / xw;
        __stcs(out + e, s_x[r * ld + (e - r * xw)]);
    }
}

// Dynamic shared memory of k_gather_x: the staged rows.
static size_t gather_smem(int gb, int dxb)
{
    return (size_t)kGatherRows * (gb * dxb + 1) * sizeof(float);
}

// The gather's grid; 0 when the shape is outside its limits.
static int64_t gather_blocks(int64_t n_groups, int64_t n_pad, int gb, int dxb)
{
    if (gb > kGatherJobsPerWarp * (kGatherThreads / 32) || gb * dxb > kGatherMaxWidth ||
        n_pad % kGatherRows)
        return 0;
    const int64_t b = n_groups * (n_pad / kGatherRows);
    return b > 0x7fffffff ? 0 : b;
}

// cmi[job] = psi(k) + (sum over query tiles, in order) / n.
__global__ void k_finalize(const double *partial, int n_jobs, int n_qt, const double *psi, int k,
                           int64_t n, double *cmi)
{
    const int job = blockIdx.x * blockDim.x + threadIdx.x;
    if (job >= n_jobs) return;
    double s = 0.0;
    for (int t = 0; t < n_qt; ++t) s += partial[(int64_t)job * n_qt + t];
    cmi[job] = psi[k] + s / (double)n;
}

// Max-statistic gate.  est_a [n_cand][1 + sa]: every candidate's estimate and
// its first sa surrogates; est_b [n_keep][n_surr - sa]: the remaining
// surrogates of the candidates listed in keep (screened mode; n_keep = 0 and
// sa = n_surr otherwise).  T_obs = largest estimate (ties to the lowest
// candidate, which comes first); surrogate s's maximum runs over all
// candidates for s < sa and over the kept ones for s >= sa.
__global__ void k_gate(const double *est_a, int n_cand, int sa, const double *est_b, int n_keep,
                       int n_surr, const int32_t *ids, double alpha, idtx_step *out)
{
    __shared__ double s_tobs;
    __shared__ int s_best;
    __shared__ int s_cnt[32];
    const int tid = threadIdx.x;
    const int row_a = 1 + sa, row_b = n_surr - sa;
    if (tid == 0) {
        double t = -INFINITY;
        int b = -1;
        for (int c = 0; c < n_cand; ++c) {
            const double v = est_a[(int64_t)c * row_a];
            if (v > t) {
                t = v;
                b = c;
            }
        }
        s_tobs = t;
        s_best = b;
    }
    __syncthreads();
    int cnt = 0;
    for (int s = tid; s < n_surr; s += blockDim.x) {
        double ts = -INFINITY;
        if (s < sa) {
            for (int c = 0; c < n_cand; ++c) ts = fmax(ts, est_a[(int64_t)c * row_a + 1 + s]);
        } else {
            for (int c = 0; c < n_keep; ++c) ts = fmax(ts, est_b[(int64_t)c * row_b + s - sa]);
        }
        cnt += ts >= s_tobs ? 1 : 0;
    }
    for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        int total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += s_cnt[w];
        const double p = (double)total / (double)n_surr;
        out->cand = s_best >= 0 ? ids[s_best] : -1;
        out->significant = (s_best >= 0 && p < alpha) ? 1 : 0;
        out->stat = s_tobs;
        out->pval = p;
        out->n_cand = n_cand;
        out->n_full = sa == n_surr ? n_cand : n_keep;
        out->surr_done = n_surr;
        out->reserved = 0;
    }
}

// Screened steps: T_obs, its candidate, and the count over the first sa
// surrogate indices (every candidate has them) into out / *count.
// Tests after the greedy selection.  est: [m][1+S], row i = parent ids[i]'s
// leave-one-out estimate and its surrogates.
//
// Minimum statistic (pruning round): T_min = min_i T_i (ties: lowest i),
// p = #{s : min_i T_i,s >= T_min} / S.  One block.
__global__ void k_min_stat(const double *est, int m, int n_surr, const int32_t *ids, double alpha,
                           idtx_step *out)
{
    __shared__ double s_tmin;
    __shared__ int s_at;
    __shared__ int s_cnt[32];
    const int tid = threadIdx.x, row = 1 + n_surr;
    if (tid == 0) {
        int at = 0;
        for (int i = 1; i < m; ++i)
            if (est[(int64_t)i * row] < est[(int64_t)at * row]) at = i;
        s_at = at;
        s_tmin = est[(int64_t)at * row];
    }
    __syncthreads();
    int cnt = 0;
    for (int sidx = tid; sidx < n_surr; sidx += blockDim.x) {
        double mn = INFINITY;
        for (int i = 0; i < m; ++i) mn = fmin(mn, est[(int64_t)i * row + 1 + sidx]);
        cnt += mn >= s_tmin ? 1 : 0;
    }
    for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        int total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += s_cnt[w];
        const double p = (double)total / (double)n_surr;
        out->cand = ids[s_at];
        out->significant = p < alpha ? 1 : 0;
        out->stat = s_tmin;
        out->pval = p;
        out->n_cand = m;
        out->n_full = m;
        out->surr_done = n_surr;
        out->reserved = 0;
    }
}

// Per-candidate p-values against each candidate's own surrogates (bivariate
// TE): out[c] = #{s : T_s(c) >= T(c)} / S for candidate ids with a row
// (row_of[c] >= 0), NaN otherwise.  One thread per candidate id.
__global__ void k_cand_pvals(const double *est, const int32_t *row_of, int n_cand_total,
                             int n_surr, double *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cand_total) return;
    const int r = row_of[c];
    if (r < 0) {
        out[c] = NAN;
        return;
    }
    const double *row = est + (int64_t)r * (1 + n_surr);
    int cnt = 0;
    for (int sidx = 0; sidx < n_surr; ++sidx) cnt += row[1 + sidx] >= row[0] ? 1 : 0;
    out[c] = (double)cnt / (double)n_surr;
}

// Single statistic against its own surrogates (omnibus test): p = #{s : T_s >= T} / S.
__global__ void k_single_stat(const double *est, int n_surr, double alpha, idtx_step *out)
{
    __shared__ int s_cnt[32];
    const int tid = threadIdx.x;
    int cnt = 0;
    for (int sidx = tid; sidx < n_surr; sidx += blockDim.x) cnt += est[1 + sidx] >= est[0] ? 1 : 0;
    for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        int total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += s_cnt[w];
        const double p = (double)total / (double)n_surr;
        out->cand = -1;
        out->significant = p < alpha ? 1 : 0;
        out->stat = est[0];
        out->pval = p;
        out->n_cand = 1;
        out->n_full = 1;
        out->surr_done = n_surr;
        out->reserved = 0;
    }
}

// Sequential maximum statistic: parents in decreasing T_i (ties: lower i
// first); the r-th is compared with the surrogate maxima over itself and the
// parents after it; significant down to the first p >= alpha.  One block;
// rank[] (m ints) is scratch.  stats, pvals, sig indexed like the parents.
__global__ void k_seqmax_stat(const double *est, int m, int n_surr, double alpha, int32_t *rank,
                              double *stats, double *pvals, int32_t *sig)
{
    __shared__ int s_cnt[32];
    const int tid = threadIdx.x, row = 1 + n_surr;
    if (tid == 0) {
        for (int i = 0; i < m; ++i) {
            int j = i;
            while (j > 0 && est[(int64_t)i * row] > est[(int64_t)rank[j - 1] * row]) {
                rank[j] = rank[j - 1];
                --j;
            }
            rank[j] = i;
        }
    }
    __syncthreads();
    int still = 1;
    for (int r = 0; r < m; ++r) {
        const int c = rank[r];
        const double t = est[(int64_t)c * row];
        int cnt = 0;
        for (int sidx = tid; sidx < n_surr; sidx += blockDim.x) {
            double mx = -INFINITY;
            for (int q = r; q < m; ++q) mx = fmax(mx, est[(int64_t)rank[q] * row + 1 + sidx]);
            cnt += mx >= t ? 1 : 0;
        }
        for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
        __syncthreads();
        if (tid == 0) {
            int total = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += s_cnt[w];
            const double p = (double)total / (double)n_surr;
            still = still && p < alpha;
            stats[c] = t;
            pvals[c] = p;
            sig[c] = still;
        }
        __syncthreads();
    }
}

__global__ void k_gate_begin(const double *est_a, int n_cand, int sa, const int32_t *ids,
                             idtx_step *out, int *count)
{
    __shared__ double s_tobs;
    __shared__ int s_cnt;
    if (threadIdx.x == 0) {
        double t = -INFINITY;
        int b = -1;
        for (int c = 0; c < n_cand; ++c) {
            const double v = est_a[(int64_t)c * (1 + sa)];
            if (v > t) {
                t = v;
                b = c;
            }
        }
        s_tobs = t;
        s_cnt = 0;
        out->cand = b >= 0 ? ids[b] : -1;
        out->stat = t;
        out->n_cand = n_cand;
        out->reserved = 0;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < sa; s += blockDim.x) {
        double ts = -INFINITY;
        for (int c = 0; c < n_cand; ++c) ts = fmax(ts, est_a[(int64_t)c * (1 + sa) + 1 + s]);
        if (ts >= s_tobs) atomicAdd(&s_cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *count = s_cnt;
}

// Adds to *count the surrogate indices of a block est [n_rows][ncol] (one
// chunk of indices for the kept candidates) whose maximum reaches T_obs.
__global__ void k_gate_chunk(const double *est, int n_rows, int ncol, const idtx_step *step,
                             int *count)
{
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
        double ts = -INFINITY;
        for (int r = 0; r < n_rows; ++r) ts = fmax(ts, est[(int64_t)r * ncol + j]);
        if (ts >= step->stat) atomicAdd(count, 1);
    }
}

__global__ void k_gate_end(idtx_step *out, const int *count, int n_surr, int surr_done,
                           int n_full, double alpha)
{
    const double p = (double)*count / (double)n_surr;
    out->pval = p;
    out->significant = (out->cand >= 0 && p < alpha) ? 1 : 0;
    out->n_full = n_full;
    out->surr_done = surr_done;
}

// Screen features of every candidate from its estimate and first s0 surrogate
// estimates (est [n_cand][1+s0]); the definition is the one in idtx.h.
__global__ void k_screen_features(const double *est, int n_cand, int s0, float ln_n, int dx,
                                  int dy, int dz, int k, float ln_s, float *feats)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cand) return;
    const double *r = est + (int64_t)c * (1 + s0);
    double mean = 0.0, mx = -INFINITY;
    for (int s = 0; s < s0; ++s) {
        mean += r[1 + s];
        mx = fmax(mx, r[1 + s]);
    }
    mean /= s0;
    double var = 0.0;
    for (int s = 0; s < s0; ++s) var += (r[1 + s] - mean) * (r[1 + s] - mean);
    var /= s0;
    float *f = feats + (int64_t)c * IDTX_SCREEN_F;
    f[0] = (float)r[0];
    f[1] = ln_n;
    f[2] = (float)dx;
    f[3] = (float)dy;
    f[4] = (float)dz;
    f[5] = (float)k;
    f[6] = (float)mean;
    f[7] = (float)sqrt(var);
    f[8] = (float)mx;
    f[9] = ln_s;
}

// Keep candidate c iff m_c + max(pred[c], 0) + delta >= T_obs, m_c the largest of
// its s0 cheap surrogate estimates (a lower bound of its largest surrogate
// estimate) and pred[c] the network's prediction of the excess over m_c; kept
// candidates listed in ascending order in keep[], their count in *n_keep.
__global__ void k_screen_keep(const double *est, int n_cand, int s0, const float *pred,
                              float delta, int32_t *keep, int32_t *n_keep)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = -INFINITY;
    for (int c = 0; c < n_cand; ++c) t = fmax(t, est[(int64_t)c * (1 + s0)]);
    int n = 0;
    for (int c = 0; c < n_cand; ++c) {
        double m = -INFINITY;
        for (int s = 0; s < s0; ++s) m = fmax(m, est[(int64_t)c * (1 + s0) + 1 + s]);
        if (m + fmax((double)pred[c], 0.0) + (double)delta >= t) keep[n++] = c;
    }
    *n_keep = n;
}

static int grid_for(int64_t total, int block)
{
    int64_t g = (total + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

}  // namespace idtx

using namespace idtx;

// ------------------------------------------------------------------ context
enum {
    B_IN = 0,   // copied host inputs
    B_DESC,     // per-call descriptor arena (columns, jobs, streams, seeds)
    B_SH,
    B_XI,
    B_PERM,
    B_PARTIAL,
    B_CMI,
    B_EPS,
    B_CNT,
    B_STEP,
    B_ORDER,    // sample order along the Morton curve, sort keys, column ranges
    B_SORT,     // radix-sort temporary storage
    B_WORK,     // fused-kernel work counters, kNumWork per group
    B_SCREEN,   // screen parameters, normalisation, features, predictions, keep list
    B_MLP,      // screen network work area
    B_TRAIN,    // screen training data, order, Adam moments
    B_TABLE,    // persistent multi-problem launches: problem table, task offsets, counters
    B_LIST,     // per-query sorted neighbour lists of the list kernel
    kNumBufs
};

// Shape of one fused launch, to turn its work counters into operations.
struct WorkShape {
    bool list;  // the list kernel ran (else the tile kernel)
    int dx, dy, dz_eff, gb;
    double job_frac;  // real jobs / (groups * gb)
    double exhaustive_pairs;
};

struct idtx_ctx {
    int device = 0;
    void *buf[kNumBufs] = {};
    size_t cap[kNumBufs] = {};
    double *psi = nullptr;
    int64_t psi_n = 0;
    int *d_err = nullptr;
    int *h_err = nullptr;  // pinned
    std::vector<KsgVariant> variants;
    // measurement counters
    bool profiling = false;
    idtx_stats stats = {};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // fused launches of this call
    std::vector<cudaEvent_t> event_pool;
    std::vector<WorkShape> call_shapes;  // launches of the current call, by work slot
    unsigned long long *h_work = nullptr;  // pinned copy of the counters
    size_t h_work_cap = 0;
    bool has_screen = false;
    idtx_screen screen;  // installed by idtx_screen_set
    // CUDA-graph replay of idtx_cmi_batch: the graph's own scratch buffers,
    // the arguments it was captured for, the capture stream
    bool graphs = false;
    void *gbuf[kNumBufs] = {};
    size_t gcap[kNumBufs] = {};
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_key;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side_stream = nullptr;  // second stream of a call (prep_group)
    // kernel choice: IDTX_KERNEL_AUTO picks per (variant, log2 N) by timing
    // both kernels on the first call of that shape; list capacities (0: default)
    int kernel_pref = IDTX_KERNEL_AUTO;
    struct Choice {
        bool list;         // list kernel (else tile kernel)
        int cap_a, cap_b;  // its list capacities
    };
    std::map<std::pair<const KsgVariant *, int>, Choice> tuned;
    int cap_a = 0, cap_b = 0;
    long long wait_ns = 0;  // bound of device waits (0: settings->timeout_ms)
};

void drop_graph(idtx_ctx *c)
{
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    c->graph_key.clear();
}

// Exchange the context's scratch buffers with the graph's.
void swap_buffer_sets(idtx_ctx *c)
{
    for (int i = 0; i < kNumBufs; ++i) {
        std::swap(c->buf[i], c->gbuf[i]);
        std::swap(c->cap[i], c->gcap[i]);
    }
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int ensure(idtx_ctx *c, int slot, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (c->cap[slot] >= bytes) return IDTX_OK;
    if (c->buf[slot]) {
        cudaFree(c->buf[slot]);
        c->buf[slot] = nullptr;
        c->cap[slot] = 0;
    }
    size_t want = std::max(bytes, c->cap[slot] + c->cap[slot] / 2);
    want = (want + (1u << 21) - 1) & ~((size_t)(1u << 21) - 1);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(IDTX_ENOMEM, "cudaMalloc of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    c->buf[slot] = p;
    c->cap[slot] = want;
    return IDTX_OK;
}

int ensure_psi(idtx_ctx *c, int64_t n_max, cudaStream_t st)
{
    if (c->psi_n >= n_max) return IDTX_OK;
    int64_t want = std::max<int64_t>(n_max, 1 << 16);
    if (c->psi) cudaFree(c->psi);
    c->psi = nullptr;
    c->psi_n = 0;
    IDTX_CUDA(cudaMalloc(&c->psi, sizeof(double) * (size_t)(want + 1)));
    k_psi_table<<<grid_for(want + 1, 256), 256, 0, st>>>(c->psi, want);
    IDTX_CUDA(cudaGetLastError());
    c->stats.kernel_launches += 1;
    c->psi_n = want;
    return IDTX_OK;
}

bool device_accessible(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

const int kZBuckets[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16};

const KsgVariant *pick_variant(const idtx_ctx *c, int dx, int dy, int dz, int k)
{
    const int dze = std::max(dz, 1);
    if (k == 4 && dx <= 2 && dy <= 2) {
        int zb = 0;
        for (int b : kZBuckets)
            if (b >= dze) {
                zb = b;
                break;
            }
        for (const KsgVariant &v : c->variants)
            if (v.exact && v.k1 == 5 && v.dx == dx && v.dy == dy && v.dz == zb) return &v;
    }
    for (const KsgVariant &v : c->variants)
        if (!v.exact && v.dx >= dx && v.dy >= dy && v.dz >= dze && v.k1 > k) return &v;
    return nullptr;
}

// Host-side description of one group of jobs sharing Y and Z.
struct Group {
    int64_t n = 0;
    int dx = 0, dy = 0, dz = 0, k = 0;
    std::vector<Col> xcols;  // [n_src][dx]
    std::vector<Col> ycols, zcols;
    std::vector<Job> jobs;
    std::vector<uint64_t> slot_stream, slot_seed;
    // filled by plan()
    const KsgVariant *v = nullptr;
    int64_t n_pad = 0;
    int n_qt = 0, n_groups = 0;
    size_t off_x = 0, off_y = 0, off_z = 0, off_jobs = 0, off_streams = 0, off_seeds = 0;
    size_t off_cmi = 0;  // index of the group's first job in the call's cmi buffer
    bool sort = false;   // order the samples along a Morton curve first
    bool plain = false;  // one launch per estimate (IDTX_MODE_PLAIN)
    int work_slot = 0;   // index of the group's work counters in the call
    int64_t n_reps = 0;     // > 0: surrogates permute n_reps whole replications
    bool use_list = false;  // run the list kernel (ksg_list.cuh)
    bool tune = false;      // time both kernels first (shape not tuned yet)
    int cap_a = 0, cap_b = 0;  // list capacities
};

// Memory the lists of one group may take; larger N gets shorter lists.
constexpr size_t kListBudget = size_t(8) << 30;

size_t list_bytes(int64_t n, int cap_a, int cap_b);

// List capacities for n samples (0, 0: no lists).
void list_caps(const idtx_ctx *c, int64_t n, int &cap_a, int &cap_b)
{
    const int all = (int)std::min<int64_t>((n - 1 + 31) / 32 * 32, 1 << 30);
    cap_a = std::min(c->cap_a > 0 ? c->cap_a : kMaxListA, all);
    cap_b = std::min(c->cap_b > 0 ? c->cap_b : kMaxListB, all);
    while (cap_a >= 64 && list_bytes(n, cap_a, cap_b) > kListBudget) {
        cap_a = cap_a / 64 * 32;
        cap_b = std::max(32, cap_b / 64 * 32);
    }
    if (list_bytes(n, cap_a, cap_b) > kListBudget) cap_a = cap_b = 0;
}

std::pair<const KsgVariant *, int> tune_key(const Group &g)
{
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= g.n) ++lg;
    return {g.v, lg};
}

int plan(idtx_ctx *c, Group &g)
{
    g.v = pick_variant(c, g.dx, g.dy, g.dz, g.k);
    if (!g.v)
        return fail(IDTX_EINVAL, "no kernel for dx=%d dy=%d dz=%d k=%d", g.dx, g.dy, g.dz, g.k);
    g.n_pad = (g.n + kTJ - 1) / kTJ * kTJ;
    g.n_qt = (int)(g.n_pad / g.v->qc);
    g.n_groups = (int)((g.jobs.size() + g.v->gb - 1) / g.v->gb);
    if (g.n_groups > 65535) return fail(IDTX_EINVAL, "too many estimates in one group");
    g.sort = !g.plain && g.n > 2 * kTJ;
    if (g.plain) g.n_qt = (int)(g.n_pad / kPlainQueriesPerPartial);
    // The list kernel needs a Z subspace (with dz = 0 list B would hold every
    // sample) and lists that fit the memory budget.
    g.use_list = g.tune = false;
    g.cap_a = g.cap_b = 0;
    if (!g.plain && g.dz >= 1 && c->kernel_pref != IDTX_KERNEL_TILE) {
        list_caps(c, g.n, g.cap_a, g.cap_b);
        if (g.cap_a > 0) {
            if (c->kernel_pref == IDTX_KERNEL_LIST) {
                g.use_list = true;
            } else {
                auto it = c->tuned.find(tune_key(g));
                if (it == c->tuned.end()) {
                    g.tune = true;
                } else {
                    g.use_list = it->second.list;
                    if (g.use_list) {
                        g.cap_a = it->second.cap_a;
                        g.cap_b = it->second.cap_b;
                    }
                }
            }
        }
    }
    return IDTX_OK;
}

// Bits per coordinate and number of coordinates of the Morton key.
void morton_shape(int n_shared, int &nk, int &bits)
{
    nk = std::min(n_shared, 32);
    bits = std::max(1, std::min(10, 32 / std::max(nk, 1)));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Lay out the descriptor arrays of all groups in one host arena.
void pack_desc(std::vector<Group> &gs, std::vector<unsigned char> &arena)
{
    size_t off = 0;
    auto put = [&](const void *src, size_t bytes) {
        off = align_up(off, 16);
        size_t at = off;
        arena.resize(off + bytes);
        if (bytes) memcpy(arena.data() + at, src, bytes);
        off += bytes;
        return at;
    };
    for (Group &g : gs) {
        g.off_x = put(g.xcols.data(), g.xcols.size() * sizeof(Col));
        g.off_y = put(g.ycols.data(), g.ycols.size() * sizeof(Col));
        g.off_z = put(g.zcols.data(), g.zcols.size() * sizeof(Col));
        g.off_jobs = put(g.jobs.data(), g.jobs.size() * sizeof(Job));
        g.off_streams = put(g.slot_stream.data(), g.slot_stream.size() * sizeof(uint64_t));
        g.off_seeds = put(g.slot_seed.data(), g.slot_seed.size() * sizeof(uint64_t));
    }
    if (arena.empty()) arena.resize(16);
}

struct CallBuffers {
    size_t sh = 0, xi = 0, perm = 0, partial = 0, order = 0, sort_tmp = 0, lists = 0;
};

// B_LIST layout for n queries: list_a [n][cap_a] | list_b [n][cap_b] | meta [n]
// | the list kernel's term ring.
size_t list_bytes(int64_t n, int cap_a, int cap_b)
{
    return align_up((size_t)n * cap_a * sizeof(int2), 256) +
           align_up((size_t)n * cap_b * sizeof(int2), 256) +
           align_up((size_t)n * sizeof(int4), 256) + kListRingBytes;
}

// B_ORDER layout for n samples: order | idx | keys_in | keys_out | column ranges.
size_t order_bytes(int64_t n) { return 4 * align_up((size_t)n * 4, 256) + 256; }

// Scratch bytes one group needs (each rounded up to 256 bytes).
CallBuffers bytes_of(const Group &g)
{
    CallBuffers b;
    b.sh = align_up((size_t)(g.n_pad / kTJ) * kTileRows * g.v->dsp * sizeof(float), 256);
    if (g.sort) {
        b.order = align_up(order_bytes(g.n), 256);
        size_t tmp = 0;
        sort_pairs_u32(nullptr, tmp, nullptr, nullptr, nullptr, nullptr, (int)g.n, 32, nullptr);
        b.sort_tmp = align_up(tmp, 256);
    }
    b.xi = align_up((size_t)g.n_groups * g.n_pad * g.v->gb * g.v->dx * sizeof(float), 256);
    b.perm = align_up(g.slot_stream.size() * (size_t)(g.n + g.n_reps) * sizeof(int32_t), 256);
    b.partial = align_up(g.jobs.size() * (size_t)g.n_qt * sizeof(double), 256);
    if (g.use_list || g.tune) b.lists = list_bytes(g.n, g.cap_a, g.cap_b);
    return b;
}

// Buffers for groups enqueued one after another (each reuses the same scratch).
void sizes_of(const Group &g, CallBuffers &b)
{
    const CallBuffers o = bytes_of(g);
    b.sh = std::max(b.sh, o.sh);
    b.order = std::max(b.order, o.order);
    b.sort_tmp = std::max(b.sort_tmp, o.sort_tmp);
    b.xi = std::max(b.xi, o.xi);
    b.perm = std::max(b.perm, o.perm);
    b.partial = std::max(b.partial, o.partial);
    b.lists = std::max(b.lists, o.lists);
}

// Where one group's scratch lives.
struct Slices {
    float *sh;
    float *xi;
    int32_t *perm;
    double *partial;
    unsigned char *order;
    void *sort_tmp;
    size_t sort_cap;
    unsigned char *lists;  // B_LIST region (list groups only)
};

int take_event(idtx_ctx *c, cudaEvent_t *ev)
{
    if (!c->event_pool.empty()) {
        *ev = c->event_pool.back();
        c->event_pool.pop_back();
        return IDTX_OK;
    }
    IDTX_CUDA(cudaEventCreate(ev));
    return IDTX_OK;
}

// Whether this device's blocks may hold the kShufWide row (per device).
static bool g_shuffle_wide[kMaxDevices];

// One-time attributes of the shared-memory shuffles (per device; the
// attribute is per function and device).  Also called before a graph capture.
int init_permutation_kernel()
{
    static DeviceOnce attr;
    IDTX_CUDA(once_per_device(attr, [](int dev) {
        cudaError_t e = cudaFuncSetAttribute(k_shuffle_smem<kShufPosFlag>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             shuffle_smem_bytes(kPosFlagMaxN, kShufPosFlag));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_shuffle_smem<kShufBitmap>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     shuffle_smem_bytes(65536, kShufBitmap));
        int optin = 0;
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int wide = shuffle_smem_bytes(kWideMaxN, kShufWide);
        g_shuffle_wide[dev] = e == cudaSuccess && optin >= wide;
        if (e == cudaSuccess && g_shuffle_wide[dev])
            e = cudaFuncSetAttribute(k_shuffle_smem<kShufWide>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, wide);
        return e;
    }));
    return IDTX_OK;
}

// Enqueue the surrogate permutations of n_slots rows of length n.  With
// `order` the rows shuffled in shared memory (n <= kWideMaxN) are written
// composed with it; *composed says whether they were.
int enqueue_permutations(int32_t *perm, const uint64_t *streams, const uint64_t *seeds,
                         int n_slots, int64_t n, const int32_t *order, cudaStream_t st,
                         int &launches, bool *composed)
{
    *composed = false;
    if (n_slots <= 0) return IDTX_OK;
    IDTX_TRY(init_permutation_kernel());
    int dev = 0;
    IDTX_CUDA(cudaGetDevice(&dev));
    int mode = shuffle_mode(n);
    if (mode == kShufWide && !g_shuffle_wide[dev]) mode = -1;
    const unsigned grid = (unsigned)n_slots;
    const int ni = (int)std::min<int64_t>(n, kWideMaxN);
    switch (mode) {
    case kShufPosFlag:
        k_shuffle_smem<kShufPosFlag><<<grid, 32, shuffle_smem_bytes(ni, mode), st>>>(
            perm, streams, seeds, ni, order);
        break;
    case kShufBitmap:
        k_shuffle_smem<kShufBitmap><<<grid, 32, shuffle_smem_bytes(ni, mode), st>>>(
            perm, streams, seeds, ni, order);
        break;
    case kShufWide:
        k_shuffle_smem<kShufWide><<<grid, 32, shuffle_smem_bytes(ni, mode), st>>>(
            perm, streams, seeds, ni, order);
        break;
    default:
        k_fisher_yates<<<grid, 32, 0, st>>>(perm, streams, seeds, n);
        break;
    }
    *composed = mode >= 0 && order != nullptr;
    IDTX_CUDA(cudaGetLastError());
    launches += 1;
    return IDTX_OK;
}

// The fused kernel's launch description of a group prepared into sl.
void fill_launch(const idtx_ctx *c, const Group &g, const Slices &sl, float *eps_out,
                 int32_t *cnt_out, long long timeout_ns, KsgLaunch &a)
{
    a.sh = sl.sh;
    a.xi = sl.xi;
    a.psi = c->psi;
    a.partial = sl.partial;
    a.eps_out = eps_out;
    a.cnt_out = cnt_out;
    a.order = g.sort ? (const int32_t *)sl.order : nullptr;
    a.work = (unsigned long long *)c->buf[B_WORK] + (size_t)g.work_slot * kNumWork;
    a.err = c->d_err;
    a.n = g.n;
    a.n_pad = g.n_pad;
    a.n_jobs = (int)g.jobs.size();
    a.n_qt = g.n_qt;
    a.k = g.k;
    a.timeout_ns = timeout_ns;
    a.list_a = nullptr;
    a.list_b = nullptr;
    a.lmeta = nullptr;
    a.ring = nullptr;
    a.cap_a = g.cap_a;
    a.cap_b = g.cap_b;
    if ((g.use_list || g.tune) && sl.lists) {
        const size_t oa = align_up((size_t)g.n * g.cap_a * sizeof(int2), 256);
        const size_t ob = align_up((size_t)g.n * g.cap_b * sizeof(int2), 256);
        const size_t om = align_up((size_t)g.n * sizeof(int4), 256);
        a.list_a = (const int2 *)sl.lists;
        a.list_b = (const int2 *)(sl.lists + oa);
        a.lmeta = (const int4 *)(sl.lists + oa + ob);
        a.ring = (double *)(sl.lists + oa + ob + om);
    }
}

// Enqueue the preparation of one planned group into its scratch slices
// (sample order, shared-coordinate tiles, permutations, gathered X) and fill
// the fused kernel's launch description.
int prep_group(idtx_ctx *c, const Group &g, cudaStream_t st, const Slices &sl, float *eps_out,
               int32_t *cnt_out, long long timeout_ns, KsgLaunch &a, int &launches)
{
    const unsigned char *desc = (const unsigned char *)c->buf[B_DESC];
    const Col *xc = (const Col *)(desc + g.off_x);
    const Col *yc = (const Col *)(desc + g.off_y);
    const Col *zc = (const Col *)(desc + g.off_z);
    const Job *jobs = (const Job *)(desc + g.off_jobs);
    const uint64_t *streams = (const uint64_t *)(desc + g.off_streams);
    const uint64_t *seeds = (const uint64_t *)(desc + g.off_seeds);
    float *sh = sl.sh;
    float *xi = sl.xi;
    int32_t *perm = sl.perm;
    double *partial = sl.partial;
    const KsgVariant &v = *g.v;
    const int n_jobs = (int)g.jobs.size();
    const int n_slots = (int)g.slot_stream.size();

    const int dzb = v.dz, dyb = v.dy;
    const int32_t *order = nullptr;
    launches = 0;
    if (g.sort) {
        // Order the samples along a Morton curve of the shared coordinates, so
        // that a warp's queries and a tile's references are spatial neighbours.
        unsigned char *ob = sl.order;
        const size_t col = align_up((size_t)g.n * 4, 256);
        int32_t *ord = (int32_t *)ob;
        int32_t *idx = (int32_t *)(ob + col);
        uint32_t *kin = (uint32_t *)(ob + 2 * col);
        uint32_t *kout = (uint32_t *)(ob + 3 * col);
        float *mm = (float *)(ob + 4 * col);
        int nk, bits;
        morton_shape(g.dz + g.dy, nk, bits);
        k_minmax_cols<<<nk, 256, 0, st>>>(zc, g.dz, yc, g.dy, g.n, mm);
        IDTX_CUDA(cudaGetLastError());
        k_morton_keys<<<grid_for(g.n, 256), 256, 0, st>>>(zc, g.dz, yc, nk, bits, g.n, mm, kin,
                                                          idx);
        IDTX_CUDA(cudaGetLastError());
        size_t tmp_bytes = sl.sort_cap;
        IDTX_CUDA(sort_pairs_u32(sl.sort_tmp, tmp_bytes, kin, kout, idx, ord, (int)g.n,
                                 nk * bits, st));
        order = ord;
        launches += 3;
    }
    k_pack_shared<<<grid_for(g.n_pad * v.dsp, 256), 256, 0, st>>>(
        zc, g.dz, dzb, yc, g.dy, dyb, v.dsp, g.n, g.n_pad, order, sh, c->d_err);
    IDTX_CUDA(cudaGetLastError());
    k_tile_boxes<<<(unsigned)(g.n_pad / kTJ), kTJ, 0, st>>>(sh, v.dsp, g.n);
    IDTX_CUDA(cudaGetLastError());
    fill_launch(c, g, sl, eps_out, cnt_out, timeout_ns, a);
    if ((g.use_list || g.tune) && !a.list_a)
        return fail(IDTX_EINTERNAL, "list kernel chosen without a list buffer");
    // The permutations and the X gather do not depend on the lists: with
    // lists to build they run on the context's second stream, forked from st
    // after the sample order is known and joined back before the estimator.
    cudaStream_t xs = st;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (a.list_a) {
        IDTX_TRY(take_event(c, &fork));
        IDTX_TRY(take_event(c, &join));
        IDTX_CUDA(cudaEventRecord(fork, st));
        IDTX_CUDA(cudaStreamWaitEvent(c->side_stream, fork, 0));
        xs = c->side_stream;
    }
    // Permutation rows composed with the sample order where the shuffle can
    // write them so (the gather then reads them in sequence).
    bool composed = false;
    if (n_slots > 0 && g.n_reps > 0) {
        // permutations of the replications after the sample rows, then expanded
        int32_t *blk = perm + (int64_t)n_slots * g.n;
        bool unused = false;
        IDTX_TRY(enqueue_permutations(blk, streams, seeds, n_slots, g.n_reps, nullptr, xs,
                                      launches, &unused));
        k_expand_reps<<<grid_for((int64_t)n_slots * g.n, 256), 256, 0, xs>>>(
            blk, n_slots, g.n_reps, g.n / g.n_reps, order, perm);
        IDTX_CUDA(cudaGetLastError());
        composed = order != nullptr;
        launches += 1;
    } else if (n_slots > 0) {
        IDTX_TRY(enqueue_permutations(perm, streams, seeds, n_slots, g.n, order, xs, launches,
                                      &composed));
    }
    // X of every job, permuted: gb jobs interleaved per sample row for the
    // fused kernels; the plain schedule takes each job's values on their own
    // ([job][n_pad][dx], the same bytes).
    const int gx = g.plain ? 1 : v.gb, ngx = g.plain ? n_jobs : g.n_groups;
    const int64_t gblocks = gather_blocks(ngx, g.n_pad, gx, v.dx);
    if (gblocks <= 0) return fail(IDTX_EINTERNAL, "gather shape out of range");
    k_gather_x<<<(unsigned)gblocks, kGatherThreads, gather_smem(gx, v.dx), xs>>>(
        xc, g.dx, v.dx, jobs, n_jobs, perm, g.n, g.n_pad, gx, order, composed, xi, c->d_err);
    IDTX_CUDA(cudaGetLastError());
    if (a.list_a) {
        IDTX_CUDA(cudaEventRecord(join, xs));
        IDTX_CUDA(build_lists(sh, v.dsp, v.dz, v.dz + v.dy, g.n, g.cap_a, g.cap_b,
                              const_cast<int2 *>(a.list_a), const_cast<int2 *>(a.list_b),
                              const_cast<int4 *>(a.lmeta), st));
        IDTX_CUDA(cudaStreamWaitEvent(st, join, 0));
        // a later record of these events does not disturb the waits above
        c->event_pool.push_back(fork);
        c->event_pool.push_back(join);
        launches += 1;
    }
    launches += 5;  // pack, boxes, gather, fused, finalize
    return IDTX_OK;
}

// Record a group's shape for its work counters and count its launches.
void note_group(idtx_ctx *c, const Group &g, int launches, bool list)
{
    const int n_jobs = (int)g.jobs.size();
    if (g.plain) {
        c->stats.fused_launches += n_jobs;
        c->stats.kernel_launches += launches - 1 + n_jobs;
        return;
    }
    WorkShape ws;
    ws.list = list;
    ws.dx = g.dx;
    ws.dy = g.dy;
    ws.dz_eff = std::max(g.dz, 1);
    ws.gb = g.v->gb;
    ws.job_frac = (double)n_jobs / ((double)g.n_groups * g.v->gb);
    ws.exhaustive_pairs = 2.0 * (double)g.n * (double)g.n * (double)g.n_groups;
    if ((int)c->call_shapes.size() <= g.work_slot) c->call_shapes.resize(g.work_slot + 1);
    c->call_shapes[g.work_slot] = ws;
    c->stats.fused_launches += 1;
    c->stats.kernel_launches += launches;
    if (list) c->stats.list_launches += 1;
}

// Time the candidate ways of running a prepared group -- the tile kernel, and
// the list kernel (list building included) with the group's list capacities
// and with two smaller ones -- and remember the fastest for this (variant,
// log2 N).  Every candidate writes the same partial sums.  On return the
// lists in the buffer, and a's capacities, are those of the choice.
int tune_group(idtx_ctx *c, const Group &g, KsgLaunch &a, cudaStream_t st, bool &use_list)
{
    struct Cand {
        bool list;
        int ca, cb;
        float ms;
    };
    std::vector<Cand> cands{{false, 0, 0, 0.0f}, {true, g.cap_a, g.cap_b, 0.0f}};
    if (c->cap_a == 0 && c->cap_b == 0)  // capacities not fixed by the caller
        for (int sh = 1; sh <= 2; ++sh) {
            const int ca = (g.cap_a >> sh) / 32 * 32, cb = (g.cap_b >> sh) / 32 * 32;
            if (ca >= 256 && cb >= 256) cands.push_back({true, ca, cb, 0.0f});
        }
    const KsgVariant &v = *g.v;
    KsgLaunch t = a;
    t.work = nullptr;
    std::vector<cudaEvent_t> ev(cands.size() + 1);
    for (auto &e : ev) IDTX_TRY(take_event(c, &e));
    IDTX_CUDA(cudaEventRecord(ev[0], st));
    int built_a = g.cap_a, built_b = g.cap_b;  // the lists prep_group built
    for (size_t i = 0; i < cands.size(); ++i) {
        const Cand &cd = cands[i];
        if (!cd.list) {
            IDTX_CUDA(v.fn(t, g.n_groups, st));
        } else {
            // the first list candidate re-times the build prep_group did
            IDTX_CUDA(build_lists(t.sh, v.dsp, v.dz, v.dz + v.dy, g.n, cd.ca, cd.cb,
                                  const_cast<int2 *>(t.list_a), const_cast<int2 *>(t.list_b),
                                  const_cast<int4 *>(t.lmeta), st));
            built_a = cd.ca;
            built_b = cd.cb;
            t.cap_a = cd.ca;
            t.cap_b = cd.cb;
            IDTX_CUDA(v.fn_list(t, g.n_groups, st));
        }
        IDTX_CUDA(cudaEventRecord(ev[i + 1], st));
    }
    IDTX_CUDA(cudaEventSynchronize(ev.back()));
    size_t best = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        IDTX_CUDA(cudaEventElapsedTime(&cands[i].ms, ev[i], ev[i + 1]));
        if (cands[i].ms < cands[best].ms) best = i;
    }
    for (auto &e : ev) c->event_pool.push_back(e);
    const Cand &b = cands[best];
    use_list = b.list;
    c->tuned[tune_key(g)] = idtx_ctx::Choice{b.list, b.ca, b.cb};
    if (b.list && (built_a != b.ca || built_b != b.cb)) {
        IDTX_CUDA(build_lists(a.sh, v.dsp, v.dz, v.dz + v.dy, g.n, b.ca, b.cb,
                              const_cast<int2 *>(a.list_a), const_cast<int2 *>(a.list_b),
                              const_cast<int4 *>(a.lmeta), st));
        c->stats.kernel_launches += 1;
    }
    if (b.list) {
        a.cap_a = b.ca;
        a.cap_b = b.cb;
    }
    c->stats.tune_trials += 1;
    c->stats.kernel_launches += (int64_t)(2 * cands.size() - 1);
    return IDTX_OK;
}

// Enqueue one planned group on the context's shared scratch.  cmi: device
// [n_jobs] (the group's slice).
int enqueue_group(idtx_ctx *c, const Group &g, cudaStream_t st, double *cmi, float *eps_out,
                  int32_t *cnt_out, long long timeout_ns)
{
    const Slices sl{(float *)c->buf[B_SH],       (float *)c->buf[B_XI],
                    (int32_t *)c->buf[B_PERM],   (double *)c->buf[B_PARTIAL],
                    (unsigned char *)c->buf[B_ORDER], c->buf[B_SORT], c->cap[B_SORT],
                    (unsigned char *)c->buf[B_LIST]};
    KsgLaunch a;
    int launches = 0;
    IDTX_TRY(prep_group(c, g, st, sl, eps_out, cnt_out, timeout_ns, a, launches));
    const KsgVariant &v = *g.v;
    bool use_list = g.use_list;
    if (g.tune) IDTX_TRY(tune_group(c, g, a, st, use_list));
    const int n_jobs = (int)g.jobs.size();
    float *xi = sl.xi;
    double *partial = sl.partial;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->profiling) {
        IDTX_TRY(take_event(c, &ev0));
        IDTX_TRY(take_event(c, &ev1));
        IDTX_CUDA(cudaEventRecord(ev0, st));
    }
    if (g.plain) {
        // one launch per estimate; prep_group gathered each job's X on its own
        for (int jb = 0; jb < n_jobs; ++jb)
            IDTX_CUDA(v.fn_plain(sl.sh, xi + (size_t)jb * g.n_pad * v.dx, c->psi, g.n, g.n_pad,
                                 g.k, partial + (size_t)jb * g.n_qt,
                                 eps_out ? eps_out + (size_t)jb * g.n : nullptr,
                                 cnt_out ? cnt_out + (size_t)jb * 3 * g.n : nullptr, st));
    } else if (use_list) {
        IDTX_CUDA(v.fn_list(a, g.n_groups, st));
        c->stats.list_cap_a = a.cap_a;
        c->stats.list_cap_b = a.cap_b;
    } else {
        IDTX_CUDA(v.fn(a, g.n_groups, st));
    }
    if (c->profiling) {
        IDTX_CUDA(cudaEventRecord(ev1, st));
        c->pending.emplace_back(ev0, ev1);
    }
    note_group(c, g, launches, use_list && !g.plain);
    k_finalize<<<(n_jobs + 127) / 128, 128, 0, st>>>(partial, n_jobs, g.n_qt, c->psi, g.k, g.n,
                                                      cmi);
    IDTX_CUDA(cudaGetLastError());
    return IDTX_OK;
}

// A batch of planned groups laid out for persistent fused launches: every
// group gets its own scratch slices; the groups of each kernel variant form
// the tasks of one launch, largest N first (long tasks start early).
struct BatchPlan {
    std::vector<Slices> sl;
    std::vector<const KsgVariant *> vars;
    std::vector<std::vector<int>> bucket;
    std::vector<size_t> b_probs, b_start;
    std::vector<int64_t> b_tasks;
    std::vector<int> list_groups;  // run one after another on the shared B_LIST
    KsgLaunch *probs_d = nullptr;
    int64_t *start_d = nullptr;
    int *next_d = nullptr;
};

// Host part of a batch: scratch, launch descriptions and task offsets, the
// latter uploaded to the device (B_TABLE) on st.
int batch_plan(idtx_ctx *c, const std::vector<Group> &gs, cudaStream_t st, long long timeout_ns,
               BatchPlan &bp)
{
    const size_t n = gs.size();
    std::vector<CallBuffers> off(n);
    CallBuffers tot;
    for (size_t i = 0; i < n; ++i) {
        const CallBuffers b = bytes_of(gs[i]);
        off[i] = tot;
        tot.sh += b.sh;
        tot.xi += b.xi;
        tot.perm += b.perm;
        tot.partial += b.partial;
        tot.order += b.order;
        tot.sort_tmp += b.sort_tmp;
    }
    IDTX_TRY(ensure(c, B_SH, tot.sh));
    IDTX_TRY(ensure(c, B_XI, tot.xi));
    IDTX_TRY(ensure(c, B_PERM, tot.perm));
    IDTX_TRY(ensure(c, B_PARTIAL, tot.partial));
    IDTX_TRY(ensure(c, B_ORDER, tot.order));
    IDTX_TRY(ensure(c, B_SORT, tot.sort_tmp));
    size_t list_max = 0;
    for (size_t i = 0; i < n; ++i) list_max = std::max(list_max, bytes_of(gs[i]).lists);
    IDTX_TRY(ensure(c, B_LIST, list_max));
    bp.sl.resize(n);
    for (size_t i = 0; i < n; ++i)
        bp.sl[i] = Slices{(float *)((unsigned char *)c->buf[B_SH] + off[i].sh),
                          (float *)((unsigned char *)c->buf[B_XI] + off[i].xi),
                          (int32_t *)((unsigned char *)c->buf[B_PERM] + off[i].perm),
                          (double *)((unsigned char *)c->buf[B_PARTIAL] + off[i].partial),
                          (unsigned char *)c->buf[B_ORDER] + off[i].order,
                          (unsigned char *)c->buf[B_SORT] + off[i].sort_tmp,
                          bytes_of(gs[i]).sort_tmp, (unsigned char *)c->buf[B_LIST]};

    // List-kernel groups run one by one; the others form the persistent
    // launches of their variants.
    for (size_t i = 0; i < n; ++i) {
        const Group &g = gs[i];
        if (g.use_list) {
            bp.list_groups.push_back((int)i);
            continue;
        }
        if (std::find(bp.vars.begin(), bp.vars.end(), g.v) == bp.vars.end()) bp.vars.push_back(g.v);
    }
    const size_t nv = bp.vars.size();
    bp.bucket.assign(nv, {});
    for (size_t i = 0; i < n; ++i)
        if (!gs[i].use_list)
            bp.bucket[std::find(bp.vars.begin(), bp.vars.end(), gs[i].v) - bp.vars.begin()]
                .push_back((int)i);
    for (auto &b : bp.bucket)
        std::stable_sort(b.begin(), b.end(), [&](int x, int y) { return gs[x].n > gs[y].n; });

    std::vector<KsgLaunch> probs(n);
    std::vector<int64_t> start;
    bp.b_probs.assign(nv, 0);
    bp.b_start.assign(nv, 0);
    bp.b_tasks.assign(nv, 0);
    size_t at = 0;
    for (size_t b = 0; b < nv; ++b) {
        bp.b_probs[b] = at;
        bp.b_start[b] = start.size();
        int64_t t = 0;
        for (int i : bp.bucket[b]) {
            fill_launch(c, gs[i], bp.sl[i], nullptr, nullptr, timeout_ns, probs[at++]);
            start.push_back(t);
            t += (int64_t)gs[i].n_qt * gs[i].n_groups;
        }
        start.push_back(t);
        bp.b_tasks[b] = t;
    }
    const size_t probs_bytes = align_up(n * sizeof(KsgLaunch), 256);
    const size_t start_bytes = align_up(start.size() * sizeof(int64_t), 256);
    IDTX_TRY(ensure(c, B_TABLE, probs_bytes + start_bytes + nv * sizeof(int)));
    unsigned char *tb = (unsigned char *)c->buf[B_TABLE];
    bp.probs_d = (KsgLaunch *)tb;
    bp.start_d = (int64_t *)(tb + probs_bytes);
    bp.next_d = (int *)(tb + probs_bytes + start_bytes);
    IDTX_CUDA(cudaMemcpyAsync(bp.probs_d, probs.data(), n * sizeof(KsgLaunch),
                              cudaMemcpyHostToDevice, st));
    IDTX_CUDA(cudaMemcpyAsync(bp.start_d, start.data(), start.size() * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    return IDTX_OK;
}

// Device part of a batch (stream operations only, so it can be captured):
// prepare every group, reset the task counters, one persistent fused launch
// per variant, finalise every group.  cmi: device [sum of jobs], group g's
// slice at g.off_cmi.
int batch_enqueue(idtx_ctx *c, const std::vector<Group> &gs, const BatchPlan &bp,
                  cudaStream_t st, double *cmi, long long timeout_ns)
{
    const size_t n = gs.size(), nv = bp.vars.size();
    std::vector<int> launches(n, 0);
    for (size_t i = 0; i < n; ++i) {
        if (gs[i].use_list) continue;
        KsgLaunch unused;
        IDTX_TRY(prep_group(c, gs[i], st, bp.sl[i], nullptr, nullptr, timeout_ns, unused,
                            launches[i]));
    }
    IDTX_CUDA(cudaMemsetAsync(bp.next_d, 0, nv * sizeof(int), st));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->profiling) {
        IDTX_TRY(take_event(c, &ev0));
        IDTX_TRY(take_event(c, &ev1));
        IDTX_CUDA(cudaEventRecord(ev0, st));
    }
    for (size_t b = 0; b < nv; ++b) {
        KsgTable t;
        t.probs = bp.probs_d + bp.b_probs[b];
        t.start = bp.start_d + bp.b_start[b];
        t.next = bp.next_d + b;
        t.n_probs = (int)bp.bucket[b].size();
        t.n_tasks = bp.b_tasks[b];
        IDTX_CUDA(bp.vars[b]->fn_table(t, st));
    }
    if (c->profiling) {
        IDTX_CUDA(cudaEventRecord(ev1, st));
        c->pending.emplace_back(ev0, ev1);
    }
    for (int i : bp.list_groups) {
        const Group &g = gs[i];
        KsgLaunch a;
        IDTX_TRY(prep_group(c, g, st, bp.sl[i], nullptr, nullptr, timeout_ns, a, launches[i]));
        a.work = (unsigned long long *)c->buf[B_WORK] + (size_t)g.work_slot * kNumWork;
        cudaEvent_t l0 = nullptr, l1 = nullptr;
        if (c->profiling) {
            IDTX_TRY(take_event(c, &l0));
            IDTX_TRY(take_event(c, &l1));
            IDTX_CUDA(cudaEventRecord(l0, st));
        }
        IDTX_CUDA(g.v->fn_list(a, g.n_groups, st));
        c->stats.list_cap_a = a.cap_a;
        c->stats.list_cap_b = a.cap_b;
        if (c->profiling) {
            IDTX_CUDA(cudaEventRecord(l1, st));
            c->pending.emplace_back(l0, l1);
        }
    }
    for (size_t i = 0; i < n; ++i) {
        const Group &g = gs[i];
        const int n_jobs = (int)g.jobs.size();
        note_group(c, g, launches[i], g.use_list);
        k_finalize<<<(n_jobs + 127) / 128, 128, 0, st>>>(bp.sl[i].partial, n_jobs, g.n_qt,
                                                          c->psi, g.k, g.n, cmi + g.off_cmi);
        IDTX_CUDA(cudaGetLastError());
    }
    // One fused launch per variant instead of one per tile-kernel group.
    const int64_t n_tile = (int64_t)(n - bp.list_groups.size());
    c->stats.fused_launches -= n_tile - (int64_t)nv;
    c->stats.kernel_launches -= n_tile - (int64_t)nv;
    return IDTX_OK;
}

// Settle the kernel choice of every group whose shape is not tuned yet, by a
// timed trial on that group (prepared into the single-group scratch; the
// descriptors must already be in B_DESC).  Runs outside any stream capture.
int resolve_tuning(idtx_ctx *c, std::vector<Group> &gs, cudaStream_t st, long long timeout_ns)
{
    for (Group &g : gs) {
        if (!g.tune) continue;
        if (c->tuned.find(tune_key(g)) == c->tuned.end()) {
            CallBuffers b;
            sizes_of(g, b);
            IDTX_TRY(ensure(c, B_SH, b.sh));
            IDTX_TRY(ensure(c, B_XI, b.xi));
            IDTX_TRY(ensure(c, B_PERM, b.perm));
            IDTX_TRY(ensure(c, B_PARTIAL, b.partial));
            IDTX_TRY(ensure(c, B_ORDER, b.order));
            IDTX_TRY(ensure(c, B_SORT, b.sort_tmp));
            IDTX_TRY(ensure(c, B_LIST, b.lists));
            const Slices sl{(float *)c->buf[B_SH],       (float *)c->buf[B_XI],
                            (int32_t *)c->buf[B_PERM],   (double *)c->buf[B_PARTIAL],
                            (unsigned char *)c->buf[B_ORDER], c->buf[B_SORT], c->cap[B_SORT],
                            (unsigned char *)c->buf[B_LIST]};
            KsgLaunch a;
            int launches = 0;
            IDTX_TRY(prep_group(c, g, st, sl, nullptr, nullptr, timeout_ns, a, launches));
            bool unused = false;
            IDTX_TRY(tune_group(c, g, a, st, unused));
            c->stats.kernel_launches += launches - 2;
        }
        const idtx_ctx::Choice ch = c->tuned[tune_key(g)];
        g.use_list = ch.list;
        if (ch.list) {
            g.cap_a = ch.cap_a;
            g.cap_b = ch.cap_b;
        }
        g.tune = false;
    }
    return IDTX_OK;
}

// Copy the caller's columns (host memory) into device scratch; returns the
// device base and sets the leading dimension to n.
struct HostCopy {
    const float *src;
    int dims;
    int64_t ld;
    size_t off;  // float offset in B_IN
};

// Reset the per-call work counters for n_slots fused launches.
int begin_call(idtx_ctx *c, int n_slots, cudaStream_t st)
{
    c->call_shapes.clear();
    const size_t bytes = (size_t)std::max(n_slots, 1) * kNumWork * sizeof(unsigned long long);
    IDTX_TRY(ensure(c, B_WORK, bytes));
    if (c->h_work_cap < bytes) {
        if (c->h_work) cudaFreeHost(c->h_work);
        c->h_work = nullptr;
        c->h_work_cap = 0;
        IDTX_CUDA(cudaMallocHost(&c->h_work, bytes));
        c->h_work_cap = bytes;
    }
    IDTX_CUDA(cudaMemsetAsync(c->buf[B_WORK], 0, bytes, st));
    IDTX_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    return IDTX_OK;
}

int finish_call(idtx_ctx *c, cudaStream_t st)
{
    IDTX_CUDA(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    const size_t n_shapes = c->call_shapes.size();
    if (n_shapes)
        IDTX_CUDA(cudaMemcpyAsync(c->h_work, c->buf[B_WORK],
                                  n_shapes * kNumWork * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st));
    IDTX_CUDA(cudaStreamSynchronize(st));
    for (size_t w = 0; w < n_shapes; ++w) {
        // Algorithmic lane operations of the work the fused kernel did:
        //  neighbour pass: per scanned pair 2(dy+dz')+1 (|d| and max per shared
        //    dimension, bound compare); per passing pair and job 2dx+1;
        //  count pass: per scanned pair 2dz'+1; per passing pair 2dy (Y
        //    distance) and per job 2dx+7 (X distance, three compares, three adds).
        const WorkShape &ws = c->call_shapes[w];
        const unsigned long long *k = c->h_work + w * kNumWork;
        const double jobs = ws.gb * ws.job_frac;
        c->stats.exhaustive_pairs += ws.exhaustive_pairs;
        if (ws.list) {
            // List kernel.  A list A entry a warp walks shared costs every
            // job of the warp 2dx+2 (X distance, max with d_YZ, compare), a
            // list B entry 2dx+4 (X distance, two compares, two adds): those
            // two counters are per (query, group) and scale with the jobs.
            // A full-scan sample costs 2(dx+dy+dz')+2 (pass A) or +6 (pass
            // B) for the one job being rescanned, a (job, entry) pair of the
            // count walk's repacked phases 2dx+4 and of the neighbour walk's
            // lane-split tails 2dx+2: those counters are already per job.
            // The useful part: n_yz entries of list A and n_z of list B per
            // (query, job), what a walk visiting exactly the entries each job
            // needs would do.
            const double dall = 2.0 * (ws.dx + ws.dy + ws.dz_eff);
            c->stats.fused_lane_ops += jobs * ((double)k[0] * (2.0 * ws.dx + 2.0) +
                                               (double)k[1] * (2.0 * ws.dx + 4.0)) +
                                      (double)k[2] * (dall + 2.0) +
                                      (double)k[3] * (dall + 6.0) +
                                      (double)k[6] * (2.0 * ws.dx + 4.0) +
                                      (double)k[7] * (2.0 * ws.dx + 2.0);
            c->stats.useful_lane_ops += (double)k[8] * (2.0 * ws.dx + 4.0) +
                                        (double)k[9] * (2.0 * ws.dx + 2.0);
            c->stats.list_sum_nz += (double)k[8];
            c->stats.list_sum_nyz += (double)k[9];
            c->stats.list_tail_b += (double)k[6];
            c->stats.list_tail_a += (double)k[7];
            c->stats.list_walk_a += (double)k[0];
            c->stats.list_walk_b += (double)k[1];
            c->stats.brute_samples += (double)(k[2] + k[3]);
            c->stats.fallbacks += (double)k[4];
            c->stats.warp_cycles += (double)k[5];
            continue;
        }
        c->stats.fused_lane_ops += (double)k[0] * (2.0 * (ws.dy + ws.dz_eff) + 1.0) +
                                   (double)k[1] * jobs * (2.0 * ws.dx + 1.0) +
                                   (double)k[2] * (2.0 * ws.dz_eff + 1.0) +
                                   (double)k[3] * (2.0 * ws.dy + jobs * (2.0 * ws.dx + 7.0));
        c->stats.scanned_a += (double)k[0];
        c->stats.passed_a += (double)k[1];
        c->stats.scanned_b += (double)k[2];
        c->stats.passed_b += (double)k[3];
        c->stats.wait_cycles += (double)k[4];
        c->stats.warp_cycles += (double)k[5];
    }
    c->call_shapes.clear();
    for (auto &pe : c->pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, pe.first, pe.second) == cudaSuccess) c->stats.fused_ms += ms;
        c->event_pool.push_back(pe.first);
        c->event_pool.push_back(pe.second);
    }
    c->pending.clear();
    const int e = *c->h_err;
    if (e & kErrNonFinite) return fail(IDTX_EINVAL, "input contains NaN or Inf");
    if (e & kErrTimeout) return fail(IDTX_ETIMEOUT, "a bounded device wait ran out");
    if (e) return fail(IDTX_EINTERNAL, "device error word 0x%x", e);
    return IDTX_OK;
}

long long timeout_of(const idtx_settings *s)
{
    const long long ms = (s && s->timeout_ms > 0) ? s->timeout_ms : 2000;
    return ms * 1000000ll;
}

// The bound of the device waits of a call on c: the context's limit if one
// is set (idtx_ctx_set_wait_limit_ns), else the settings'.
long long timeout_of(const idtx_ctx *c, const idtx_settings *s)
{
    return c->wait_ns > 0 ? c->wait_ns : timeout_of(s);
}

int check_cols(const float *p, int dims, const char *name)
{
    if (dims > 0 && !p) return fail(IDTX_EINVAL, "%s is NULL", name);
    return IDTX_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int idtx_version(void) { return 100; }

const char *idtx_last_error(void) { return t_err.c_str(); }

int idtx_ctx_create(idtx_ctx **out, int device)
{
    if (!out) return fail(IDTX_EINVAL, "ctx is NULL");
    *out = nullptr;
    int n_dev = 0;
    IDTX_CUDA(cudaGetDeviceCount(&n_dev));
    if (device < 0 || device >= n_dev) return fail(IDTX_EINVAL, "device %d out of range", device);
    DeviceGuard guard(device);
    idtx_ctx *c = new idtx_ctx();
    c->device = device;
    KsgVariant tmp[64];
    int n = 0;
    n += ksg_variants_d11(tmp + n);
    n += ksg_variants_d12(tmp + n);
    n += ksg_variants_d21(tmp + n);
    n += ksg_variants_d22(tmp + n);
    n += ksg_variants_generic(tmp + n);
    c->variants.assign(tmp, tmp + n);
    cudaError_t e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        idtx_ctx_destroy(c);
        return fail(IDTX_ENOMEM, "context allocation failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return IDTX_OK;
}

int idtx_ctx_set_profiling(idtx_ctx *c, int enable)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    c->profiling = enable != 0;
    return IDTX_OK;
}

int idtx_ctx_set_graphs(idtx_ctx *c, int enable)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    c->graphs = enable != 0;
    if (!c->graphs) drop_graph(c);
    return IDTX_OK;
}

int idtx_ctx_set_kernel(idtx_ctx *c, int kernel)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (kernel != IDTX_KERNEL_AUTO && kernel != IDTX_KERNEL_TILE && kernel != IDTX_KERNEL_LIST)
        return fail(IDTX_EINVAL, "unknown kernel choice %d", kernel);
    DeviceGuard guard(c->device);
    c->kernel_pref = kernel;
    drop_graph(c);
    return IDTX_OK;
}

int idtx_ctx_set_list_caps(idtx_ctx *c, int cap_a, int cap_b)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    auto bad = [](int v, int mx) { return v != 0 && (v < 32 || v > mx || v % 32 != 0); };
    if (bad(cap_a, kMaxListA) || bad(cap_b, kMaxListB))
        return fail(IDTX_EINVAL, "list capacities %d, %d: 0 or multiples of 32 up to %d, %d",
                    cap_a, cap_b, kMaxListA, kMaxListB);
    DeviceGuard guard(c->device);
    c->cap_a = cap_a;
    c->cap_b = cap_b;
    c->tuned.clear();
    drop_graph(c);
    return IDTX_OK;
}

int idtx_ctx_set_wait_limit_ns(idtx_ctx *c, int64_t ns)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (ns < 0) return fail(IDTX_EINVAL, "wait limit %lld ns is negative", (long long)ns);
    c->wait_ns = ns;
    return IDTX_OK;
}

int idtx_ctx_get_stats(idtx_ctx *c, idtx_stats *out)
{
    if (!c || !out) return fail(IDTX_EINVAL, "NULL argument");
    *out = c->stats;
    return IDTX_OK;
}

int idtx_ctx_reset_stats(idtx_ctx *c)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    c->stats = idtx_stats{};
    return IDTX_OK;
}

int idtx_ctx_destroy(idtx_ctx *c)
{
    if (!c) return IDTX_OK;
    DeviceGuard guard(c->device);
    cudaDeviceSynchronize();
    for (auto &pe : c->pending) c->event_pool.push_back(pe.first), c->event_pool.push_back(pe.second);
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    drop_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    for (int i = 0; i < kNumBufs; ++i) {
        if (c->buf[i]) cudaFree(c->buf[i]);
        if (c->gbuf[i]) cudaFree(c->gbuf[i]);
    }
    if (c->psi) cudaFree(c->psi);
    if (c->d_err) cudaFree(c->d_err);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_work) cudaFreeHost(c->h_work);
    delete c;
    return IDTX_OK;
}

static int cmi_ksg_impl(idtx_ctx *c, const float *x, int dx, const float *y, int dy,
                        const float *z, int dz, int64_t n, int64_t ld, int64_t n_reps,
                        const idtx_settings *s, double *cmi_out, float *eps_out,
                        int32_t *counts_out, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!s) return fail(IDTX_EINVAL, "settings is NULL");
    if (!cmi_out) return fail(IDTX_EINVAL, "cmi_out is NULL");
    if (dx < 1 || dx > IDTX_MAX_DX || dy < 1 || dy > IDTX_MAX_DY || dz < 0 || dz > IDTX_MAX_DZ)
        return fail(IDTX_EINVAL, "dims out of range (dx=%d dy=%d dz=%d)", dx, dy, dz);
    if (n < 2 || n > IDTX_MAX_N || ld < n)
        return fail(IDTX_EINVAL, "bad n=%lld / ld=%lld", (long long)n, (long long)ld);
    if (s->k < 1 || s->k > IDTX_MAX_K || s->k > n - 1)
        return fail(IDTX_EINVAL, "k=%d out of range for n=%lld", s->k, (long long)n);
    if (s->n_surr < 0) return fail(IDTX_EINVAL, "n_surr < 0");
    if (s->mode != IDTX_MODE_BATCHED && s->mode != IDTX_MODE_PLAIN)
        return fail(IDTX_EINVAL, "unknown mode %d", s->mode);
    IDTX_TRY(check_cols(x, dx, "x"));
    IDTX_TRY(check_cols(y, dy, "y"));
    IDTX_TRY(check_cols(z, dz, "z"));
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_jobs = 1 + s->n_surr;

    // Inputs: device pointers are used in place, host pointers are copied.
    const float *src[3] = {x, y, z};
    const int dims[3] = {dx, dy, dz};
    const float *dev[3] = {x, y, z};
    int64_t lds[3] = {ld, ld, ld};
    size_t in_floats = 0;
    bool host[3] = {false, false, false};
    for (int t = 0; t < 3; ++t)
        if (dims[t] > 0 && !device_accessible(src[t])) {
            host[t] = true;
            in_floats += (size_t)dims[t] * (size_t)n;
        }
    IDTX_TRY(ensure(c, B_IN, in_floats * sizeof(float)));
    IDTX_TRY(begin_call(c, 1, st));
    {
        size_t off = 0;
        for (int t = 0; t < 3; ++t)
            if (host[t]) {
                float *d = (float *)c->buf[B_IN] + off;
                IDTX_CUDA(cudaMemcpy2DAsync(d, (size_t)n * sizeof(float), src[t],
                                            (size_t)ld * sizeof(float), (size_t)n * sizeof(float),
                                            (size_t)dims[t], cudaMemcpyHostToDevice, st));
                dev[t] = d;
                lds[t] = n;
                off += (size_t)dims[t] * (size_t)n;
            }
    }

    std::vector<Group> gs(1);
    Group &g = gs[0];
    g.n = n;
    g.dx = dx;
    g.dy = dy;
    g.dz = dz;
    g.k = s->k;
    for (int d = 0; d < dx; ++d) g.xcols.push_back(Col{dev[0] + d * lds[0], 0});
    for (int d = 0; d < dy; ++d) g.ycols.push_back(Col{dev[1] + d * lds[1], 0});
    for (int d = 0; d < dz; ++d) g.zcols.push_back(Col{dev[2] + d * lds[2], 0});
    g.jobs.push_back(Job{0, -1});
    for (int sidx = 0; sidx < s->n_surr; ++sidx) {
        g.jobs.push_back(Job{0, sidx});
        g.slot_stream.push_back((uint64_t)sidx);
        g.slot_seed.push_back(s->seed);
    }
    g.plain = s->mode == IDTX_MODE_PLAIN;
    g.n_reps = n_reps;
    IDTX_TRY(plan(c, g));
    std::vector<unsigned char> arena;
    pack_desc(gs, arena);
    CallBuffers b;
    sizes_of(g, b);
    const bool eps_dev = eps_out && device_accessible(eps_out);
    const bool cnt_dev = counts_out && device_accessible(counts_out);
    const bool cmi_dev = device_accessible(cmi_out);
    IDTX_TRY(ensure(c, B_DESC, arena.size()));
    IDTX_TRY(ensure(c, B_SH, b.sh));
    IDTX_TRY(ensure(c, B_XI, b.xi));
    IDTX_TRY(ensure(c, B_PERM, b.perm));
    IDTX_TRY(ensure(c, B_PARTIAL, b.partial));
    IDTX_TRY(ensure(c, B_ORDER, b.order));
    IDTX_TRY(ensure(c, B_SORT, b.sort_tmp));
    IDTX_TRY(ensure(c, B_LIST, b.lists));
    IDTX_TRY(ensure(c, B_CMI, (size_t)n_jobs * sizeof(double)));
    if (eps_out && !eps_dev) IDTX_TRY(ensure(c, B_EPS, (size_t)n_jobs * n * sizeof(float)));
    if (counts_out && !cnt_dev)
        IDTX_TRY(ensure(c, B_CNT, (size_t)n_jobs * 3 * n * sizeof(int32_t)));
    IDTX_TRY(ensure_psi(c, std::max<int64_t>(n, s->k) + 1, st));
    IDTX_CUDA(cudaMemcpyAsync(c->buf[B_DESC], arena.data(), arena.size(), cudaMemcpyHostToDevice,
                              st));
    float *eps_d = eps_out ? (eps_dev ? eps_out : (float *)c->buf[B_EPS]) : nullptr;
    int32_t *cnt_d = counts_out ? (cnt_dev ? counts_out : (int32_t *)c->buf[B_CNT]) : nullptr;
    double *cmi_d = (double *)c->buf[B_CMI];
    IDTX_TRY(enqueue_group(c, g, st, cmi_d, eps_d, cnt_d, timeout_of(c, s)));
    IDTX_CUDA(cudaMemcpyAsync(cmi_out, cmi_d, (size_t)n_jobs * sizeof(double),
                              cmi_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (eps_out && !eps_dev)
        IDTX_CUDA(cudaMemcpyAsync(eps_out, eps_d, (size_t)n_jobs * n * sizeof(float),
                                  cudaMemcpyDeviceToHost, st));
    if (counts_out && !cnt_dev)
        IDTX_CUDA(cudaMemcpyAsync(counts_out, cnt_d, (size_t)n_jobs * 3 * n * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st));
    return finish_call(c, st);
}

int idtx_cmi_ksg(idtx_ctx *c, const float *x, int dx, const float *y, int dy, const float *z,
                 int dz, int64_t n, int64_t ld, const idtx_settings *s, double *cmi_out,
                 float *eps_out, int32_t *counts_out, void *stream)
{
    return cmi_ksg_impl(c, x, dx, y, dy, z, dz, n, ld, 0, s, cmi_out, eps_out, counts_out, stream);
}

int idtx_cmi_ksg_reps(idtx_ctx *c, const float *x, int dx, const float *y, int dy, const float *z,
                      int dz, int64_t n, int64_t ld, int64_t n_reps, const idtx_settings *s,
                      double *cmi_out, float *eps_out, int32_t *counts_out, void *stream)
{
    if (n_reps < 1 || n_reps > n || (n_reps > 0 && n % n_reps != 0))
        return fail(IDTX_EINVAL, "n_reps=%lld must divide n=%lld", (long long)n_reps,
                    (long long)n);
    return cmi_ksg_impl(c, x, dx, y, dy, z, dz, n, ld, n_reps, s, cmi_out, eps_out, counts_out,
                        stream);
}

int idtx_cmi_batch(idtx_ctx *c, const idtx_problem *probs, int n_probs, int k, double *out,
                   void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!probs || n_probs < 1 || !out) return fail(IDTX_EINVAL, "bad problem list or output");
    if (k < 1 || k > IDTX_MAX_K) return fail(IDTX_EINVAL, "k=%d out of range", k);
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;

    size_t in_floats = 0;
    int64_t n_max = 0;
    size_t total_jobs = 0;
    std::vector<std::array<bool, 3>> host(n_probs);
    for (int p = 0; p < n_probs; ++p) {
        const idtx_problem &q = probs[p];
        if (q.dx < 1 || q.dx > IDTX_MAX_DX || q.dy < 1 || q.dy > IDTX_MAX_DY || q.dz < 0 ||
            q.dz > IDTX_MAX_DZ)
            return fail(IDTX_EINVAL, "problem %d: dims out of range", p);
        if (q.n < 2 || q.n > IDTX_MAX_N || q.ld < q.n || k > q.n - 1 || q.n_surr < 0)
            return fail(IDTX_EINVAL, "problem %d: bad n/ld/k/n_surr", p);
        IDTX_TRY(check_cols(q.x, q.dx, "x"));
        IDTX_TRY(check_cols(q.y, q.dy, "y"));
        IDTX_TRY(check_cols(q.z, q.dz, "z"));
        const float *src[3] = {q.x, q.y, q.z};
        const int dims[3] = {q.dx, q.dy, q.dz};
        for (int t = 0; t < 3; ++t) {
            host[p][t] = dims[t] > 0 && !device_accessible(src[t]);
            if (host[p][t]) in_floats += (size_t)dims[t] * (size_t)q.n;
        }
        n_max = std::max(n_max, q.n);
        total_jobs += 1 + (size_t)q.n_surr;
    }
    // CUDA-graph replay: same arguments as the captured call, all on the device.
    const bool use_graph = c->graphs && !c->profiling && in_floats == 0;
    const cudaMemcpyKind out_kind =
        device_accessible(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    std::vector<uint64_t> key;
    if (use_graph) {
        key = {(uint64_t)n_probs, (uint64_t)k, (uint64_t)(uintptr_t)stream,
               (uint64_t)(uintptr_t)c->psi};
        for (int p = 0; p < n_probs; ++p) {
            const idtx_problem &q = probs[p];
            const uint64_t w[] = {(uint64_t)(uintptr_t)q.x, (uint64_t)(uintptr_t)q.y,
                                  (uint64_t)(uintptr_t)q.z, (uint64_t)q.dx, (uint64_t)q.dy,
                                  (uint64_t)q.dz, (uint64_t)q.n, (uint64_t)q.ld,
                                  (uint64_t)q.n_surr, q.seed};
            key.insert(key.end(), w, w + 10);
        }
        if (c->graph_exec && key == c->graph_key) {
            IDTX_TRY(begin_call(c, n_probs, st));
            IDTX_CUDA(cudaGraphLaunch(c->graph_exec, st));
            c->stats.graph_launches += 1;
            IDTX_CUDA(cudaMemcpyAsync(out, c->gbuf[B_CMI], total_jobs * sizeof(double), out_kind,
                                      st));
            return finish_call(c, st);
        }
        drop_graph(c);
    }
    IDTX_TRY(ensure(c, B_IN, in_floats * sizeof(float)));
    IDTX_TRY(begin_call(c, n_probs, st));
    std::vector<Group> gs(n_probs);
    size_t in_off = 0, job_off = 0;
    for (int p = 0; p < n_probs; ++p) {
        const idtx_problem &q = probs[p];
        const float *src[3] = {q.x, q.y, q.z};
        const int dims[3] = {q.dx, q.dy, q.dz};
        const float *dev[3] = {q.x, q.y, q.z};
        int64_t lds[3] = {q.ld, q.ld, q.ld};
        for (int t = 0; t < 3; ++t)
            if (host[p][t]) {
                float *d = (float *)c->buf[B_IN] + in_off;
                IDTX_CUDA(cudaMemcpy2DAsync(d, (size_t)q.n * sizeof(float), src[t],
                                            (size_t)q.ld * sizeof(float),
                                            (size_t)q.n * sizeof(float), (size_t)dims[t],
                                            cudaMemcpyHostToDevice, st));
                dev[t] = d;
                lds[t] = q.n;
                in_off += (size_t)dims[t] * (size_t)q.n;
            }
        Group &g = gs[p];
        g.n = q.n;
        g.dx = q.dx;
        g.dy = q.dy;
        g.dz = q.dz;
        g.k = k;
        for (int d = 0; d < q.dx; ++d) g.xcols.push_back(Col{dev[0] + d * lds[0], 0});
        for (int d = 0; d < q.dy; ++d) g.ycols.push_back(Col{dev[1] + d * lds[1], 0});
        for (int d = 0; d < q.dz; ++d) g.zcols.push_back(Col{dev[2] + d * lds[2], 0});
        g.jobs.push_back(Job{0, -1});
        for (int sidx = 0; sidx < q.n_surr; ++sidx) {
            g.jobs.push_back(Job{0, sidx});
            g.slot_stream.push_back((uint64_t)sidx);
            g.slot_seed.push_back(q.seed);
        }
        IDTX_TRY(plan(c, g));
        g.work_slot = p;
        g.off_cmi = job_off;
        job_off += g.jobs.size();
    }
    std::vector<unsigned char> arena;
    pack_desc(gs, arena);
    const long long tmo = timeout_of(c, nullptr);
    IDTX_TRY(ensure_psi(c, std::max<int64_t>(n_max, k) + 1, st));
    // Shapes met for the first time: time both kernels on them now (on the
    // context's own buffers, before any capture).
    if (std::any_of(gs.begin(), gs.end(), [](const Group &g) { return g.tune; })) {
        IDTX_TRY(ensure(c, B_DESC, arena.size()));
        IDTX_CUDA(cudaMemcpyAsync(c->buf[B_DESC], arena.data(), arena.size(),
                                  cudaMemcpyHostToDevice, st));
        IDTX_TRY(resolve_tuning(c, gs, st, tmo));
    }
    if (use_graph) {
        // Capture into a graph that owns its scratch: plan and upload on st
        // with the graph's buffers in place, record the device work on the
        // capture stream, launch the graph on st.
        key[3] = (uint64_t)(uintptr_t)c->psi;
        if (!c->cap_stream)
            IDTX_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        swap_buffer_sets(c);
        int rc = IDTX_OK;
        cudaGraph_t graph = nullptr;
        BatchPlan bp;
        rc = ensure(c, B_DESC, arena.size());
        if (rc == IDTX_OK) rc = ensure(c, B_CMI, total_jobs * sizeof(double));
        if (rc == IDTX_OK) rc = ensure(c, B_WORK, (size_t)n_probs * kNumWork * 8);
        if (rc == IDTX_OK) rc = batch_plan(c, gs, st, tmo, bp);
        if (rc == IDTX_OK && cudaMemcpyAsync(c->buf[B_DESC], arena.data(), arena.size(),
                                             cudaMemcpyHostToDevice, st) != cudaSuccess)
            rc = fail(IDTX_ECUDA, "descriptor upload failed");
        // one-time kernel attributes and occupancy queries, outside the capture
        if (rc == IDTX_OK) rc = init_permutation_kernel();
        // events for the fork and join of every group, created before the capture
        for (size_t i = c->event_pool.size(); rc == IDTX_OK && i < 2 * gs.size() + 4; ++i) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreate(&ev) != cudaSuccess)
                rc = fail(IDTX_ECUDA, "event creation failed");
            else
                c->event_pool.push_back(ev);
        }
        if (rc == IDTX_OK && build_lists(nullptr, 4, 1, 1, 0, 0, 0, nullptr, nullptr, nullptr, st) !=
                                 cudaSuccess)
            rc = fail(IDTX_ECUDA, "list kernel attribute setup failed");
        for (const KsgVariant *v : bp.vars)
            if (rc == IDTX_OK && v->fn_table(KsgTable{nullptr, nullptr, nullptr, 0, 0}, st) !=
                                     cudaSuccess)
                rc = fail(IDTX_ECUDA, "kernel attribute setup failed");
        for (const Group &g : gs)
            if (rc == IDTX_OK && g.use_list) {
                KsgLaunch none{};  // no tiles: set-up only
                if (g.v->fn_list(none, 0, st) != cudaSuccess)
                    rc = fail(IDTX_ECUDA, "list kernel attribute setup failed");
            }
        if (rc == IDTX_OK) {
            if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess) {
                rc = fail(IDTX_ECUDA, "stream capture could not start");
            } else {
                rc = batch_enqueue(c, gs, bp, c->cap_stream, (double *)c->buf[B_CMI], tmo);
                const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
                if (rc == IDTX_OK && e != cudaSuccess)
                    rc = fail(IDTX_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
            }
        }
        if (rc == IDTX_OK) {
            const cudaError_t e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
            if (e != cudaSuccess) {
                c->graph_exec = nullptr;
                rc = fail(IDTX_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
            }
        }
        if (graph) cudaGraphDestroy(graph);
        swap_buffer_sets(c);
        c->call_shapes.clear();  // the graph's work counters are not read back
        if (rc != IDTX_OK) {
            drop_graph(c);
            cudaGetLastError();
            return rc;
        }
        c->graph_key = key;
        IDTX_CUDA(cudaGraphLaunch(c->graph_exec, st));
        c->stats.graph_launches += 1;
        IDTX_CUDA(
            cudaMemcpyAsync(out, c->gbuf[B_CMI], total_jobs * sizeof(double), out_kind, st));
        return finish_call(c, st);
    }
    IDTX_TRY(ensure(c, B_DESC, arena.size()));
    IDTX_TRY(ensure(c, B_CMI, total_jobs * sizeof(double)));
    IDTX_CUDA(cudaMemcpyAsync(c->buf[B_DESC], arena.data(), arena.size(), cudaMemcpyHostToDevice,
                              st));
    double *cmi_d = (double *)c->buf[B_CMI];
    BatchPlan bp;
    IDTX_TRY(batch_plan(c, gs, st, tmo, bp));
    IDTX_TRY(batch_enqueue(c, gs, bp, st, cmi_d, tmo));
    IDTX_CUDA(cudaMemcpyAsync(out, cmi_d, total_jobs * sizeof(double), out_kind, st));
    return finish_call(c, st);
}

}  // extern "C"

namespace {

// One greedy step; allowed (nullable) [n_proc * n_lags] limits the candidates
// to the ids it marks (the target-past selection uses the target's own).
int mte_step_impl(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target, int n_past,
                  int min_lag, int max_lag, const int32_t *selected, int n_selected,
                  int step_index, const idtx_settings *s, idtx_step *result, double *est_out,
                  const char *allowed, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!s || !result || !series) return fail(IDTX_EINVAL, "NULL settings/result/series");
    if (n_proc < 1 || target < 0 || target >= n_proc || n_past < 0 || min_lag < 1 ||
        max_lag < min_lag || n_selected < 0 || (n_selected > 0 && !selected) || step_index < 0 ||
        step_index >= (1 << 16))
        return fail(IDTX_EINVAL, "bad greedy-step arguments");
    const int n_lags = max_lag - min_lag + 1;
    const int n_cand_total = n_proc * n_lags;
    if (n_cand_total >= (1 << 24)) return fail(IDTX_EINVAL, "too many candidates");
    const int64_t L = std::max(max_lag, n_past);
    if (T <= L || T - L > IDTX_MAX_N) return fail(IDTX_EINVAL, "bad T for the lags");
    const int64_t n = T - L;
    if (s->k < 1 || s->k > IDTX_MAX_K || s->k > n - 1) return fail(IDTX_EINVAL, "bad k");
    if (s->n_surr < 1 || s->n_surr >= (1 << 24)) return fail(IDTX_EINVAL, "n_surr out of range");
    if (!(s->alpha > 0.0 && s->alpha < 1.0)) return fail(IDTX_EINVAL, "alpha out of (0,1)");
    if (s->mode != IDTX_MODE_BATCHED && s->mode != IDTX_MODE_PLAIN &&
        s->mode != IDTX_MODE_SCREENED)
        return fail(IDTX_EINVAL, "unknown mode %d", s->mode);
    const bool screened = s->mode == IDTX_MODE_SCREENED;
    if (screened && !c->has_screen)
        return fail(IDTX_EINVAL, "screened mode needs a screen (idtx_screen_set)");
    const int s0 = screened ? c->screen.s0 : s->n_surr;
    if (screened && (s0 < 1 || s0 >= s->n_surr))
        return fail(IDTX_EINVAL, "screen s0=%d must be in [1, n_surr)", s0);
    const int dz = n_past + n_selected;
    if (dz > IDTX_MAX_DZ) return fail(IDTX_EINVAL, "dz=%d exceeds %d", dz, IDTX_MAX_DZ);
    std::vector<char> alive(n_cand_total, 1);
    for (int lag = min_lag; lag <= std::min(max_lag, n_past); ++lag)
        alive[target * n_lags + (lag - min_lag)] = 0;
    if (allowed)
        for (int cid = 0; cid < n_cand_total; ++cid) alive[cid] &= allowed[cid];
    for (int t = 0; t < n_selected; ++t) {
        if (selected[t] < 0 || selected[t] >= n_cand_total)
            return fail(IDTX_EINVAL, "selected id %d out of range", selected[t]);
        alive[selected[t]] = 0;
    }
    std::vector<int32_t> ids;
    for (int cid = 0; cid < n_cand_total; ++cid)
        if (alive[cid]) ids.push_back(cid);
    if (ids.empty()) return fail(IDTX_EINVAL, "no candidate left");
    const int n_alive = (int)ids.size();
    const size_t jobs_a = (size_t)n_alive * (1 + s0);
    const size_t jobs_b_max = screened ? (size_t)n_alive * (s->n_surr - s0) : 0;

    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float *ser = series;
    const bool host_series = !device_accessible(series);
    IDTX_TRY(ensure(c, B_IN, host_series ? (size_t)n_proc * T * sizeof(float) : 0));
    IDTX_TRY(begin_call(c, screened ? 2 : 1, st));
    if (host_series) {
        IDTX_CUDA(cudaMemcpyAsync(c->buf[B_IN], series, (size_t)n_proc * T * sizeof(float),
                                  cudaMemcpyHostToDevice, st));
        ser = (const float *)c->buf[B_IN];
    }

    // Sample i is time L + i; the variable (p, lag) at sample i is series[p][L + i - lag].
    auto col = [&](int p, int lag) { return Col{ser + (int64_t)p * T, L - lag}; };
    auto stream_of = [&](int cid, int sidx) {
        return ((uint64_t)step_index << 48) | ((uint64_t)cid << 24) | (uint64_t)sidx;
    };
    // One group of jobs over candidates cand[] (indices into ids), surrogates [s_lo, s_hi);
    // with_orig adds each candidate's estimate before its surrogates.
    auto make_group = [&](Group &g, const std::vector<int> &cand, bool with_orig, int s_lo,
                          int s_hi) {
        g.n = n;
        g.dx = 1;
        g.dy = 1;
        g.dz = dz;
        g.k = s->k;
        g.ycols.push_back(col(target, 0));
        for (int lag = 1; lag <= n_past; ++lag) g.zcols.push_back(col(target, lag));
        for (int t = 0; t < n_selected; ++t)
            g.zcols.push_back(col(selected[t] / n_lags, min_lag + selected[t] % n_lags));
        for (size_t a = 0; a < cand.size(); ++a) {
            const int cid = ids[cand[a]];
            g.xcols.push_back(col(cid / n_lags, min_lag + cid % n_lags));
            if (with_orig) g.jobs.push_back(Job{(int32_t)a, -1});
            for (int sidx = s_lo; sidx < s_hi; ++sidx) {
                g.jobs.push_back(Job{(int32_t)a, (int32_t)g.slot_stream.size()});
                g.slot_stream.push_back(stream_of(cid, sidx));
                g.slot_seed.push_back(s->seed);
            }
        }
        g.plain = s->mode == IDTX_MODE_PLAIN;
    };
    auto upload = [&](std::vector<Group> &gs, std::vector<unsigned char> &arena,
                      size_t cmi_bytes) -> int {
        pack_desc(gs, arena);
        CallBuffers b;
        for (const Group &g : gs) sizes_of(g, b);
        IDTX_TRY(ensure(c, B_DESC, arena.size()));
        IDTX_TRY(ensure(c, B_SH, b.sh));
        IDTX_TRY(ensure(c, B_XI, b.xi));
        IDTX_TRY(ensure(c, B_PERM, b.perm));
        IDTX_TRY(ensure(c, B_PARTIAL, b.partial));
        IDTX_TRY(ensure(c, B_ORDER, b.order));
        IDTX_TRY(ensure(c, B_SORT, b.sort_tmp));
        IDTX_TRY(ensure(c, B_LIST, b.lists));
        IDTX_TRY(ensure(c, B_CMI, cmi_bytes));
        IDTX_CUDA(cudaMemcpyAsync(c->buf[B_DESC], arena.data(), arena.size(),
                                  cudaMemcpyHostToDevice, st));
        return IDTX_OK;
    };

    std::vector<int> all(n_alive);
    for (int a = 0; a < n_alive; ++a) all[a] = a;
    std::vector<Group> ga(1);
    make_group(ga[0], all, true, 0, s0);
    IDTX_TRY(plan(c, ga[0]));
    const size_t cmi_bytes = (jobs_a + jobs_b_max) * sizeof(double);
    IDTX_TRY(ensure(c, B_STEP, sizeof(idtx_step) + (size_t)n_cand_total * sizeof(int32_t) + 64));
    IDTX_TRY(ensure_psi(c, std::max<int64_t>(n, s->k) + 1, st));
    std::vector<unsigned char> arena;
    IDTX_TRY(upload(ga, arena, cmi_bytes));
    double *cmi_a = (double *)c->buf[B_CMI];
    double *cmi_b = cmi_a + jobs_a;
    IDTX_TRY(enqueue_group(c, ga[0], st, cmi_a, nullptr, nullptr, timeout_of(c, s)));

    // ids (and, in screened mode, the keep list) live in the step buffer
    unsigned char *stepbuf = (unsigned char *)c->buf[B_STEP];
    idtx_step *step_d = (idtx_step *)stepbuf;
    int32_t *ids_d = (int32_t *)(stepbuf + align_up(sizeof(idtx_step), 16));
    IDTX_CUDA(cudaMemcpyAsync(ids_d, ids.data(), ids.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st));
    int n_keep = 0;
    std::vector<int32_t> keep;
    if (screened) {
        // Features, predictions and the keep list of the screen.
        const int nc = n_alive;
        const size_t scr_floats = IDTX_SCREEN_NPARAMS + 2 * IDTX_SCREEN_F +
                                  (size_t)nc * IDTX_SCREEN_F + nc + 2 * (size_t)nc + 64;
        IDTX_TRY(ensure(c, B_SCREEN, scr_floats * sizeof(float)));
        IDTX_TRY(ensure(c, B_MLP, mlp_work_floats(nc) * sizeof(float)));
        float *sp = (float *)c->buf[B_SCREEN];
        float *params = sp, *mean = params + IDTX_SCREEN_NPARAMS, *scale = mean + IDTX_SCREEN_F;
        float *feats = scale + IDTX_SCREEN_F;
        int32_t *keep_d = (int32_t *)(feats + (size_t)nc * IDTX_SCREEN_F);
        int32_t *nkeep_d = keep_d + nc;
        IDTX_CUDA(cudaMemcpyAsync(params, c->screen.params, sizeof(c->screen.params),
                                  cudaMemcpyHostToDevice, st));
        IDTX_CUDA(cudaMemcpyAsync(mean, c->screen.feat_mean, sizeof(c->screen.feat_mean),
                                  cudaMemcpyHostToDevice, st));
        IDTX_CUDA(cudaMemcpyAsync(scale, c->screen.feat_scale, sizeof(c->screen.feat_scale),
                                  cudaMemcpyHostToDevice, st));
        k_screen_features<<<(nc + 127) / 128, 128, 0, st>>>(
            cmi_a, nc, s0, (float)std::log((double)n), 1, 1, dz, s->k,
            (float)std::log((double)s->n_surr), feats);
        IDTX_CUDA(cudaGetLastError());
        MlpWork w;
        mlp_work_carve((float *)c->buf[B_MLP], nc, &w);
        IDTX_CUDA(mlp_round(params, w, st));
        IDTX_CUDA(mlp_forward(params, w, feats, nullptr, 0, nc, mean, scale, st));
        k_screen_keep<<<1, 1, 0, st>>>(cmi_a, nc, s0, w.y, c->screen.delta, keep_d, nkeep_d);
        IDTX_CUDA(cudaGetLastError());
        c->stats.kernel_launches += 7;
        keep.resize(nc + 1);
        IDTX_CUDA(cudaMemcpyAsync(keep.data(), keep_d, (size_t)(nc + 1) * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st));
        IDTX_CUDA(cudaStreamSynchronize(st));
        n_keep = keep[nc];
    }
    // chunks of the remaining surrogate indices run for the kept candidates:
    // (first index, count, offset of the block [n_keep][count] in cmi_b)
    struct Chunk {
        int lo, cnt;
        size_t off;
    };
    std::vector<Chunk> chunks;
    if (!screened) {
        k_gate<<<1, 256, 0, st>>>(cmi_a, n_alive, s0, cmi_b, n_keep, s->n_surr, ids_d, s->alpha,
                                  step_d);
        IDTX_CUDA(cudaGetLastError());
        c->stats.kernel_launches += 1;
    } else {
        // Count over the cheap surrogates, then chunk after chunk of the rest
        // until the count decides "not significant" or all indices are done.
        int *count_d = (int *)((unsigned char *)ids_d + align_up((size_t)n_cand_total * 4, 16));
        k_gate_begin<<<1, 256, 0, st>>>(cmi_a, n_alive, s0, ids_d, step_d, count_d);
        IDTX_CUDA(cudaGetLastError());
        c->stats.kernel_launches += 1;
        int decide = 0;  // smallest count c with c / n_surr >= alpha
        while ((double)decide / (double)s->n_surr < s->alpha) ++decide;
        int count = 0;
        IDTX_CUDA(cudaMemcpyAsync(&count, count_d, sizeof(int), cudaMemcpyDeviceToHost, st));
        IDTX_CUDA(cudaStreamSynchronize(st));
        int lo = s0, width = 16;
        size_t off = 0;
        while (n_keep > 0 && lo < s->n_surr && count < decide) {
            const int hi = std::min(s->n_surr, lo + width);
            std::vector<int> kc(keep.begin(), keep.begin() + n_keep);
            std::vector<Group> gb(1);
            make_group(gb[0], kc, false, lo, hi);
            gb[0].work_slot = 1;
            IDTX_TRY(plan(c, gb[0]));
            std::vector<unsigned char> arena_b;
            IDTX_TRY(upload(gb, arena_b, cmi_bytes));
            IDTX_TRY(enqueue_group(c, gb[0], st, cmi_b + off, nullptr, nullptr, timeout_of(c, s)));
            k_gate_chunk<<<1, 256, 0, st>>>(cmi_b + off, n_keep, hi - lo, step_d, count_d);
            IDTX_CUDA(cudaGetLastError());
            c->stats.kernel_launches += 1;
            chunks.push_back(Chunk{lo, hi - lo, off});
            off += (size_t)n_keep * (hi - lo);
            IDTX_CUDA(cudaMemcpyAsync(&count, count_d, sizeof(int), cudaMemcpyDeviceToHost, st));
            IDTX_CUDA(cudaStreamSynchronize(st));
            lo = hi;
            width *= 2;
        }
        // Without kept candidates no index past s0 can add to the count, so the
        // count is final; otherwise indices from `lo` on were not evaluated.
        const int surr_done = n_keep == 0 ? s->n_surr : lo;
        k_gate_end<<<1, 1, 0, st>>>(step_d, count_d, s->n_surr, surr_done,
                                    chunks.empty() ? 0 : n_keep, s->alpha);
        IDTX_CUDA(cudaGetLastError());
        c->stats.kernel_launches += 1;
    }
    IDTX_CUDA(cudaMemcpyAsync(result, step_d, sizeof(idtx_step),
                              device_accessible(result) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost,
                              st));
    if (est_out) {
        // Rows of est_out are [1 + n_surr] per candidate id; columns the kernel
        // did not compute (screened mode, skipped candidates) are left untouched.
        const bool dev = device_accessible(est_out);
        const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const size_t row = (size_t)(1 + s->n_surr) * sizeof(double);
        for (int a = 0; a < n_alive; ++a)
            IDTX_CUDA(cudaMemcpyAsync((unsigned char *)est_out + (size_t)ids[a] * row,
                                      cmi_a + (size_t)a * (1 + s0), (size_t)(1 + s0) * 8, kind,
                                      st));
        for (const Chunk &ch : chunks)
            for (int t = 0; t < n_keep; ++t)
                IDTX_CUDA(cudaMemcpyAsync((unsigned char *)est_out + (size_t)ids[keep[t]] * row +
                                              (size_t)(1 + ch.lo) * 8,
                                          cmi_b + ch.off + (size_t)t * ch.cnt, (size_t)ch.cnt * 8,
                                          kind, st));
    }
    return finish_call(c, st);
}

}  // namespace

extern "C" {

int idtx_mte_step(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target, int n_past,
                  int min_lag, int max_lag, const int32_t *selected, int n_selected,
                  int step_index, const idtx_settings *s, idtx_step *result, double *est_out,
                  void *stream)
{
    return mte_step_impl(c, series, n_proc, T, target, n_past, min_lag, max_lag, selected,
                         n_selected, step_index, s, result, est_out, nullptr, stream);
}

// ------------------------------------------------------------------ learned screen
namespace {

constexpr int kScreenP = IDTX_SCREEN_NPARAMS, kScreenF = IDTX_SCREEN_F;

int check_screen(const idtx_screen *sc)
{
    if (!sc) return fail(IDTX_EINVAL, "screen is NULL");
    for (int i = 0; i < kScreenP; ++i)
        if (!std::isfinite(sc->params[i])) return fail(IDTX_EINVAL, "non-finite screen parameter");
    for (int i = 0; i < kScreenF; ++i)
        if (!std::isfinite(sc->feat_mean[i]) || !std::isfinite(sc->feat_scale[i]))
            return fail(IDTX_EINVAL, "non-finite screen normalisation");
    if (!std::isfinite(sc->delta)) return fail(IDTX_EINVAL, "non-finite screen delta");
    return IDTX_OK;
}

// Device copies of the screen's parameters and normalisation at the start of
// B_SCREEN, followed by `extra` floats of room.
int upload_screen(idtx_ctx *c, const idtx_screen *sc, size_t extra, cudaStream_t st,
                  float **params, float **mean, float **scale, float **rest)
{
    IDTX_TRY(ensure(c, B_SCREEN, (kScreenP + 2 * kScreenF + extra + 64) * sizeof(float)));
    float *sp = (float *)c->buf[B_SCREEN];
    *params = sp;
    *mean = sp + kScreenP;
    *scale = *mean + kScreenF;
    *rest = *scale + kScreenF;
    IDTX_CUDA(cudaMemcpyAsync(*params, sc->params, sizeof(sc->params), cudaMemcpyHostToDevice, st));
    IDTX_CUDA(cudaMemcpyAsync(*mean, sc->feat_mean, sizeof(sc->feat_mean), cudaMemcpyHostToDevice,
                              st));
    IDTX_CUDA(cudaMemcpyAsync(*scale, sc->feat_scale, sizeof(sc->feat_scale),
                              cudaMemcpyHostToDevice, st));
    return IDTX_OK;
}

// Device pointer to n*width floats of `src` (copied into dst when src is host memory).
int device_floats(const float *src, size_t count, float *dst, cudaStream_t st, const float **out)
{
    if (device_accessible(src)) {
        *out = src;
        return IDTX_OK;
    }
    IDTX_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(float), cudaMemcpyHostToDevice, st));
    *out = dst;
    return IDTX_OK;
}

}  // namespace

extern "C" int idtx_screen_set(idtx_ctx *c, const idtx_screen *sc)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    IDTX_TRY(check_screen(sc));
    c->screen = *sc;
    c->has_screen = true;
    return IDTX_OK;
}

// The screen file (idtx.h): "IDTXSCR1", version, F, H, parameter count,
// s0, delta, then params, feat_mean, feat_scale; little-endian.
extern "C" int idtx_screen_load(idtx_ctx *c, const char *path)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!path) return fail(IDTX_EINVAL, "path is NULL");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(IDTX_EINVAL, "cannot open screen file %s", path);
    struct Header {
        char magic[8];
        uint32_t version, nf, nh, np;
        int32_t s0;
        float delta;
    } h;
    static_assert(sizeof(Header) == 32, "screen file header is 32 bytes");
    idtx_screen sc;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1;
    if (ok) ok = std::memcmp(h.magic, "IDTXSCR1", 8) == 0 && h.version == 1 &&
                 h.nf == kScreenF && h.nh == IDTX_SCREEN_H && h.np == (uint32_t)kScreenP;
    if (ok) ok = std::fread(sc.params, sizeof(float), kScreenP, f) == (size_t)kScreenP &&
                 std::fread(sc.feat_mean, sizeof(float), kScreenF, f) == (size_t)kScreenF &&
                 std::fread(sc.feat_scale, sizeof(float), kScreenF, f) == (size_t)kScreenF;
    if (ok) ok = std::fgetc(f) == EOF;  // nothing after the arrays
    std::fclose(f);
    if (!ok) return fail(IDTX_EINVAL, "%s is not a screen file of this library's layout", path);
    sc.s0 = h.s0;
    sc.delta = h.delta;
    if (sc.s0 < 1) return fail(IDTX_EINVAL, "screen file s0=%d", sc.s0);
    return idtx_screen_set(c, &sc);
}

extern "C" int idtx_screen_features(idtx_ctx *c, const double *est, int n_cand, int s0,
                                    int64_t n, int dx, int dy, int dz, int k, int n_surr,
                                    float *feats_out, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!est || !feats_out) return fail(IDTX_EINVAL, "est or feats_out is NULL");
    if (n_cand < 0 || s0 < 1 || n < 2 || n_surr < 1)
        return fail(IDTX_EINVAL, "bad n_cand=%d s0=%d n=%lld n_surr=%d", n_cand, s0,
                    (long long)n, n_surr);
    if (n_cand == 0) return IDTX_OK;
    DeviceGuard dg(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t est_bytes = (size_t)n_cand * (1 + s0) * sizeof(double);
    const size_t feat_bytes = (size_t)n_cand * kScreenF * sizeof(float);
    IDTX_TRY(ensure(c, B_TRAIN, align_up(est_bytes, 256) + feat_bytes));
    const double *est_d = est;
    if (!device_accessible(est)) {
        IDTX_CUDA(cudaMemcpyAsync(c->buf[B_TRAIN], est, est_bytes, cudaMemcpyHostToDevice, st));
        est_d = (const double *)c->buf[B_TRAIN];
    }
    const bool dev_out = device_accessible(feats_out);
    float *f_d = dev_out ? feats_out
                         : (float *)((unsigned char *)c->buf[B_TRAIN] + align_up(est_bytes, 256));
    k_screen_features<<<(n_cand + 127) / 128, 128, 0, st>>>(
        est_d, n_cand, s0, (float)std::log((double)n), dx, dy, dz, k,
        (float)std::log((double)n_surr), f_d);
    IDTX_CUDA(cudaGetLastError());
    c->stats.kernel_launches += 1;
    if (!dev_out)
        IDTX_CUDA(cudaMemcpyAsync(feats_out, f_d, feat_bytes, cudaMemcpyDeviceToHost, st));
    IDTX_CUDA(cudaStreamSynchronize(st));
    return IDTX_OK;
}

extern "C" int idtx_screen_predict(idtx_ctx *c, const idtx_screen *sc, const float *feats, int n,
                                   float *out, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!feats || !out || n < 1) return fail(IDTX_EINVAL, "bad features or output");
    IDTX_TRY(check_screen(sc));
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    IDTX_TRY(begin_call(c, 0, st));
    float *params, *mean, *scale, *rest;
    IDTX_TRY(upload_screen(c, sc, (size_t)n * kScreenF, st, &params, &mean, &scale, &rest));
    IDTX_TRY(ensure(c, B_MLP, mlp_work_floats(n) * sizeof(float)));
    const float *fd;
    IDTX_TRY(device_floats(feats, (size_t)n * kScreenF, rest, st, &fd));
    MlpWork w;
    mlp_work_carve((float *)c->buf[B_MLP], n, &w);
    IDTX_CUDA(mlp_round(params, w, st));
    IDTX_CUDA(mlp_forward(params, w, fd, nullptr, 0, n, mean, scale, st));
    c->stats.kernel_launches += 5;
    IDTX_CUDA(cudaMemcpyAsync(out, w.y, (size_t)n * sizeof(float),
                              device_accessible(out) ? cudaMemcpyDeviceToDevice
                                                     : cudaMemcpyDeviceToHost,
                              st));
    return finish_call(c, st);
}

extern "C" int idtx_screen_loss_grad(idtx_ctx *c, const idtx_screen *sc, const float *feats,
                                     const float *targets, int n, float quantile, double *loss,
                                     float *grad, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!feats || !targets || !loss || !grad || n < 1)
        return fail(IDTX_EINVAL, "bad features, targets or outputs");
    if (!(quantile >= 0.0f && quantile < 1.0f)) return fail(IDTX_EINVAL, "quantile not in [0,1)");
    IDTX_TRY(check_screen(sc));
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    IDTX_TRY(begin_call(c, 0, st));
    float *params, *mean, *scale, *rest;
    IDTX_TRY(upload_screen(c, sc, (size_t)n * (kScreenF + 1) + 16, st, &params, &mean, &scale,
                           &rest));
    IDTX_TRY(ensure(c, B_MLP, mlp_work_floats(n) * sizeof(float) + 64));
    const float *fd, *td;
    IDTX_TRY(device_floats(feats, (size_t)n * kScreenF, rest, st, &fd));
    IDTX_TRY(device_floats(targets, (size_t)n, rest + (size_t)n * kScreenF, st, &td));
    double *loss_d = (double *)((float *)c->buf[B_MLP] + mlp_work_floats(n) + 2);
    loss_d = (double *)(((uintptr_t)loss_d + 7) & ~(uintptr_t)7);
    IDTX_CUDA(cudaMemsetAsync(loss_d, 0, sizeof(double), st));
    MlpWork w;
    mlp_work_carve((float *)c->buf[B_MLP], n, &w);
    IDTX_CUDA(mlp_round(params, w, st));
    IDTX_CUDA(mlp_forward(params, w, fd, nullptr, 0, n, mean, scale, st));
    IDTX_CUDA(mlp_loss(w, td, nullptr, 0, n, (quantile > 0.0f ? 1.0f : 2.0f) / (float)n, quantile,
                       true, loss_d, st));
    IDTX_CUDA(mlp_backward(w, n, false, st));
    c->stats.kernel_launches += 11;
    double lsum = 0.0;
    IDTX_CUDA(cudaMemcpyAsync(&lsum, loss_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    IDTX_CUDA(cudaMemcpyAsync(grad, w.grad, (size_t)kScreenP * sizeof(float),
                              cudaMemcpyDeviceToHost, st));
    const int rc = finish_call(c, st);
    *loss = lsum / (double)n;
    return rc;
}

extern "C" int idtx_screen_train(idtx_ctx *c, idtx_screen *sc, const float *feats,
                                 const float *targets, int n, int epochs, int batch, float lr,
                                 float quantile, uint64_t seed, double *final_loss, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!feats || !targets || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.0f))
        return fail(IDTX_EINVAL, "bad training arguments");
    if (!(quantile >= 0.0f && quantile < 1.0f)) return fail(IDTX_EINVAL, "quantile not in [0,1)");
    IDTX_TRY(check_screen(sc));
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    IDTX_TRY(begin_call(c, 0, st));
    batch = std::min(batch, n);
    float *params, *mean, *scale, *rest;
    IDTX_TRY(upload_screen(c, sc, 0, st, &params, &mean, &scale, &rest));
    // training area: features, targets, order, Adam moments, loss accumulator
    const size_t tr_floats = (size_t)n * (kScreenF + 1) + (size_t)n + 2 * (size_t)kScreenP + 16;
    IDTX_TRY(ensure(c, B_TRAIN, tr_floats * sizeof(float)));
    const int wb = std::max(batch, std::min(n, 4096));
    IDTX_TRY(ensure(c, B_MLP, mlp_work_floats(wb) * sizeof(float)));
    float *tr = (float *)c->buf[B_TRAIN];
    float *fbuf = tr, *tbuf = fbuf + (size_t)n * kScreenF;
    int32_t *order = (int32_t *)(tbuf + n);
    float *m = (float *)(order + n), *v = m + kScreenP;
    double *loss_d = (double *)(((uintptr_t)(v + kScreenP) + 7) & ~(uintptr_t)7);
    const float *fd, *td;
    IDTX_TRY(device_floats(feats, (size_t)n * kScreenF, fbuf, st, &fd));
    IDTX_TRY(device_floats(targets, (size_t)n, tbuf, st, &td));
    IDTX_CUDA(cudaMemsetAsync(m, 0, 2 * (size_t)kScreenP * sizeof(float), st));
    IDTX_TRY(ensure(c, B_DESC, 64));
    uint64_t *rng = (uint64_t *)c->buf[B_DESC];  // [0] stream, [1] seed of the shuffle
    MlpWork w;
    mlp_work_carve((float *)c->buf[B_MLP], wb, &w);
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        const uint64_t rs[2] = {(uint64_t)ep, seed};
        IDTX_CUDA(cudaMemcpyAsync(rng, rs, sizeof(rs), cudaMemcpyHostToDevice, st));
        k_fisher_yates<<<1, 32, 0, st>>>(order, rng, rng + 1, n);
        IDTX_CUDA(cudaGetLastError());
        for (int start = 0; start < n; start += batch) {
            const int bsz = std::min(batch, n - start);
            IDTX_CUDA(mlp_round(params, w, st));
            IDTX_CUDA(mlp_forward(params, w, fd, order, start, bsz, mean, scale, st));
            IDTX_CUDA(mlp_loss(w, td, order, start, bsz,
                               (quantile > 0.0f ? 1.0f : 2.0f) / (float)bsz, quantile, true,
                               loss_d, st));
            IDTX_CUDA(mlp_backward(w, bsz, false, st));
            IDTX_CUDA(mlp_adam(params, w.grad, m, v, ++step, lr, st));
            c->stats.kernel_launches += 12;
        }
        IDTX_CUDA(cudaStreamSynchronize(st));  // keep the host copy of rs alive
    }
    // full-data loss of the trained parameters
    IDTX_CUDA(cudaMemsetAsync(loss_d, 0, sizeof(double), st));
    IDTX_CUDA(mlp_round(params, w, st));
    for (int start = 0; start < n; start += wb) {
        const int bsz = std::min(wb, n - start);
        IDTX_CUDA(mlp_forward(params, w, fd, nullptr, start, bsz, mean, scale, st));
        IDTX_CUDA(mlp_loss(w, td, nullptr, start, bsz, 0.0f, quantile, false, loss_d, st));
    }
    double lsum = 0.0;
    IDTX_CUDA(cudaMemcpyAsync(&lsum, loss_d, sizeof(double), cudaMemcpyDeviceToHost, st));
    IDTX_CUDA(cudaMemcpyAsync(sc->params, params, sizeof(sc->params), cudaMemcpyDeviceToHost, st));
    const int rc = finish_call(c, st);
    if (final_loss) *final_loss = lsum / (double)n;
    return rc;
}

int idtx_mte_select_target(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target,
                           int n_past, int min_lag, int max_lag, const idtx_settings *s,
                           int max_parents, int32_t *parents_out, int *n_parents,
                           idtx_step *steps_out, int *n_steps, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (max_parents < 0 || !n_parents || !n_steps || !steps_out ||
        (max_parents > 0 && !parents_out))
        return fail(IDTX_EINVAL, "bad outputs");
    if (!series) return fail(IDTX_EINVAL, "series is NULL");
    *n_parents = 0;
    *n_steps = 0;
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    // Keep a device copy of host series for all steps.
    const float *ser = series;
    std::vector<float> none;
    void *dev_series = nullptr;
    if (!device_accessible(series)) {
        IDTX_CUDA(cudaMalloc(&dev_series, (size_t)n_proc * T * sizeof(float)));
        cudaError_t e = cudaMemcpyAsync(dev_series, series, (size_t)n_proc * T * sizeof(float),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(dev_series);
            return fail(IDTX_ECUDA, "series copy failed: %s", cudaGetErrorString(e));
        }
        ser = (const float *)dev_series;
    }
    const int n_lags = max_lag - min_lag + 1;
    const int n_cand_total = n_proc * n_lags;
    int n_left = n_cand_total - std::max(0, std::min(max_lag, n_past) - min_lag + 1);
    std::vector<int32_t> sel;
    int rc = IDTX_OK;
    for (int step = 0; step <= max_parents; ++step) {
        if (n_left <= 0 || step == max_parents) break;
        idtx_step r;
        rc = idtx_mte_step(c, ser, n_proc, T, target, n_past, min_lag, max_lag, sel.data(),
                           (int)sel.size(), step, s, &r, nullptr, stream);
        if (rc != IDTX_OK) break;
        steps_out[(*n_steps)++] = r;
        if (!r.significant) break;
        sel.push_back(r.cand);
        parents_out[(*n_parents)++] = r.cand;
        --n_left;
    }
    if (dev_series) {
        cudaStreamSynchronize(st);
        cudaFree(dev_series);
    }
    return rc;
}

namespace {

// Greedy loop over the candidates `allowed` marks (nullable: all), Z
// starting from init[0..n_init) (candidate ids), step s with step index
// step_base + s.  The series is copied to the device once if needed.
int greedy_loop(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target, int min_lag,
                int max_lag, const int32_t *init, int n_init, const char *allowed,
                int step_base, const idtx_settings *s, int max_sel, int32_t *sel_out,
                int *n_sel, idtx_step *steps_out, int *n_steps, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const float *ser = series;
    void *dev_series = nullptr;
    if (!device_accessible(series)) {
        IDTX_CUDA(cudaMalloc(&dev_series, (size_t)n_proc * T * sizeof(float)));
        cudaError_t e = cudaMemcpyAsync(dev_series, series, (size_t)n_proc * T * sizeof(float),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            cudaFree(dev_series);
            return fail(IDTX_ECUDA, "series copy failed: %s", cudaGetErrorString(e));
        }
        ser = (const float *)dev_series;
    }
    const int n_all = n_proc * (max_lag - min_lag + 1);
    std::vector<int32_t> zsel(init, init + n_init);
    int n_left = 0;
    for (int cid = 0; cid < n_all; ++cid)
        n_left += (!allowed || allowed[cid]) &&
                  std::find(zsel.begin(), zsel.end(), cid) == zsel.end();
    int rc = IDTX_OK;
    for (int step = 0; step < max_sel && n_left > 0; ++step) {
        idtx_step r;
        rc = mte_step_impl(c, ser, n_proc, T, target, 0, min_lag, max_lag, zsel.data(),
                           (int)zsel.size(), step_base + step, s, &r, nullptr, allowed, stream);
        if (rc != IDTX_OK) break;
        steps_out[(*n_steps)++] = r;
        if (!r.significant) break;
        zsel.push_back(r.cand);
        sel_out[(*n_sel)++] = r.cand;
        --n_left;
    }
    if (dev_series) {
        cudaStreamSynchronize(st);
        cudaFree(dev_series);
    }
    return rc;
}

}  // namespace

int idtx_mte_select_past(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target,
                         int min_lag, int max_lag, const idtx_settings *s, int max_past,
                         int32_t *past_out, int *n_past, idtx_step *steps_out, int *n_steps,
                         void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!series || max_past < 0 || !n_past || !n_steps || !steps_out ||
        (max_past > 0 && !past_out))
        return fail(IDTX_EINVAL, "bad arguments");
    if (n_proc < 1 || target < 0 || target >= n_proc || min_lag < 1 || max_lag < min_lag)
        return fail(IDTX_EINVAL, "bad target or lags");
    *n_past = 0;
    *n_steps = 0;
    DeviceGuard guard(c->device);
    const int n_lags = max_lag - min_lag + 1;
    std::vector<char> allowed((size_t)n_proc * n_lags, 0);
    for (int l = 0; l < n_lags; ++l) allowed[(size_t)target * n_lags + l] = 1;
    return greedy_loop(c, series, n_proc, T, target, min_lag, max_lag, nullptr, 0, allowed.data(),
                       0xD000, s, max_past, past_out, n_past, steps_out, n_steps, stream);
}

int idtx_mte_select_sources(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target,
                            const int32_t *past, int n_past_ids, int min_lag, int max_lag,
                            const idtx_settings *s, int max_parents, int32_t *parents_out,
                            int *n_parents, idtx_step *steps_out, int *n_steps, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!series || max_parents < 0 || !n_parents || !n_steps || !steps_out ||
        (max_parents > 0 && !parents_out) || n_past_ids < 0 || (n_past_ids > 0 && !past))
        return fail(IDTX_EINVAL, "bad arguments");
    if (n_proc < 1 || target < 0 || target >= n_proc || min_lag < 1 || max_lag < min_lag)
        return fail(IDTX_EINVAL, "bad target or lags");
    *n_parents = 0;
    *n_steps = 0;
    DeviceGuard guard(c->device);
    return greedy_loop(c, series, n_proc, T, target, min_lag, max_lag, past, n_past_ids, nullptr,
                       0, s, max_parents, parents_out, n_parents, steps_out, n_steps, stream);
}


// ------------------------------------------------------------------ tests after selection
namespace {

constexpr uint64_t kTagPrune = 0x9000, kTagOmnibus = 0xA000, kTagSeqmax = 0xB000;

// Common checks of a post-selection call; puts the series on the device
// (host series are copied into B_IN) and sets the sample range.
int post_begin(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target, int n_past,
               int min_lag, int max_lag, const int32_t *parents, int m, const idtx_settings *s,
               int dx_max_needed, int dz_needed, cudaStream_t st, const float **ser, int64_t *L)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!series || !s || !parents) return fail(IDTX_EINVAL, "NULL series/settings/parents");
    if (n_proc < 1 || target < 0 || target >= n_proc || n_past < 0 || min_lag < 1 ||
        max_lag < min_lag || m < 1)
        return fail(IDTX_EINVAL, "bad arguments");
    const int n_lags = max_lag - min_lag + 1;
    for (int i = 0; i < m; ++i) {
        const int cid = parents[i];
        if (cid < 0 || cid >= n_proc * n_lags)
            return fail(IDTX_EINVAL, "parent id %d out of range", cid);
        if (cid / n_lags == target && min_lag + cid % n_lags <= n_past)
            return fail(IDTX_EINVAL, "parent id %d is a target-past variable", cid);
        for (int j = 0; j < i; ++j)
            if (parents[j] == cid) return fail(IDTX_EINVAL, "parent id %d repeated", cid);
    }
    *L = std::max(max_lag, n_past);
    if (T <= *L || T - *L > IDTX_MAX_N) return fail(IDTX_EINVAL, "bad T for the lags");
    if (s->k < 1 || s->k > IDTX_MAX_K || s->k > T - *L - 1) return fail(IDTX_EINVAL, "bad k");
    if (s->n_surr < 1) return fail(IDTX_EINVAL, "n_surr must be >= 1");
    if (!(s->alpha > 0.0 && s->alpha < 1.0)) return fail(IDTX_EINVAL, "alpha out of (0,1)");
    if (s->mode != IDTX_MODE_BATCHED) return fail(IDTX_EINVAL, "only IDTX_MODE_BATCHED");
    if (dx_max_needed > IDTX_MAX_DX || dz_needed > IDTX_MAX_DZ)
        return fail(IDTX_EINVAL, "parent set too large (dx=%d dz=%d)", dx_max_needed, dz_needed);
    *ser = series;
    if (!device_accessible(series)) {
        IDTX_TRY(ensure(c, B_IN, (size_t)n_proc * T * sizeof(float)));
        IDTX_CUDA(cudaMemcpyAsync(c->buf[B_IN], series, (size_t)n_proc * T * sizeof(float),
                                  cudaMemcpyHostToDevice, st));
        *ser = (const float *)c->buf[B_IN];
    }
    return ensure_psi(c, std::max<int64_t>(T - *L, s->k) + 1, st);
}

// Run fully described groups as one batch; estimates land in B_CMI at each
// group's off_cmi.
int run_groups(idtx_ctx *c, std::vector<Group> &gs, cudaStream_t st, long long tmo, size_t n_est)
{
    std::vector<unsigned char> arena;
    pack_desc(gs, arena);
    IDTX_TRY(ensure(c, B_DESC, arena.size()));
    IDTX_CUDA(cudaMemcpyAsync(c->buf[B_DESC], arena.data(), arena.size(), cudaMemcpyHostToDevice,
                              st));
    if (std::any_of(gs.begin(), gs.end(), [](const Group &g) { return g.tune; }))
        IDTX_TRY(resolve_tuning(c, gs, st, tmo));
    IDTX_TRY(ensure(c, B_CMI, n_est * sizeof(double)));
    BatchPlan bp;
    IDTX_TRY(batch_plan(c, gs, st, tmo, bp));
    return batch_enqueue(c, gs, bp, st, (double *)c->buf[B_CMI], tmo);
}

// Leave-one-out estimates of a parent list: group i estimates
// I(X_{c_i}; Y | target past, X_{c_j} for j != i) and its surrogates
// (streams tag<<48 | c_i<<24 | s) into B_CMI row i.
int enqueue_loo(idtx_ctx *c, const float *ser, int64_t T, int64_t L, int target, int n_past,
                int min_lag, int max_lag, const std::vector<int32_t> &par,
                const idtx_settings *s, uint64_t tag, cudaStream_t st)
{
    const int n_lags = max_lag - min_lag + 1, m = (int)par.size();
    auto col = [&](int cid) {
        return Col{ser + (int64_t)(cid / n_lags) * T, L - (min_lag + cid % n_lags)};
    };
    std::vector<Group> gs(m);
    size_t off = 0;
    for (int i = 0; i < m; ++i) {
        Group &g = gs[i];
        g.n = T - L;
        g.dx = 1;
        g.dy = 1;
        g.dz = n_past + m - 1;
        g.k = s->k;
        g.ycols.push_back(Col{ser + (int64_t)target * T, L});
        for (int lag = 1; lag <= n_past; ++lag) g.zcols.push_back(Col{ser + (int64_t)target * T, L - lag});
        for (int j = 0; j < m; ++j)
            if (j != i) g.zcols.push_back(col(par[j]));
        g.xcols.push_back(col(par[i]));
        g.jobs.push_back(Job{0, -1});
        for (int sidx = 0; sidx < s->n_surr; ++sidx) {
            g.jobs.push_back(Job{0, sidx});
            g.slot_stream.push_back((tag << 48) | ((uint64_t)par[i] << 24) | (uint64_t)sidx);
            g.slot_seed.push_back(s->seed);
        }
        IDTX_TRY(plan(c, g));
        g.work_slot = i;
        g.off_cmi = off;
        off += 1 + (size_t)s->n_surr;
    }
    return run_groups(c, gs, st, timeout_of(c, s), off);
}

}  // namespace

int idtx_mte_prune(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target, int n_past,
                   int min_lag, int max_lag, const int32_t *parents, int n_parents,
                   const idtx_settings *s, int32_t *kept_out, int *n_kept, idtx_step *rounds_out,
                   int *n_rounds, void *stream)
{
    if (!kept_out || !n_kept) return fail(IDTX_EINVAL, "kept_out / n_kept is NULL");
    *n_kept = 0;
    if (n_rounds) *n_rounds = 0;
    if (c == nullptr) return fail(IDTX_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float *ser = nullptr;
    int64_t L = 0;
    IDTX_TRY(post_begin(c, series, n_proc, T, target, n_past, min_lag, max_lag, parents, n_parents,
                        s, 1, n_past + n_parents - 1, st, &ser, &L));
    std::vector<int32_t> cur(parents, parents + n_parents);
    for (int round = 0; !cur.empty(); ++round) {
        const int m = (int)cur.size();
        IDTX_TRY(begin_call(c, m, st));
        IDTX_TRY(enqueue_loo(c, ser, T, L, target, n_past, min_lag, max_lag, cur, s,
                             kTagPrune + (uint64_t)round, st));
        IDTX_TRY(ensure(c, B_STEP, align_up(sizeof(idtx_step), 16) + (size_t)m * 4 + 64));
        idtx_step *step_d = (idtx_step *)c->buf[B_STEP];
        int32_t *ids_d = (int32_t *)((unsigned char *)c->buf[B_STEP] + align_up(sizeof(idtx_step), 16));
        IDTX_CUDA(cudaMemcpyAsync(ids_d, cur.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st));
        k_min_stat<<<1, 256, 0, st>>>((const double *)c->buf[B_CMI], m, s->n_surr, ids_d, s->alpha,
                                      step_d);
        IDTX_CUDA(cudaGetLastError());
        c->stats.kernel_launches += 1;
        idtx_step r;
        IDTX_CUDA(cudaMemcpyAsync(&r, step_d, sizeof(idtx_step), cudaMemcpyDeviceToHost, st));
        IDTX_TRY(finish_call(c, st));
        if (rounds_out) rounds_out[round] = r;
        if (n_rounds) *n_rounds = round + 1;
        if (r.significant) break;
        cur.erase(std::find(cur.begin(), cur.end(), r.cand));
    }
    for (size_t i = 0; i < cur.size(); ++i) kept_out[i] = cur[i];
    *n_kept = (int)cur.size();
    return IDTX_OK;
}

int idtx_mte_omnibus(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target,
                     int n_past, int min_lag, int max_lag, const int32_t *parents, int n_parents,
                     const idtx_settings *s, idtx_step *result, void *stream)
{
    if (!result) return fail(IDTX_EINVAL, "result is NULL");
    if (c == nullptr) return fail(IDTX_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float *ser = nullptr;
    int64_t L = 0;
    IDTX_TRY(post_begin(c, series, n_proc, T, target, n_past, min_lag, max_lag, parents, n_parents,
                        s, n_parents, n_past, st, &ser, &L));
    const int n_lags = max_lag - min_lag + 1;
    IDTX_TRY(begin_call(c, 1, st));
    std::vector<Group> gs(1);
    Group &g = gs[0];
    g.n = T - L;
    g.dx = n_parents;
    g.dy = 1;
    g.dz = n_past;
    g.k = s->k;
    g.ycols.push_back(Col{ser + (int64_t)target * T, L});
    for (int lag = 1; lag <= n_past; ++lag) g.zcols.push_back(Col{ser + (int64_t)target * T, L - lag});
    for (int i = 0; i < n_parents; ++i)
        g.xcols.push_back(Col{ser + (int64_t)(parents[i] / n_lags) * T,
                              L - (min_lag + parents[i] % n_lags)});
    g.jobs.push_back(Job{0, -1});
    for (int sidx = 0; sidx < s->n_surr; ++sidx) {
        g.jobs.push_back(Job{0, sidx});
        g.slot_stream.push_back((kTagOmnibus << 48) | ((uint64_t)0xFFFFFF << 24) | (uint64_t)sidx);
        g.slot_seed.push_back(s->seed);
    }
    IDTX_TRY(plan(c, g));
    IDTX_TRY(run_groups(c, gs, st, timeout_of(c, s), 1 + (size_t)s->n_surr));
    IDTX_TRY(ensure(c, B_STEP, sizeof(idtx_step) + 64));
    idtx_step *step_d = (idtx_step *)c->buf[B_STEP];
    k_single_stat<<<1, 256, 0, st>>>((const double *)c->buf[B_CMI], s->n_surr, s->alpha, step_d);
    IDTX_CUDA(cudaGetLastError());
    c->stats.kernel_launches += 1;
    IDTX_CUDA(cudaMemcpyAsync(result, step_d, sizeof(idtx_step),
                              device_accessible(result) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyDeviceToHost,
                              st));
    return finish_call(c, st);
}

int idtx_mte_seqmax(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target,
                    int n_past, int min_lag, int max_lag, const int32_t *parents, int n_parents,
                    const idtx_settings *s, double *stat_out, double *pval_out,
                    int32_t *significant_out, void *stream)
{
    if (!stat_out || !pval_out || !significant_out) return fail(IDTX_EINVAL, "NULL output");
    if (c == nullptr) return fail(IDTX_EINVAL, "ctx is NULL");
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float *ser = nullptr;
    int64_t L = 0;
    IDTX_TRY(post_begin(c, series, n_proc, T, target, n_past, min_lag, max_lag, parents, n_parents,
                        s, 1, n_past + n_parents - 1, st, &ser, &L));
    const int m = n_parents;
    std::vector<int32_t> par(parents, parents + m);
    IDTX_TRY(begin_call(c, m, st));
    IDTX_TRY(enqueue_loo(c, ser, T, L, target, n_past, min_lag, max_lag, par, s, kTagSeqmax, st));
    const size_t o_stats = 256, o_pvals = o_stats + align_up((size_t)m * 8, 16),
                 o_sig = o_pvals + align_up((size_t)m * 8, 16);
    IDTX_TRY(ensure(c, B_STEP, o_sig + align_up((size_t)m * 4, 16)));
    unsigned char *b = (unsigned char *)c->buf[B_STEP];
    int32_t *rank_d = (int32_t *)b;  // m <= IDTX_MAX_DZ + 1 ints fit in the first 256 bytes
    double *stats_d = (double *)(b + o_stats), *pvals_d = (double *)(b + o_pvals);
    int32_t *sig_d = (int32_t *)(b + o_sig);
    k_seqmax_stat<<<1, 256, 0, st>>>((const double *)c->buf[B_CMI], m, s->n_surr, s->alpha, rank_d,
                                     stats_d, pvals_d, sig_d);
    IDTX_CUDA(cudaGetLastError());
    c->stats.kernel_launches += 1;
    auto out = [&](void *dst, const void *src, size_t bytes) -> int {
        IDTX_CUDA(cudaMemcpyAsync(dst, src, bytes,
                                  device_accessible(dst) ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost,
                                  st));
        return IDTX_OK;
    };
    IDTX_TRY(out(stat_out, stats_d, (size_t)m * 8));
    IDTX_TRY(out(pval_out, pvals_d, (size_t)m * 8));
    IDTX_TRY(out(significant_out, sig_d, (size_t)m * 4));
    return finish_call(c, st);
}

int idtx_bivariate_te(idtx_ctx *c, const float *series, int n_proc, int64_t T, int target,
                      int n_past, int min_lag, int max_lag, const idtx_settings *s,
                      double *est_out, double *pval_out, void *stream)
{
    if (!c) return fail(IDTX_EINVAL, "ctx is NULL");
    if (!series || !s || !pval_out) return fail(IDTX_EINVAL, "NULL series/settings/pval_out");
    if (n_proc < 2 || target < 0 || target >= n_proc || n_past < 0 || min_lag < 1 ||
        max_lag < min_lag)
        return fail(IDTX_EINVAL, "bad arguments");
    const int n_lags = max_lag - min_lag + 1;
    const int n_cand_total = n_proc * n_lags;
    if (n_cand_total >= (1 << 24)) return fail(IDTX_EINVAL, "too many candidates");
    const int64_t L = std::max(max_lag, n_past);
    if (T <= L || T - L > IDTX_MAX_N) return fail(IDTX_EINVAL, "bad T for the lags");
    if (s->k < 1 || s->k > IDTX_MAX_K || s->k > T - L - 1) return fail(IDTX_EINVAL, "bad k");
    if (s->n_surr < 1 || s->n_surr >= (1 << 24)) return fail(IDTX_EINVAL, "n_surr out of range");
    if (s->mode != IDTX_MODE_BATCHED) return fail(IDTX_EINVAL, "only IDTX_MODE_BATCHED");
    if (n_past > IDTX_MAX_DZ) return fail(IDTX_EINVAL, "n_past exceeds %d", IDTX_MAX_DZ);
    DeviceGuard guard(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const float *ser = series;
    if (!device_accessible(series)) {
        IDTX_TRY(ensure(c, B_IN, (size_t)n_proc * T * sizeof(float)));
        IDTX_CUDA(cudaMemcpyAsync(c->buf[B_IN], series, (size_t)n_proc * T * sizeof(float),
                                  cudaMemcpyHostToDevice, st));
        ser = (const float *)c->buf[B_IN];
    }
    IDTX_TRY(ensure_psi(c, std::max<int64_t>(T - L, s->k) + 1, st));
    IDTX_TRY(begin_call(c, 1, st));
    std::vector<int32_t> row_of(n_cand_total, -1), ids;
    std::vector<Group> gs(1);
    Group &g = gs[0];
    g.n = T - L;
    g.dx = 1;
    g.dy = 1;
    g.dz = n_past;
    g.k = s->k;
    g.ycols.push_back(Col{ser + (int64_t)target * T, L});
    for (int lag = 1; lag <= n_past; ++lag) g.zcols.push_back(Col{ser + (int64_t)target * T, L - lag});
    for (int cid = 0; cid < n_cand_total; ++cid) {
        if (cid / n_lags == target) continue;
        const int a = (int)ids.size();
        row_of[cid] = a;
        ids.push_back(cid);
        g.xcols.push_back(Col{ser + (int64_t)(cid / n_lags) * T, L - (min_lag + cid % n_lags)});
        g.jobs.push_back(Job{a, -1});
        for (int sidx = 0; sidx < s->n_surr; ++sidx) {
            g.jobs.push_back(Job{a, (int32_t)g.slot_stream.size()});
            g.slot_stream.push_back((0xC000ull << 48) | ((uint64_t)cid << 24) | (uint64_t)sidx);
            g.slot_seed.push_back(s->seed);
        }
    }
    IDTX_TRY(plan(c, g));
    const size_t row = 1 + (size_t)s->n_surr;
    IDTX_TRY(run_groups(c, gs, st, timeout_of(c, s), ids.size() * row));
    const double *est = (const double *)c->buf[B_CMI];
    IDTX_TRY(ensure(c, B_STEP, align_up((size_t)n_cand_total * 4, 256) + (size_t)n_cand_total * 8));
    int32_t *row_of_d = (int32_t *)c->buf[B_STEP];
    double *p_d = (double *)((unsigned char *)c->buf[B_STEP] + align_up((size_t)n_cand_total * 4, 256));
    IDTX_CUDA(cudaMemcpyAsync(row_of_d, row_of.data(), (size_t)n_cand_total * 4,
                              cudaMemcpyHostToDevice, st));
    k_cand_pvals<<<(n_cand_total + 127) / 128, 128, 0, st>>>(est, row_of_d, n_cand_total,
                                                             s->n_surr, p_d);
    IDTX_CUDA(cudaGetLastError());
    c->stats.kernel_launches += 1;
    const cudaMemcpyKind pk = device_accessible(pval_out) ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyDeviceToHost;
    IDTX_CUDA(cudaMemcpyAsync(pval_out, p_d, (size_t)n_cand_total * 8, pk, st));
    if (est_out) {
        // rows of the source variables only (the target's own rows are left untouched)
        const cudaMemcpyKind ek = device_accessible(est_out) ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyDeviceToHost;
        for (size_t a = 0; a < ids.size(); ++a)
            IDTX_CUDA(cudaMemcpyAsync(est_out + (size_t)ids[a] * row, est + a * row, row * 8, ek,
                                      st));
    }
    return finish_call(c, st);
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free variant
//
// For callers that cannot allocate device memory: code running where the
// caller's memory pool owns the device and forbids other allocations, code
// on a path where a cudaMalloc would synchronise the device (and so stall
// other work), or long-running services that must not grow their footprint
// after start-up.  It runs idtx_cmi_ksg's preparation kernels and its tile
// kernel (the list kernel's lists would not fit a fixed array), with every
// scratch buffer carved out of one file-scope device array instead.
namespace {

constexpr size_t kNoAllocBytes = IDTX_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoAllocDescBytes = 64 * 1024;  // descriptor block at the start

// The shared scratch: present on every device that loads this library, until
// the process exits.  Host code must not use the name as an address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

void *g_noalloc_ptr[kMaxDevices] = {};  // device address of the array, per device
std::mutex g_noalloc_mu;

// Once per device, with that device current: resolve the array's address.
int noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return fail(IDTX_EINVAL, "device %d", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(IDTX_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                        cudaGetErrorString(e));
        g_noalloc_ptr[device] = p;
    }
    *out = (unsigned char *)g_noalloc_ptr[device];
    return IDTX_OK;
}

const KsgVariant *noalloc_variant(int dx, int dy, int dz, int k)
{
    static KsgVariant table[64];
    static int n_table = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int n = 0;
        n += ksg_variants_d11(table + n);
        n += ksg_variants_d12(table + n);
        n += ksg_variants_d21(table + n);
        n += ksg_variants_d22(table + n);
        n += ksg_variants_generic(table + n);
        n_table = n;
    });
    const int dze = std::max(dz, 1);
    if (k == 4 && dx <= 2 && dy <= 2) {
        int zb = 0;
        for (int b : kZBuckets)
            if (b >= dze) {
                zb = b;
                break;
            }
        for (int i = 0; i < n_table; ++i) {
            const KsgVariant &v = table[i];
            if (v.exact && v.k1 == 5 && v.dx == dx && v.dy == dy && v.dz == zb) return &v;
        }
    }
    for (int i = 0; i < n_table; ++i) {
        const KsgVariant &v = table[i];
        if (!v.exact && v.dx >= dx && v.dy >= dy && v.dz >= dze && v.k1 > k) return &v;
    }
    return nullptr;
}

}  // namespace

extern "C" int idtx_cmi_ksg_noalloc(const float *x, int dx, const float *y, int dy,
                                    const float *z, int dz, int64_t n, int64_t ld,
                                    const idtx_settings *s, double *cmi_out, void *stream)
{
    if (!s || !cmi_out) return fail(IDTX_EINVAL, "settings or cmi_out is NULL");
    if (dx < 1 || dx > IDTX_MAX_DX || dy < 1 || dy > IDTX_MAX_DY || dz < 0 || dz > IDTX_MAX_DZ)
        return fail(IDTX_EINVAL, "dims out of range (dx=%d dy=%d dz=%d)", dx, dy, dz);
    if (n < 2 || n > IDTX_MAX_N || ld < n)
        return fail(IDTX_EINVAL, "bad n=%lld / ld=%lld", (long long)n, (long long)ld);
    if (s->k < 1 || s->k > IDTX_MAX_K || s->k > n - 1)
        return fail(IDTX_EINVAL, "k=%d out of range for n=%lld", s->k, (long long)n);
    if (s->n_surr < 0 || s->n_surr > IDTX_NOALLOC_MAX_SURR)
        return fail(IDTX_EINVAL, "n_surr=%d outside [0, %d]", s->n_surr, IDTX_NOALLOC_MAX_SURR);
    if (!x || !y || (dz > 0 && !z)) return fail(IDTX_EINVAL, "NULL input column");
    if (!device_accessible(x) || !device_accessible(y) || (dz > 0 && !device_accessible(z)) ||
        !device_accessible(cmi_out))
        return fail(IDTX_EINVAL, "inputs and cmi_out must be device memory");
    const KsgVariant *v = noalloc_variant(dx, dy, dz, s->k);
    if (!v) return fail(IDTX_EINVAL, "no kernel for dx=%d dy=%d dz=%d k=%d", dx, dy, dz, s->k);

    // Carve the scratch: [descriptors | err | psi | sh | xi | perm | partial].
    const int n_jobs = 1 + s->n_surr;
    const int n_slots = s->n_surr;
    const int64_t n_pad = (n + kTJ - 1) / kTJ * kTJ;
    const int n_qt = (int)(n_pad / v->qc);
    const int n_groups = (n_jobs + v->gb - 1) / v->gb;
    const int64_t gblocks = gather_blocks(n_groups, n_pad, v->gb, v->dx);
    if (gblocks <= 0) return fail(IDTX_EINVAL, "n = %lld is too large", (long long)n);
    size_t off = kNoAllocDescBytes;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t at_err = take(sizeof(int));
    const size_t at_psi = take((size_t)(std::max<int64_t>(n, s->k) + 2) * sizeof(double));
    const size_t at_sh = take((size_t)(n_pad / kTJ) * kTileRows * v->dsp * sizeof(float));
    const size_t at_xi = take((size_t)n_groups * n_pad * v->gb * v->dx * sizeof(float));
    const size_t at_perm = take((size_t)n_slots * n * sizeof(int32_t));
    const size_t at_partial = take((size_t)n_jobs * n_qt * sizeof(double));
    if (off > kNoAllocBytes)
        return fail(IDTX_EINVAL,
                    "problem needs %zu bytes of scratch; the allocation-free entry point has "
                    "%zu (use idtx_cmi_ksg)",
                    off, kNoAllocBytes);

    int device = 0;
    IDTX_CUDA(cudaGetDevice(&device));
    unsigned char *base = nullptr;
    IDTX_TRY(noalloc_scratch(device, &base));
    cudaStream_t st = (cudaStream_t)stream;

    // Descriptors, built in a fixed host block (no allocation) and copied in.
    unsigned char host_desc[kNoAllocDescBytes];
    size_t doff = 0;
    auto put = [&](const void *src, size_t bytes) {
        doff = align_up(doff, 16);
        const size_t at = doff;
        memcpy(host_desc + at, src, bytes);
        doff += bytes;
        return at;
    };
    Col xc[IDTX_MAX_DX], yc[IDTX_MAX_DY], zc[IDTX_MAX_DZ > 0 ? IDTX_MAX_DZ : 1];
    for (int d = 0; d < dx; ++d) xc[d] = Col{x + d * ld, 0};
    for (int d = 0; d < dy; ++d) yc[d] = Col{y + d * ld, 0};
    for (int d = 0; d < dz; ++d) zc[d] = Col{z + d * ld, 0};
    const size_t o_x = put(xc, sizeof(Col) * dx);
    const size_t o_y = put(yc, sizeof(Col) * dy);
    const size_t o_z = put(zc, sizeof(Col) * std::max(dz, 1));
    doff = align_up(doff, 16);
    const size_t o_jobs = doff;
    for (int j = 0; j < n_jobs; ++j) {
        const Job jb{0, j - 1};
        memcpy(host_desc + doff, &jb, sizeof(Job));
        doff += sizeof(Job);
    }
    doff = align_up(doff, 16);
    const size_t o_streams = doff;
    for (int sl = 0; sl < n_slots; ++sl) {
        const uint64_t v64 = (uint64_t)sl;
        memcpy(host_desc + doff, &v64, sizeof(uint64_t));
        doff += sizeof(uint64_t);
    }
    const size_t o_seeds = doff;
    for (int sl = 0; sl < n_slots; ++sl) {
        memcpy(host_desc + doff, &s->seed, sizeof(uint64_t));
        doff += sizeof(uint64_t);
    }
    if (doff > kNoAllocDescBytes) return fail(IDTX_EINTERNAL, "descriptor block overflow");
    int *err = (int *)(base + at_err);
    double *psi = (double *)(base + at_psi);
    float *sh = (float *)(base + at_sh);
    float *xi = (float *)(base + at_xi);
    int32_t *perm = (int32_t *)(base + at_perm);
    double *partial = (double *)(base + at_partial);
    const int64_t psi_n = std::max<int64_t>(n, s->k) + 1;
    int h_err = 0;
    // Everything from the first enqueue on: on an error the stream is
    // synchronised before returning, so no kernel of this call still uses
    // the shared array when the caller retries.
    auto enqueue = [&]() -> int {
        IDTX_CUDA(cudaMemcpyAsync(base, host_desc, doff, cudaMemcpyHostToDevice, st));
        // The error word must start at zero; every other region is fully
        // written before it is read, so the previous call's contents do not
        // matter.
        IDTX_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
        k_psi_table<<<grid_for(psi_n + 1, 256), 256, 0, st>>>(psi, psi_n);
        IDTX_CUDA(cudaGetLastError());
        k_pack_shared<<<grid_for(n_pad * v->dsp, 256), 256, 0, st>>>(
            (const Col *)(base + o_z), dz, v->dz, (const Col *)(base + o_y), dy, v->dy, v->dsp, n,
            n_pad, nullptr, sh, err);
        IDTX_CUDA(cudaGetLastError());
        k_tile_boxes<<<(unsigned)(n_pad / kTJ), kTJ, 0, st>>>(sh, v->dsp, n);
        IDTX_CUDA(cudaGetLastError());
        int unused_launches = 0;
        bool composed = false;
        IDTX_TRY(enqueue_permutations(perm, (const uint64_t *)(base + o_streams),
                                      (const uint64_t *)(base + o_seeds), n_slots, n, nullptr, st,
                                      unused_launches, &composed));
        k_gather_x<<<(unsigned)gblocks, kGatherThreads, gather_smem(v->gb, v->dx), st>>>(
            (const Col *)(base + o_x), dx, v->dx, (const Job *)(base + o_jobs), n_jobs, perm, n,
            n_pad, v->gb, nullptr, false, xi, err);
        IDTX_CUDA(cudaGetLastError());
        KsgLaunch a;
        a.sh = sh;
        a.xi = xi;
        a.psi = psi;
        a.partial = partial;
        a.eps_out = nullptr;
        a.cnt_out = nullptr;
        a.order = nullptr;
        a.work = nullptr;
        a.err = err;
        a.n = n;
        a.n_pad = n_pad;
        a.n_jobs = n_jobs;
        a.n_qt = n_qt;
        a.k = s->k;
        a.timeout_ns = timeout_of(s);
        IDTX_CUDA(v->fn(a, n_groups, st));
        k_finalize<<<(n_jobs + 127) / 128, 128, 0, st>>>(partial, n_jobs, n_qt, psi, s->k, n,
                                                          cmi_out);
        IDTX_CUDA(cudaGetLastError());
        IDTX_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        return IDTX_OK;
    };
    const int rc = enqueue();
    const cudaError_t se = cudaStreamSynchronize(st);
    if (rc != IDTX_OK) return rc;
    if (se != cudaSuccess)
        return fail(IDTX_ECUDA, "cudaStreamSynchronize failed: %s", cudaGetErrorString(se));
    if (h_err & kErrNonFinite) return fail(IDTX_EINVAL, "input contains NaN or Inf");
    if (h_err & kErrTimeout) return fail(IDTX_ETIMEOUT, "a bounded device wait ran out");
    if (h_err) return fail(IDTX_EINTERNAL, "device error word 0x%x", h_err);
    return IDTX_OK;
}
