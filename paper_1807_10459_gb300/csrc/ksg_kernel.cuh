// ksg_kernel.cuh -- the fused KSG estimator kernel (kNN pass, count pass, digamma sum).
//
// Computes, for every job g of a group and every query sample i, the KSG
// conditional-MI statistics (Kraskov, Stoegbauer & Grassberger 2004, algorithm 1
// in its conditional form; the estimator named in the IDTxl paper's Summary,
// paragraph on estimators):
//   eps_i  = k-th smallest max-norm distance to j != i in (X_g, Y, Z)
//   n_xz, n_yz, n_z = strict-radius counts in the subspaces,
// then the per-query digamma term and its sum over the CTA's queries.
//
// Design (GB300).  A CTA holds 32 jobs, one per lane, and NW*QW queries; each
// of its NW warps takes QW consecutive queries and works on one query at a time
// with all 32 jobs in parallel.
//   * All jobs of a group share Y and Z (a surrogate only permutes X, and the
//     candidates of one greedy step differ only in X).  For a (query, tile)
//     the warp computes the Y/Z distances of the tile's 128 references once,
//     four per lane, and a ballot marks the references below the query's
//     bound (the largest current threshold over the 32 jobs).  The per-job
//     work then runs only for those references, warp-uniformly, every lane
//     doing its own job: no divergence and no idle lanes.
//   * Pass A keeps, per (query, job), the k+1 smallest joint distances in a
//     sorted register array.  The sample itself is never skipped: its own
//     distance 0 occupies one slot, so the (k+1)-th smallest including it is
//     the k-th smallest over j != i.
//   * Pass B counts with the same tiles; the pair (i,i) is counted when
//     eps_i > 0 and is subtracted at the end.  A pair can only count when its
//     Z distance is below the largest eps of the query's jobs.
//   * Samples are stored along a Morton curve of the shared coordinates, so a
//     warp's queries and a tile's references are spatial neighbours; tiles are
//     visited in a spiral from the CTA's own tile, and a warp (then a query)
//     skips a tile whose bounding box (stored with the tile) is at least the
//     bound away.  Skipping never changes a result.
//   * Reference tiles (128 samples of sh with the box, and of xi) are staged
//     into shared memory by 1-D TMA bulk copies (cp.async.bulk) completing on
//     per-stage mbarriers, 2-4 stages deep; both passes stream the same tiles.
//     Warps walk the tiles independently; the last warp to finish a stage
//     refills it, so there is no CTA-wide barrier per tile.  Every mbarrier
//     wait is bounded by %globaltimer; on expiry the CTA records kErrTimeout,
//     waits (bounded) for its own copies in flight and exits without output.
//   * Padding samples (j >= n) are +inf in every column, so they never enter
//     a heap or a count; padding queries and padding jobs are kept out of
//     every bound and masked out of all outputs.
#pragma once

#include <cstdint>
#include <math_constants.h>

#include "ksg_common.cuh"

// Launch-shape knobs (compile-time; the defaults are the tuned values).
#ifndef IDTX_STAGE_BUDGET_KB
#define IDTX_STAGE_BUDGET_KB 80
#endif
#ifndef IDTX_MAX_STAGES
#define IDTX_MAX_STAGES 4
#endif
#ifndef IDTX_ROWREG_MAX_DS
#define IDTX_ROWREG_MAX_DS 0
#endif
#ifndef IDTX_FAST_QW
#define IDTX_FAST_QW 2
#endif
#ifndef IDTX_FAST_NW
#define IDTX_FAST_NW 16
#endif

namespace idtx {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > timeout_ns) return false;
    }
}

// 1-D bulk copy global -> shared, completing `bytes` on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_load(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Insert d into the ascending array h[0..K1) (dropping the largest);
// caller guarantees d < h[K1-1].
template <int K1>
__device__ __forceinline__ void sorted_insert(float (&h)[K1], float d)
{
#pragma unroll
    for (int m = K1 - 1; m >= 1; --m) h[m] = fmaxf(h[m - 1], fminf(h[m], d));
    h[0] = fminf(h[0], d);
}

template <int K1>
__device__ __forceinline__ float select_kth(const float (&h)[K1], int k)
{
    float v = h[0];
#pragma unroll
    for (int m = 1; m < K1; ++m)
        if (m == k) v = h[m];
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// u-th tile of the visiting order that starts at tile `home` and alternates
// outwards (home, home+1, home-1, home+2, ...), then finishes the longer side.
__device__ __forceinline__ int spiral_tile(int home, int n_tiles, int u)
{
    if (u == 0) return home;
    const int below = home, above = n_tiles - 1 - home;
    const int m = below < above ? below : above;
    const int v = u - 1;
    if (v < 2 * m) {
        const int k = v / 2 + 1;
        return (v & 1) ? home - k : home + k;
    }
    const int r = v - 2 * m;
    return above > below ? home + m + 1 + r : home - m - 1 - r;
}

// Lower bound, over every pair (point of the query box [lo, hi], sample of the
// tile), of the max-norm distance in the first ND shared dimensions: the
// largest per-dimension gap to the tile's box (row kTJ: minima, row kTJ+1:
// maxima).  Lane d supplies lo/hi of dimension d (ignored for d >= ND).
// Rounding is monotone, so the fp32 gap never exceeds a pair's fp32 distance.
template <int ND, int DSP>
__device__ __forceinline__ float box_gap(const float *rs, float lo, float hi, int lane)
{
    float gap = 0.0f;
    if (lane < ND) gap = fmaxf(gap, fmaxf(lo - rs[(kTJ + 1) * DSP + lane], rs[kTJ * DSP + lane] - hi));
    return warp_max(gap);
}

// The same bound for a single query point q (all lanes compute it; the box
// rows are broadcast reads).
template <int ND, int DSP, int DS>
__device__ __forceinline__ float point_gap(const float *rs, const float (&q)[DS])
{
    float gap = 0.0f;
#pragma unroll
    for (int d = 0; d < ND; ++d)
        gap = fmaxf(gap, fmaxf(q[d] - rs[(kTJ + 1) * DSP + d], rs[kTJ * DSP + d] - q[d]));
    return gap;
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QW, int NWARPS>
struct KsgShape {
    static constexpr int GB = 32;  // jobs per CTA: one per lane
    static constexpr int NW = NWARPS;  // warps per CTA
    static constexpr int THREADS = NW * 32;
    static constexpr int QC = NW * QW;  // queries per CTA
    static constexpr int DS = DZ + DY;
    static constexpr int DSP = (DS + 3) & ~3;
    static constexpr int XW = GB * DX;
    static constexpr int RPL = kTJ / 32;  // references per lane in a tile
    static constexpr bool ROWREG = DS <= IDTX_ROWREG_MAX_DS;  // lane's tile rows in registers
    static constexpr uint32_t SH_BYTES = kTileRows * DSP * sizeof(float);
    static constexpr uint32_t X_BYTES = kTJ * XW * sizeof(float);
    static constexpr uint32_t STAGE_BYTES = SH_BYTES + X_BYTES;
    // Pipeline depth: as many stages as fit in the budget, between 2 and the cap.
    static constexpr int STAGES_RAW = (IDTX_STAGE_BUDGET_KB * 1024) / STAGE_BYTES;
    static constexpr int STAGES =
        STAGES_RAW < 2 ? 2 : (STAGES_RAW > IDTX_MAX_STAGES ? IDTX_MAX_STAGES : STAGES_RAW);
    static constexpr size_t Q_OFF = (size_t)STAGES * STAGE_BYTES + STAGES * sizeof(uint64_t);
    static constexpr size_t SMEM = Q_OFF + (size_t)QC * DSP * sizeof(float);
    static_assert(kTJ % QC == 0, "query tiles nest in reference tiles");
    static_assert(DS <= 32, "one lane per shared dimension in the box test");
    static_assert(STAGE_BYTES % 16 == 0, "bulk copies need 16-byte multiples");
};

template <int DX, int DY, int DZ, int K1, bool EXACT, int QW, int NWARPS>
__global__ void __launch_bounds__(KsgShape<DX, DY, DZ, K1, EXACT, QW, NWARPS>::THREADS)
    ksg_fused_kernel(const KsgLaunch a)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QW, NWARPS>;
    constexpr int DS = S::DS, DSP = S::DSP, XW = S::XW, NW = S::NW, GB = S::GB, QC = S::QC;
    constexpr int ST = S::STAGES, RPL = S::RPL;
    constexpr int kShStage = kTileRows * DSP;  // floats of one sh tile
    // The lane's tile rows live in registers r[RR][RD] when S::ROWREG, else
    // they are read from shared memory each time (r is then a 1x1 dummy).
    constexpr int RR = S::ROWREG ? RPL : 1, RD = S::ROWREG ? DSP : 1;
    auto RI = [](int k) { return S::ROWREG ? k : 0; };
    auto RJ = [](int d) { return S::ROWREG ? d : 0; };

    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem_raw + (size_t)ST * S::STAGE_BYTES);
    float *s_q = reinterpret_cast<float *>(smem_raw + S::Q_OFF);  // [QC][DSP] query rows
    __shared__ int s_abort;
    __shared__ int s_done[ST];  // warps finished with the stage's current item
    __shared__ int s_last[ST];  // last item issued into the stage
    __shared__ double s_red[NW][GB];
    volatile int *abort_flag = &s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int qt = blockIdx.x;
    const int grp = blockIdx.y;
    const int64_t q0 = static_cast<int64_t>(qt) * QC;        // CTA's first query (sorted)
    const int64_t qw0 = q0 + warp * QW;                      // warp's first query
    const int n_tiles = static_cast<int>(a.n_pad / kTJ);
    const int total = 2 * n_tiles;  // items: pass A tiles, then pass B tiles
    const int home = static_cast<int>(q0 / kTJ);
    const int job = grp * GB + lane;
    const bool job_ok = job < a.n_jobs;
    const float *xi_grp = a.xi + static_cast<int64_t>(grp) * a.n_pad * XW;

    // Query rows of the CTA into shared memory (zeros for padding queries).
    for (int idx = tid; idx < QC * DSP; idx += S::THREADS) {
        const int m = idx / DSP, d = idx - m * DSP;
        const int64_t qi = q0 + m;
        s_q[idx] = qi < a.n ? a.sh[(qi / kTJ) * kShStage + (qi % kTJ) * DSP + d] : 0.0f;
    }
    // This lane's job's X value at each of the warp's queries.
    float xq[QW][DX];
    bool qv[QW];
#pragma unroll
    for (int m = 0; m < QW; ++m) {
        qv[m] = qw0 + m < a.n;
#pragma unroll
        for (int d = 0; d < DX; ++d)
            xq[m][d] = qv[m] ? xi_grp[(qw0 + m) * XW + lane * DX + d] : 0.0f;
    }

    auto stage_sh = [&](int st) {
        return reinterpret_cast<float *>(smem_raw + (size_t)st * S::STAGE_BYTES);
    };
    auto stage_x = [&](int st) {
        return reinterpret_cast<float *>(smem_raw + (size_t)st * S::STAGE_BYTES + S::SH_BYTES);
    };
    auto issue = [&](int u) {
        const int tile = spiral_tile(home, n_tiles, u < n_tiles ? u : u - n_tiles);
        const int st = u % ST;
        mbar_arrive_expect_tx(&s_bar[st], S::STAGE_BYTES);
        tma_bulk_load(stage_sh(st), a.sh + static_cast<int64_t>(tile) * kShStage, S::SH_BYTES,
                      &s_bar[st]);
        tma_bulk_load(stage_x(st), xi_grp + static_cast<int64_t>(tile) * kTJ * XW, S::X_BYTES,
                      &s_bar[st]);
        s_last[st] = u;
    };
    if (tid == 0) {
        for (int st = 0; st < ST; ++st) {
            mbar_init(&s_bar[st], 1);
            s_done[st] = 0;
            s_last[st] = -1;
        }
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int u = 0; u < ST && u < total; ++u) issue(u);

    // Bounding box of the warp's valid queries: lane d holds dimension d.
    float qlo = CUDART_INF_F, qhi = -CUDART_INF_F;
    if (lane < DS) {
#pragma unroll
        for (int m = 0; m < QW; ++m)
            if (qv[m]) {
                const float v = s_q[(warp * QW + m) * DSP + lane];
                qlo = fminf(qlo, v);
                qhi = fmaxf(qhi, v);
            }
    }

    // Each warp walks the items on its own; the last warp to finish an item
    // refills its stage with item u + ST.  No CTA-wide barrier per tile.
    long long wait_cycles = 0;
    const long long t_begin = clock64();
    auto acquire = [&](int u) {
        const long long t0 = clock64();
        const bool got = mbar_wait_bounded(&s_bar[u % ST], static_cast<uint32_t>((u / ST) & 1),
                                           a.timeout_ns);
        wait_cycles += clock64() - t0;
        if (!got) {
            *abort_flag = 1;
            atomicOr(a.err, kErrTimeout);
        }
        return *abort_flag == 0;
    };
    auto release = [&](int u) {
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int st = u % ST;
            if (atomicAdd(&s_done[st], 1) == NW - 1) {
                s_done[st] = 0;
                if (u + ST < total && *abort_flag == 0) {
                    fence_proxy_async_smem();
                    issue(u + ST);
                }
            }
        }
        __syncwarp();
    };

    unsigned long long scanned_a = 0, scanned_b = 0, events_a = 0, events_b = 0;  // per warp

    int u = 0;
    bool ok = true;
    float e[QW];
    {
        // ---------------- pass A: per (query, job) the k+1 smallest joint distances
        float h[QW][K1];
        float kth[QW];
        float b[QW];  // per query: largest threshold over the valid jobs (warp-uniform)
#pragma unroll
        for (int m = 0; m < QW; ++m) {
#pragma unroll
            for (int t = 0; t < K1; ++t) h[m][t] = CUDART_INF_F;
            kth[m] = CUDART_INF_F;
            b[m] = qv[m] ? CUDART_INF_F : -1.0f;
        }
        for (; u < n_tiles; ++u) {
            if (!(ok = acquire(u))) break;
            const float *rs = stage_sh(u % ST);
            const float *rx = stage_x(u % ST);
            float bw = b[0];
#pragma unroll
            for (int m = 1; m < QW; ++m) bw = fmaxf(bw, b[m]);
            if (box_gap<DS, DSP>(rs, qlo, qhi, lane) < bw) {
                float r[RR][RD];
                if (S::ROWREG) {
#pragma unroll
                    for (int k = 0; k < RPL; ++k)
#pragma unroll
                        for (int t = 0; t < DSP / 4; ++t) {
                            const float4 v =
                                reinterpret_cast<const float4 *>(rs + (k * 32 + lane) * DSP)[t];
                            r[RI(k)][RJ(4 * t + 0)] = v.x;
                            r[RI(k)][RJ(4 * t + 1)] = v.y;
                            r[RI(k)][RJ(4 * t + 2)] = v.z;
                            r[RI(k)][RJ(4 * t + 3)] = v.w;
                        }
                }
#pragma unroll
                for (int m = 0; m < QW; ++m) {
                    if (!qv[m]) continue;
                    const float *qrow = s_q + (warp * QW + m) * DSP;
                    float qc[DS];
#pragma unroll
                    for (int d = 0; d < DS; ++d) qc[d] = qrow[d];
                    if (point_gap<DS, DSP>(rs, qc) >= b[m]) continue;
                    // Phase 1: the query's distance to the lane's references.
                    float dv[RPL];
                    uint32_t ball[RPL];
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        float dd = 0.0f;
#pragma unroll
                        for (int d = 0; d < DS; ++d) {
                            const float rv = S::ROWREG ? r[RI(k)][RJ(d)]
                                                       : rs[(k * 32 + lane) * DSP + d];
                            dd = d == 0 ? fabsf(qc[0] - rv) : fmaxf(dd, fabsf(qc[d] - rv));
                        }
                        dv[k] = dd;
                        ball[k] = __ballot_sync(0xffffffffu, dd < b[m]);
                    }
                    scanned_a += kTJ;
                    // Phase 2: the passing references, all lanes, one job each; two
                    // references per iteration so their loads overlap.
                    bool any = false;
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        uint32_t msk = ball[k];
                        events_a += __popc(msk);
                        any |= msk != 0;
                        while (msk) {
                            const int l0 = __ffs(msk) - 1;
                            msk &= msk - 1;
                            const bool two = msk != 0;
                            const int l1 = two ? __ffs(msk) - 1 : l0;
                            msk &= msk - 1;
                            const float dyz0 = __shfl_sync(0xffffffffu, dv[k], l0);
                            const float dyz1 = __shfl_sync(0xffffffffu, dv[k], l1);
                            const float *xr0 = rx + (k * 32 + l0) * XW + lane * DX;
                            const float *xr1 = rx + (k * 32 + l1) * XW + lane * DX;
                            float dx0 = fabsf(xq[m][0] - xr0[0]), dx1 = fabsf(xq[m][0] - xr1[0]);
#pragma unroll
                            for (int d = 1; d < DX; ++d) {
                                dx0 = fmaxf(dx0, fabsf(xq[m][d] - xr0[d]));
                                dx1 = fmaxf(dx1, fabsf(xq[m][d] - xr1[d]));
                            }
                            const float dd0 = fmaxf(dx0, dyz0), dd1 = fmaxf(dx1, dyz1);
                            if (dd0 < (EXACT ? h[m][K1 - 1] : kth[m])) {
                                sorted_insert<K1>(h[m], dd0);
                                if (!EXACT) kth[m] = select_kth<K1>(h[m], a.k);
                            }
                            if (two && dd1 < (EXACT ? h[m][K1 - 1] : kth[m])) {
                                sorted_insert<K1>(h[m], dd1);
                                if (!EXACT) kth[m] = select_kth<K1>(h[m], a.k);
                            }
                        }
                    }
                    if (any) b[m] = warp_max(job_ok ? (EXACT ? h[m][K1 - 1] : kth[m]) : -1.0f);
                }
            }
            release(u);
        }
#pragma unroll
        for (int m = 0; m < QW; ++m) e[m] = EXACT ? h[m][K1 - 1] : kth[m];
    }

    int cxz[QW], cyz[QW], cz[QW];
#pragma unroll
    for (int m = 0; m < QW; ++m) {
        cxz[m] = 0;
        cyz[m] = 0;
        cz[m] = 0;
    }
    if (ok) {
        // ---------------- pass B: strict-radius counts in the subspaces
        float b[QW];
        float bw = -1.0f;
#pragma unroll
        for (int m = 0; m < QW; ++m) {
            b[m] = qv[m] ? warp_max(job_ok ? e[m] : -1.0f) : -1.0f;
            bw = fmaxf(bw, b[m]);
        }
        for (; u < total; ++u) {
            if (!(ok = acquire(u))) break;
            const float *rs = stage_sh(u % ST);
            const float *rx = stage_x(u % ST);
            if (box_gap<DZ, DSP>(rs, qlo, qhi, lane) < bw) {
                float r[RR][RD];
                if (S::ROWREG) {
#pragma unroll
                    for (int k = 0; k < RPL; ++k)
#pragma unroll
                        for (int t = 0; t < DSP / 4; ++t) {
                            const float4 v =
                                reinterpret_cast<const float4 *>(rs + (k * 32 + lane) * DSP)[t];
                            r[RI(k)][RJ(4 * t + 0)] = v.x;
                            r[RI(k)][RJ(4 * t + 1)] = v.y;
                            r[RI(k)][RJ(4 * t + 2)] = v.z;
                            r[RI(k)][RJ(4 * t + 3)] = v.w;
                        }
                }
#pragma unroll
                for (int m = 0; m < QW; ++m) {
                    if (!qv[m]) continue;
                    const float *qrow = s_q + (warp * QW + m) * DSP;
                    float qc[DS];
#pragma unroll
                    for (int d = 0; d < DS; ++d) qc[d] = qrow[d];
                    if (point_gap<DZ, DSP>(rs, qc) >= b[m]) continue;
                    float dzv[RPL], dyzv[RPL];
                    uint32_t ball[RPL];
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        float dz = 0.0f, dy = 0.0f;
#pragma unroll
                        for (int d = 0; d < DS; ++d) {
                            const float rv = S::ROWREG ? r[RI(k)][RJ(d)]
                                                       : rs[(k * 32 + lane) * DSP + d];
                            const float ad = fabsf(qc[d] - rv);
                            if (d < DZ)
                                dz = d == 0 ? ad : fmaxf(dz, ad);
                            else
                                dy = d == DZ ? ad : fmaxf(dy, ad);
                        }
                        dzv[k] = dz;
                        dyzv[k] = fmaxf(dz, dy);
                        ball[k] = __ballot_sync(0xffffffffu, dz < b[m]);
                    }
                    scanned_b += kTJ;
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        uint32_t msk = ball[k];
                        events_b += __popc(msk);
                        while (msk) {
                            const int l0 = __ffs(msk) - 1;
                            msk &= msk - 1;
                            const bool two = msk != 0;
                            const int l1 = two ? __ffs(msk) - 1 : l0;
                            msk &= msk - 1;
                            const float dz0 = __shfl_sync(0xffffffffu, dzv[k], l0);
                            const float dz1 = __shfl_sync(0xffffffffu, dzv[k], l1);
                            const float dyz0 = __shfl_sync(0xffffffffu, dyzv[k], l0);
                            const float dyz1 = __shfl_sync(0xffffffffu, dyzv[k], l1);
                            const float *xr0 = rx + (k * 32 + l0) * XW + lane * DX;
                            const float *xr1 = rx + (k * 32 + l1) * XW + lane * DX;
                            float dx0 = fabsf(xq[m][0] - xr0[0]), dx1 = fabsf(xq[m][0] - xr1[0]);
#pragma unroll
                            for (int d = 1; d < DX; ++d) {
                                dx0 = fmaxf(dx0, fabsf(xq[m][d] - xr0[d]));
                                dx1 = fmaxf(dx1, fabsf(xq[m][d] - xr1[d]));
                            }
                            // max(dX, dZ) < e  <=>  dX < e and dZ < e
                            const float em = e[m];
                            const bool pz0 = dz0 < em, pz1 = two && dz1 < em;
                            cz[m] += (pz0 ? 1 : 0) + (pz1 ? 1 : 0);
                            cyz[m] += (dyz0 < em ? 1 : 0) + ((two && dyz1 < em) ? 1 : 0);
                            cxz[m] += ((pz0 && dx0 < em) ? 1 : 0) + ((pz1 && dx1 < em) ? 1 : 0);
                        }
                    }
                }
            }
            release(u);
        }
    }

    __syncthreads();
    if (*abort_flag) {
        // Wait (bounded) for this CTA's copies that may still be in flight, then leave.
        if (tid == 0)
            for (int st = 0; st < ST; ++st)
                if (s_last[st] >= 0)
                    (void)mbar_wait_bounded(&s_bar[st],
                                            static_cast<uint32_t>((s_last[st] / ST) & 1),
                                            a.timeout_ns);
        __syncthreads();
        return;
    }

    // ---------------- epilogue: self pair, outputs, digamma terms
    double tsum = 0.0;
#pragma unroll
    for (int m = 0; m < QW; ++m) {
        if (!qv[m] || !job_ok) continue;
        const int self = e[m] > 0.0f ? 1 : 0;
        const int nxz = cxz[m] - self, nyz = cyz[m] - self, nz = cz[m] - self;
        tsum += a.psi[nz + 1] - a.psi[nxz + 1] - a.psi[nyz + 1];
        const int64_t qi = qw0 + m;
        const int64_t orig = a.order ? static_cast<int64_t>(a.order[qi]) : qi;
        if (a.eps_out) a.eps_out[static_cast<int64_t>(job) * a.n + orig] = e[m];
        if (a.cnt_out) {
            int32_t *c = a.cnt_out + static_cast<int64_t>(job) * 3 * a.n;
            c[orig] = nxz;
            c[a.n + orig] = nyz;
            c[2 * a.n + orig] = nz;
        }
    }
    s_red[warp][lane] = tsum;
    if (a.work && lane == 0) {
        atomicAdd(&a.work[0], scanned_a);
        atomicAdd(&a.work[1], events_a);
        atomicAdd(&a.work[2], scanned_b);
        atomicAdd(&a.work[3], events_b);
        atomicAdd(&a.work[4], static_cast<unsigned long long>(wait_cycles));
        atomicAdd(&a.work[5], static_cast<unsigned long long>(clock64() - t_begin));
    }
    __syncthreads();
    if (tid < GB && job_ok) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += s_red[w][tid];
        a.partial[static_cast<int64_t>(job) * a.n_qt + qt] = s;
    }
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QW, int NWARPS>
cudaError_t launch_ksg(const KsgLaunch &a, int n_groups, cudaStream_t stream)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QW, NWARPS>;
    auto kern = ksg_fused_kernel<DX, DY, DZ, K1, EXACT, QW, NWARPS>;
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(S::SMEM));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid(static_cast<unsigned>(a.n_qt), static_cast<unsigned>(n_groups));
    kern<<<grid, S::THREADS, S::SMEM, stream>>>(a);
    return cudaGetLastError();
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QW, int NWARPS>
KsgVariant make_variant()
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QW, NWARPS>;
    return KsgVariant{DX, DY, DZ, K1, EXACT ? 1 : 0, S::GB, S::DSP, S::QC,
                      &launch_ksg<DX, DY, DZ, K1, EXACT, QW, NWARPS>};
}

}  // namespace idtx
