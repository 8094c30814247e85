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
// Design (GB300).  A CTA holds 32 jobs, one per lane, and QC queries; the
// unit of work is one (query, reference tile) pair, which a warp processes
// with all 32 jobs in parallel.
//   * All jobs of a group share Y and Z (a surrogate only permutes X, and the
//     candidates of one greedy step differ only in X).  For a unit the warp
//     computes the Y/Z distances of the tile's 128 references once, four per
//     lane, and a ballot marks the references below the query's bound (the
//     largest current threshold over the 32 jobs).  The per-job work then
//     runs only for those references, warp-uniformly, every lane doing its
//     own job: no divergence and no idle lanes.
//   * Pass A keeps, per (query, job), the k+1 smallest joint distances in a
//     sorted array.  The sample itself is never skipped: its own distance 0
//     occupies one slot, so the (k+1)-th smallest including it is the k-th
//     smallest over j != i.
//   * Pass B counts with the same tiles; the pair (i,i) is counted when
//     eps_i > 0 and is subtracted at the end.  A pair can only count when its
//     Z distance is below the largest eps of the query's jobs.
//   * Load balance.  Queries differ widely in work (dense regions pass many
//     references), so units are not owned statically: for each staged tile,
//     warps take the next query from a shared counter.  The per-(query, job)
//     state (heaps, counts, bounds) lives in shared memory; a query's heaps
//     are updated under a per-query lock (the final k+1 smallest do not
//     depend on the order of updates), its counts with shared atomics, and
//     its count units wait until all its heap units are done.
//   * Samples are stored along a Morton curve of the shared coordinates, so a
//     CTA's queries and a tile's references are spatial neighbours; tiles are
//     visited in a spiral from the CTA's own tile, and a unit is skipped when
//     the tile's bounding box (stored with the tile) is at least the query's
//     bound away.  Skipping never changes a result.
//   * Reference tiles (128 samples of sh with the box, and of xi) are staged
//     into shared memory by 1-D TMA bulk copies (cp.async.bulk) completing on
//     per-stage mbarriers, 2-4 stages deep; both passes stream the same tiles.
//     The unit that finishes a tile refills its stage; there is no CTA-wide
//     barrier per tile.  Every wait (mbarrier, lock, pass order) is bounded by
//     %globaltimer; on expiry the CTA records kErrTimeout, waits (bounded) for
//     its own copies in flight and exits without output.
//   * Padding samples (j >= n) are +inf in every column, so they never enter
//     a heap or a count; padding queries and padding jobs are kept out of
//     every bound and masked out of all outputs.
#pragma once

#include <cstdint>
#include <math_constants.h>

#include "ksg_common.cuh"

// Launch-shape knobs (compile-time; the defaults are the tuned values).
#ifndef IDTX_STAGE_BUDGET_KB
#define IDTX_STAGE_BUDGET_KB 40
#endif
#ifndef IDTX_MAX_STAGES
#define IDTX_MAX_STAGES 4
#endif
#ifndef IDTX_FAST_QC
#define IDTX_FAST_QC 64
#endif
#ifndef IDTX_FAST_NW
#define IDTX_FAST_NW 8
#endif
#ifndef IDTX_QUERY_GROUP
#define IDTX_QUERY_GROUP 8
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

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
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

template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS>
struct KsgShape {
    static constexpr int GB = 32;  // jobs per CTA: one per lane
    static constexpr int NW = NWARPS;  // warps per CTA
    static constexpr int THREADS = NW * 32;
    static constexpr int QC = QCTA;  // queries per CTA
    static constexpr int QG = QC < IDTX_QUERY_GROUP ? QC : IDTX_QUERY_GROUP;  // per claim
    static constexpr int DS = DZ + DY;
    static constexpr int DSP = (DS + 3) & ~3;
    static constexpr int XW = GB * DX;
    static constexpr int RPL = kTJ / 32;  // references per lane in a tile
    static constexpr uint32_t SH_BYTES = kTileRows * DSP * sizeof(float);
    static constexpr uint32_t X_BYTES = kTJ * XW * sizeof(float);
    static constexpr uint32_t STAGE_BYTES = SH_BYTES + X_BYTES;
    // Pipeline depth: as many stages as fit in the budget, between 2 and the cap.
    static constexpr int STAGES_RAW = (IDTX_STAGE_BUDGET_KB * 1024) / STAGE_BYTES;
    static constexpr int STAGES =
        STAGES_RAW < 2 ? 2 : (STAGES_RAW > IDTX_MAX_STAGES ? IDTX_MAX_STAGES : STAGES_RAW);
    // dynamic shared memory: stages | barriers | query rows | heaps (pass B:
    // slots 0-2 hold the counts) | k-th values (!EXACT) | query X values |
    // per-warp event lists
    static constexpr size_t BAR_OFF = (size_t)STAGES * STAGE_BYTES;
    static constexpr size_t Q_OFF = (BAR_OFF + STAGES * sizeof(uint64_t) + 15) & ~size_t(15);
    static constexpr size_t H_OFF = Q_OFF + (size_t)QC * DSP * sizeof(float);
    static constexpr size_t KTH_OFF = H_OFF + (size_t)QC * K1 * 32 * sizeof(float);
    static constexpr size_t XQ_OFF = KTH_OFF + (EXACT ? 0 : (size_t)QC * 32 * sizeof(float));
    static constexpr size_t EV_OFF = XQ_OFF + (size_t)QC * DX * 32 * sizeof(float);
    static constexpr int EV_CAP = kTJ + 4;  // a tile's references + sentinel padding
    static constexpr size_t SMEM = EV_OFF + (size_t)NW * EV_CAP * sizeof(float4);
    static_assert(kTJ % QC == 0, "query tiles nest in reference tiles");
    static_assert(QC % QG == 0 && QG <= 32, "query groups tile the CTA's queries");
    static_assert(DS <= 32, "one lane per shared dimension");
    static_assert(STAGE_BYTES % 16 == 0, "bulk copies need 16-byte multiples");
    static_assert(EV_OFF % 16 == 0, "event lists are read as float4");
};

// One CTA's work: query tile qt of job group grp.  Returns false when the
// CTA aborted (a bounded wait ran out).  Shared memory is set up afresh on
// every call, so a persistent CTA may run it repeatedly.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS>
__device__ __forceinline__ bool ksg_cta(const KsgLaunch &a, const int qt, const int grp)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>;
    constexpr int DS = S::DS, DSP = S::DSP, XW = S::XW, NW = S::NW, GB = S::GB, QC = S::QC;
    constexpr int ST = S::STAGES, RPL = S::RPL, QG = S::QG;
    constexpr int kShStage = kTileRows * DSP;  // floats of one sh tile
    constexpr unsigned kFull = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem_raw + S::BAR_OFF);
    float *s_q = reinterpret_cast<float *>(smem_raw + S::Q_OFF);      // [QC][DSP]
    float *s_h = reinterpret_cast<float *>(smem_raw + S::H_OFF);      // [QC][K1][32]
    float *s_kth = reinterpret_cast<float *>(smem_raw + S::KTH_OFF);  // [QC][32]
    float *s_xq = reinterpret_cast<float *>(smem_raw + S::XQ_OFF);    // [QC][DX][32]
    __shared__ float s_b[QC];    // per query: pass-A bound (largest job threshold)
    __shared__ int s_lock[QC];   // per query: owner of its heaps (pass A)
    __shared__ int s_next;       // next unit to take
    __shared__ int s_items_a;    // pass-A items finished
    __shared__ int s_open_b;     // pass B may start: pass A done, counts zeroed
    __shared__ int s_fin[ST];    // units finished of the stage's current item
    __shared__ int s_abort;
    __shared__ int s_last[ST];   // item last issued into the stage
    __shared__ double s_red[NW][GB];
    volatile int *abort_flag = &s_abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // this warp's event list: the references of a unit below the bound
    float4 *s_ev = reinterpret_cast<float4 *>(smem_raw + S::EV_OFF) + warp * S::EV_CAP;
    const int64_t q0 = static_cast<int64_t>(qt) * QC;  // CTA's first query (sorted)
    const int n_tiles = static_cast<int>(a.n_pad / kTJ);
    const int total = 2 * n_tiles;  // items: pass A tiles, then pass B tiles
    const int home = static_cast<int>(q0 / kTJ);
    const int qv = static_cast<int>(a.n - q0 < QC ? a.n - q0 : QC);  // valid queries
    const int job = grp * GB + lane;
    const bool job_ok = job < a.n_jobs;
    const float *xi_grp = a.xi + static_cast<int64_t>(grp) * a.n_pad * XW;
    if (qv <= 0) {
        // Only padding queries (n_pad is a multiple of the reference tile, not
        // of QC): zero partial sums, and no copy is ever issued.
        if (tid < GB && job_ok) a.partial[static_cast<int64_t>(job) * a.n_qt + qt] = 0.0;
        return true;
    }

    // ---------------- set-up: query rows and X values, empty heaps, zero counts
    for (int idx = tid; idx < QC * DSP; idx += S::THREADS) {
        const int m = idx / DSP, d = idx - m * DSP;
        const int64_t qi = q0 + m;
        s_q[idx] = qi < a.n ? a.sh[(qi / kTJ) * kShStage + (qi % kTJ) * DSP + d] : 0.0f;
    }
    for (int idx = tid; idx < QC * DX * 32; idx += S::THREADS) {
        const int m = idx / (DX * 32), r = idx - m * (DX * 32), d = r >> 5, l = r & 31;
        const int64_t qi = q0 + m;
        s_xq[idx] = qi < a.n ? xi_grp[qi * XW + l * DX + d] : 0.0f;
    }
    for (int idx = tid; idx < QC * K1 * 32; idx += S::THREADS) s_h[idx] = CUDART_INF_F;
    if (!EXACT)
        for (int idx = tid; idx < QC * 32; idx += S::THREADS) s_kth[idx] = CUDART_INF_F;
    for (int m = tid; m < QC; m += S::THREADS) {
        s_b[m] = CUDART_INF_F;
        s_lock[m] = 0;
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
            s_last[st] = -1;
            s_fin[st] = 0;
        }
        s_next = 0;
        s_items_a = 0;
        s_open_b = 0;
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int u = 0; u < ST && u < total; ++u) issue(u);

    long long wait_cycles = 0;
    const long long t_begin = clock64();
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.err, kErrTimeout);
    };
    // Control decisions that read shared state other warps may change are
    // taken by lane 0 and broadcast, so the warp never diverges around the
    // full-mask shuffles and ballots.
    auto aborting = [&]() { return __shfl_sync(kFull, *abort_flag, 0) != 0; };
    // Lane 0 waits (bounded) until try() holds, then the warp proceeds with
    // acquire ordering.  False: timed out or the CTA is aborting.
    auto warp_wait = [&](auto try_once) {
        int ok = 1;
        if (lane == 0) {
            if (!try_once()) {
                const long long t0 = global_ns(), c0 = clock64();
                while (!try_once()) {
                    if (*abort_flag || global_ns() - t0 > a.timeout_ns) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
                wait_cycles += clock64() - c0;
            }
            __threadfence_block();
        }
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok && lane == 0) fail();
        return ok != 0;
    };
    // The stage of item u holds its tiles.  The copy of item u is issued only
    // after item u - ST is finished (so its copy has landed); waiting for the
    // issue first keeps the parity test from matching a phase two behind.
    auto acquire = [&](int u) {
        volatile int *last = s_last;
        if (!warp_wait([&] { return last[u % ST] == u; })) return false;
        const long long t0 = clock64();
        const bool got = mbar_wait_bounded(&s_bar[u % ST], static_cast<uint32_t>((u / ST) & 1),
                                           a.timeout_ns);
        wait_cycles += clock64() - t0;
        const bool all = __all_sync(kFull, got);
        if (!all && lane == 0) fail();
        return all && !aborting();
    };

    unsigned long long scanned_a = 0, scanned_b = 0, events_a = 0, events_b = 0;  // per warp

    // ---------------- pass-A unit: query m against the tile of item u
    // The k+1 smallest joint distances of every job.  The heaps of a query are
    // updated under its lock; the set they end with does not depend on the
    // order of the updates.  The bound only filters candidates: any value at
    // least the largest job threshold is correct.
    auto unit_a = [&](int m, int u) {
        const float *rs = stage_sh(u % ST);
        const float *rx = stage_x(u % ST);
        const float *qrow = s_q + m * DSP;
        float qc[DS];
#pragma unroll
        for (int d = 0; d < DS; ++d) qc[d] = qrow[d];
        // Phase 1 (no lock needed): the query's joint Y/Z distance to the lane's references.
        float dv[RPL];
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
            const float *row = rs + (k * 32 + lane) * DSP;
            float dd = fabsf(qc[0] - row[0]);
#pragma unroll
            for (int d = 1; d < DS; ++d) dd = fmaxf(dd, fabsf(qc[d] - row[d]));
            dv[k] = dd;
        }
        scanned_a += kTJ;
        if (!warp_wait([&] { return atomicCAS(&s_lock[m], 0, 1) == 0; })) return false;
        const float bound = s_b[m];
        // Compact the references below the bound into the warp's event list
        // (entry: offset of the reference's X row, Y/Z distance), padded with
        // +inf sentinels to a multiple of four.
        float2 *ev = reinterpret_cast<float2 *>(s_ev);
        const uint32_t lt = (1u << lane) - 1u;
        int n_ev = 0;
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
            const bool p = dv[k] < bound;
            const uint32_t b = __ballot_sync(kFull, p);
            if (p) ev[n_ev + __popc(b & lt)] = make_float2(__int_as_float((k * 32 + lane) * XW), dv[k]);
            n_ev += __popc(b);
        }
        if (lane < 3) ev[n_ev + lane] = make_float2(__int_as_float(0), CUDART_INF_F);
        __syncwarp();
        events_a += n_ev;
        if (n_ev) {
            // The events, all lanes, one job each, four per iteration; a lane
            // inserts an event into its job's k+1 smallest when it is below
            // the job's threshold.
            float *hq = s_h + m * K1 * 32 + lane;  // slot t: hq[t * 32]
            float h[K1];
#pragma unroll
            for (int t = 0; t < K1; ++t) h[t] = hq[t * 32];
            float th = EXACT ? h[K1 - 1] : s_kth[m * 32 + lane];
            float xq[DX];
#pragma unroll
            for (int d = 0; d < DX; ++d) xq[d] = s_xq[(m * DX + d) * 32 + lane];
            const float *rxl = rx + lane * DX;
            for (int e = 0; e < n_ev; e += 4) {
                const float4 p01 = s_ev[e / 2], p23 = s_ev[e / 2 + 1];
                const int o[4] = {__float_as_int(p01.x), __float_as_int(p01.z),
                                  __float_as_int(p23.x), __float_as_int(p23.z)};
                const float dyz[4] = {p01.y, p01.w, p23.y, p23.w};
                float dd[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float dx = fabsf(xq[0] - rxl[o[i]]);
#pragma unroll
                    for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xq[d] - rxl[o[i] + d]));
                    dd[i] = fmaxf(dx, dyz[i]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (dd[i] < th) {
                        sorted_insert<K1>(h, dd[i]);
                        th = EXACT ? h[K1 - 1] : select_kth<K1>(h, a.k);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < K1; ++t) hq[t * 32] = h[t];
            if (!EXACT) s_kth[m * 32 + lane] = th;
            const float nb = warp_max(job_ok ? th : -1.0f);
            if (lane == 0) reinterpret_cast<volatile float *>(s_b)[m] = nb;
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicExch(&s_lock[m], 0);
        }
        return true;
    };

    // ---------------- pass-B unit: strict-radius counts in the subspaces
    // Runs once every pass-A item is finished.  The query's bound is then its
    // final pass-A bound, the largest eps over its jobs.  The counts live in
    // heap slots 0-2 (n_z, n_yz, n_xz; slot K1-1 keeps eps) and are integer
    // sums, added with shared atomics in any order.
    auto unit_b = [&](int m, int u) {
        const float *rs = stage_sh(u % ST);
        const float *rx = stage_x(u % ST);
        const float e = EXACT ? s_h[(m * K1 + K1 - 1) * 32 + lane] : s_kth[m * 32 + lane];
        const float bound = s_b[m];
        const float *qrow = s_q + m * DSP;
        float qc[DS];
#pragma unroll
        for (int d = 0; d < DS; ++d) qc[d] = qrow[d];
        // Compact the references whose Z distance is below the bound into the
        // warp's event list (entry: X row offset, Z distance, Y/Z distance),
        // padded with +inf sentinels to a multiple of four.
        const uint32_t lt = (1u << lane) - 1u;
        int n_ev = 0;
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
            const float *row = rs + (k * 32 + lane) * DSP;
            float dz = fabsf(qc[0] - row[0]);
#pragma unroll
            for (int d = 1; d < DZ; ++d) dz = fmaxf(dz, fabsf(qc[d] - row[d]));
            float dyz = dz;
#pragma unroll
            for (int d = DZ; d < DS; ++d) dyz = fmaxf(dyz, fabsf(qc[d] - row[d]));
            const bool p = dz < bound;
            const uint32_t b = __ballot_sync(kFull, p);
            if (p)
                s_ev[n_ev + __popc(b & lt)] =
                    make_float4(__int_as_float((k * 32 + lane) * XW), dz, dyz, 0.0f);
            n_ev += __popc(b);
        }
        scanned_b += kTJ;
        events_b += n_ev;
        if (n_ev == 0) return true;
        if (lane < 3)
            s_ev[n_ev + lane] = make_float4(__int_as_float(0), CUDART_INF_F, CUDART_INF_F, 0.0f);
        __syncwarp();
        float xq[DX];
#pragma unroll
        for (int d = 0; d < DX; ++d) xq[d] = s_xq[(m * DX + d) * 32 + lane];
        const float *rxl = rx + lane * DX;
        int cz = 0, cyz = 0, cxz = 0;
        for (int ei = 0; ei < n_ev; ei += 4) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = s_ev[ei + i];
                const int o = __float_as_int(v.x);
                float dx = fabsf(xq[0] - rxl[o]);
#pragma unroll
                for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xq[d] - rxl[o + d]));
                // max(dX, dZ) < e  <=>  dX < e and dZ < e
                const bool pz = v.y < e;
                cz += pz ? 1 : 0;
                cyz += v.z < e ? 1 : 0;
                cxz += (pz && dx < e) ? 1 : 0;
            }
        }
        int *c = reinterpret_cast<int *>(s_h) + m * K1 * 32 + lane;
        if (cz) atomicAdd(c, cz);
        if (cyz) atomicAdd(c + 32, cyz);
        if (cxz) atomicAdd(c + 64, cxz);
        __syncwarp();
        return true;
    };

    // ---------------- work loop: query groups taken dynamically
    // Unit t is query group t % NG of item t / NG, so units are taken in item
    // order and any warp takes the next one.  Every unit (one made only of
    // padding queries too) waits for its item's tiles before it counts as
    // finished, so no finish is counted against the stage's previous item.
    // The group's lanes test its queries against the tile's box in parallel;
    // the warp then runs the queries that pass one by one.  The unit that
    // finishes an item refills the item's stage with item u + ST.
    constexpr int NG = QC / QG;
    const int n_units = total * NG;
    int cur = -1;        // item whose stage this warp has acquired
    bool b_ready = false;
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&s_next, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_units) break;
        const int u = t / NG, m0 = (t - u * NG) * QG;
        bool ok = true;
        if (u != cur) {
            ok = acquire(u);
            cur = u;
        }
        const bool pass_b = u >= n_tiles;
        if (ok && pass_b && !b_ready) {
            volatile int *open_b = &s_open_b;
            ok = b_ready = warp_wait([&] { return *open_b != 0; });
        }
        if (ok) {
            const float *rs = stage_sh(u % ST);
            const int mq = m0 + lane;
            bool live = false;
            if (lane < QG && mq < qv) {
                // A bound read without the lock is never below the query's
                // current bound (bounds only shrink), so a skip is safe.
                const float bnd = reinterpret_cast<volatile float *>(s_b)[mq];
                const float *qrow = s_q + mq * DSP;
                float qc[DS];
#pragma unroll
                for (int d = 0; d < DS; ++d) qc[d] = qrow[d];
                const float gap =
                    pass_b ? point_gap<DZ, DSP>(rs, qc) : point_gap<DS, DSP>(rs, qc);
                live = gap < bnd;
            }
            uint32_t todo = __ballot_sync(kFull, live);
            while (todo && ok) {
                const int m = m0 + __ffs(todo) - 1;
                todo &= todo - 1;
                ok = pass_b ? unit_b(m, u) : unit_a(m, u);
            }
        }
        __syncwarp();
        int last_a = 0;  // this unit finished the last pass-A item
        if (lane == 0) {
            __threadfence_block();
            const int st = u % ST;
            if (atomicAdd(&s_fin[st], 1) == NG - 1) {
                s_fin[st] = 0;
                if (u < n_tiles) last_a = atomicAdd(&s_items_a, 1) == n_tiles - 1;
                if (u + ST < total && *abort_flag == 0) {
                    __threadfence_block();
                    fence_proxy_async_smem();
                    issue(u + ST);
                }
            }
        }
        if (__shfl_sync(kFull, last_a, 0)) {
            // Every heap is final: zero the count slots, then open pass B.
            int *hi = reinterpret_cast<int *>(s_h);
            for (int idx = lane; idx < qv * 3 * 32; idx += 32) {
                const int m = idx / 96, r = idx - m * 96;
                hi[m * K1 * 32 + r] = 0;
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                *reinterpret_cast<volatile int *>(&s_open_b) = 1;
            }
        }
        __syncwarp();
        if (!ok) break;
    }

    __syncthreads();
    if (*abort_flag) {
        // Wait (bounded) for this CTA's copies that may still be in flight,
        // then leave.  A copy always lands, so this wait gets at least a
        // second whatever the call's wait limit: the CTA must not exit while
        // a copy into its shared memory is pending.
        const long long drain_ns = a.timeout_ns > 1000000000ll ? a.timeout_ns : 1000000000ll;
        if (tid == 0)
            for (int st = 0; st < ST; ++st)
                if (s_last[st] >= 0)
                    (void)mbar_wait_bounded(&s_bar[st],
                                            static_cast<uint32_t>((s_last[st] / ST) & 1),
                                            drain_ns);
        __syncthreads();
        return false;
    }
    // Every issued copy has landed (each item was waited for by its units).
    if (tid == 0)
        for (int st = 0; st < ST; ++st) mbar_inval(&s_bar[st]);

    // ---------------- epilogue: self pair, outputs, digamma terms (fixed order)
    double tsum = 0.0;
    for (int m = warp; m < QC; m += NW) {
        const int64_t qi = q0 + m;
        if (qi >= a.n || !job_ok) continue;
        const float e = EXACT ? s_h[(m * K1 + K1 - 1) * 32 + lane] : s_kth[m * 32 + lane];
        const int *c = reinterpret_cast<const int *>(s_h) + m * K1 * 32 + lane;
        const int self = e > 0.0f ? 1 : 0;
        const int nz = c[0] - self, nyz = c[32] - self, nxz = c[64] - self;
        tsum += a.psi[nz + 1] - a.psi[nxz + 1] - a.psi[nyz + 1];
        const int64_t orig = a.order ? static_cast<int64_t>(a.order[qi]) : qi;
        if (a.eps_out) a.eps_out[static_cast<int64_t>(job) * a.n + orig] = e;
        if (a.cnt_out) {
            int32_t *co = a.cnt_out + static_cast<int64_t>(job) * 3 * a.n;
            co[orig] = nxz;
            co[a.n + orig] = nyz;
            co[2 * a.n + orig] = nz;
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
    __syncthreads();  // shared state may be reused by the CTA's next task
    return true;
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS>
__global__ void __launch_bounds__(KsgShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>::THREADS)
    ksg_fused_kernel(const KsgLaunch a)
{
    (void)ksg_cta<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>(a, blockIdx.x, blockIdx.y);
}

// Persistent form over the tasks of several problems (KsgTable).  A CTA takes
// the next task, finds its problem by binary search over the task offsets and
// runs it; it stops when the tasks run out or when one of its tasks aborted.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS>
__global__ void __launch_bounds__(KsgShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>::THREADS)
    ksg_fused_persistent(const KsgTable t)
{
    __shared__ KsgLaunch s_prob;
    __shared__ int64_t s_task;
    __shared__ int s_p;
    while (true) {
        if (threadIdx.x == 0) {
            const int64_t task = atomicAdd(t.next, 1);
            int p = 0;
            if (task < t.n_tasks) {
                int lo = 0, hi = t.n_probs - 1;  // last p with start[p] <= task
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (t.start[mid] <= task)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                p = lo;
                s_prob = t.probs[p];
            }
            s_task = task;
            s_p = p;
        }
        __syncthreads();
        const int64_t task = s_task;
        if (task >= t.n_tasks) break;
        const KsgLaunch a = s_prob;
        const int local = static_cast<int>(task - t.start[s_p]);
        __syncthreads();  // s_prob, s_task, s_p are rewritten by the next iteration
        if (!ksg_cta<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>(a, local % a.n_qt, local / a.n_qt))
            break;
    }
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
cudaError_t launch_ksg(const KsgLaunch &a, int n_groups, cudaStream_t stream)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    auto kern = ksg_fused_kernel<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    static DeviceOnce attr;  // the attribute is per function and device
    cudaError_t e = once_per_device(attr, [&](int) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(S::SMEM));
    });
    if (e != cudaSuccess) return e;
    dim3 grid(static_cast<unsigned>(a.n_qt), static_cast<unsigned>(n_groups));
    kern<<<grid, S::THREADS, S::SMEM, stream>>>(a);
    return cudaGetLastError();
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
cudaError_t launch_ksg_table(const KsgTable &t, cudaStream_t stream)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    auto kern = ksg_fused_persistent<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    // CTAs per SM and SMs, per device (written once under the set-up's lock)
    static DeviceOnce setup;
    static int resident[kMaxDevices], n_sms[kMaxDevices];
    cudaError_t e = once_per_device(setup, [&](int d) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(S::SMEM));
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n_sms[d], cudaDevAttrMultiProcessorCount, d);
        if (r == cudaSuccess)
            r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[d], kern, S::THREADS, S::SMEM);
        if (r == cudaSuccess && resident[d] < 1) resident[d] = 1;
        return r;
    });
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int64_t full = static_cast<int64_t>(resident[dev]) * n_sms[dev];
    const unsigned grid = static_cast<unsigned>(t.n_tasks < full ? t.n_tasks : full);
    if (grid == 0) return cudaSuccess;
    kern<<<grid, S::THREADS, S::SMEM, stream>>>(t);
    return cudaGetLastError();
}

}  // namespace idtx
