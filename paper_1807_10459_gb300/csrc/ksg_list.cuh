// ksg_list.cuh -- the KSG estimator over per-query sorted neighbour lists.
//
// Computes the same statistics as ksg_fused_kernel (ksg_kernel.cuh) -- for
// every job g of a group and every query sample i, eps_i (k-th smallest
// max-norm distance to j != i in (X_g, Y, Z)), the strict-radius counts n_xz,
// n_yz, n_z and the digamma term (KSG algorithm 1, conditional form, the
// estimator named in the IDTxl paper's Summary) -- in another order of work.
//
// Every job of a group shares Y and Z (a surrogate only permutes X; the
// candidates of one greedy step differ only in X), so the neighbourhoods in
// the (Y,Z) and Z subspaces are the same for all of them.  k_build_lists
// (lists.cu) sorts them once per query i, for all jobs together:
//   list A: every j != i with d_YZ(i,j) < r_A(i), ascending by d_YZ,
//   list B: every j != i with d_Z(i,j)  < r_B(i), ascending by d_Z,
// at most cap_a / cap_b entries, r_A and r_B chosen so.  Per (query, job):
//   pass A: eps_i = k-th smallest of max(d_X, d_YZ) over j != i.  Walking
//     list A in order, an entry whose d_YZ is at least the current k-th value
//     cannot enter (the joint distance is at least d_YZ), nor can any later
//     one, so the walk stops there.  If the list runs out while the k-th
//     value is still above r_A, an unlisted sample might enter: that job is
//     recomputed by a full scan.
//   pass B: n_yz = #{list A entries with d_YZ < eps} (binary search over the
//     prefix pass A walked); n_z and n_xz counted over the list B entries with
//     d_Z < eps, using max(d_X, d_Z) < eps <=> d_X < eps and d_Z < eps.  Both
//     are exact when eps <= r_A and eps <= r_B (every sample closer than eps
//     is listed); otherwise the job's counts come from a full scan.
// Every distance is formed from the same fp32 differences and maxima as in
// the definition, so eps and the counts are exact, and the digamma terms are
// summed in the same order as ksg_fused_kernel's: both kernels give
// bit-identical estimates and either may serve a call.
//
// Design (GB300).  The kernel is persistent: one CTA of 32 warps per SM, one
// job per lane.  A CTA takes chunks of up to 8 consecutive query tiles of one
// job group (chunks ordered query block by query block, so the CTAs in flight
// share the lists of one block of queries), and its warps take the chunk's
// queries one at a time from a shared counter.  So at any moment the
// SM's warps serve ~32 consecutive queries of one group: samples are in Morton
// order of (Z, Y), the neighbourhoods of consecutive queries overlap, and the
// X rows the walks gather (one 128-byte row of xi per list entry: the 32 jobs'
// X at that sample) are reused from L1 instead of L2.  Shared memory holds
// only the per-query digamma terms of the last few query tiles (a ring of
// tile slots, so the terms can be summed in the fixed order once a tile's 64
// queries are done), the warps' staged list entries and work counters; the
// rest of the SM's 256 KB serves as L1.
//   * Walks read their list 32 entries at a time with one coalesced load (the
//     next chunk prefetched), stage them in the warp's shared buffer and
//     consume them in sub-chunks whose X rows are loaded back to back.  The
//     shared walks are warp-uniform (they stop when every lane's job is done);
//     the one or two jobs that would lengthen a walk most finish lane-split
//     (the 32 lanes splitting the entries), two or four blocks of entries per
//     step so that the loads of a step are in flight together.
//   * The only waits are on the tile ring: a warp that takes a query of tile
//     t waits until tile t - RING has been summed (that tile's queries were
//     all taken earlier, so the wait always ends); the wait is bounded by
//     %globaltimer, and on expiry the CTA records kErrTimeout and stops.
#pragma once

#include "ksg_kernel.cuh"
#include "ksg_plain.cuh"

// List entries per sub-chunk of the neighbour-pass and count-pass walks
// (even divisors of 32; compile-time knobs, the defaults are the tuned values:
// on GB300, list kernel of the greedy step, interleaved runs, SA/SB = 16/16
// 15.55-15.73 ms, 8/16 15.53-15.55, 16/8 15.55, 8/8 16.05).
#ifndef IDTX_LIST_SA
#define IDTX_LIST_SA 8
#endif
#ifndef IDTX_LIST_SB
#define IDTX_LIST_SB 16
#endif
// Jobs of a warp whose neighbour walk goes on past the others' and is
// finished with the lanes splitting its entries.
#ifndef IDTX_LIST_TAIL_A
#define IDTX_LIST_TAIL_A 2
#endif
// The shared count walk hands over to the repacked phases once at most this
// many jobs (a power of two <= 16) still need entries.
#ifndef IDTX_LIST_REPACK
#define IDTX_LIST_REPACK 8
#endif
// Entries a lane takes per step of a repacked count phase (their X loads are
// in flight together; a step's entries past the lane's share are predicated
// off).  Measured on GB300, list kernel of the greedy step: 1 / 2 / 4 / 8
// entries 15.80 / 15.75 / 16.05 / 17.72 ms.
#ifndef IDTX_LIST_PHASE_STEP
#define IDTX_LIST_PHASE_STEP 2
#endif
// Job groups per super-block of the chunk order (see the kernel).
#ifndef IDTX_LIST_GSB
#define IDTX_LIST_GSB 16
#endif
// Most consecutive query tiles a CTA takes at a time (fewer when the call
// has too few tiles to give every SM two chunks; the ring's depth,
// kListRing, is in ksg_common.cuh).
#ifndef IDTX_LIST_CHUNK
#define IDTX_LIST_CHUNK 8
#endif

namespace idtx {

// Number of entries of the ascending list l[0..hi) whose distance is below v.
__device__ __forceinline__ int list_lower(const int2 *l, int hi, float v)
{
    int lo = 0;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__int_as_float(__ldg(&l[mid].y)) < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Warp minimum / maximum of non-negative floats (distances, +inf allowed):
// their bit patterns order like unsigned integers, so one redux does it.
__device__ __forceinline__ float warp_min_nn(float v)
{
    return __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(v)));
}

__device__ __forceinline__ float warp_max_nn(float v)
{
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}

// Launch shape of the list kernel for one specialisation.  QC, NWS: the tile
// kernel's queries per CTA and interleaved sums, which fix the partial-sum
// layout (one partial per QC queries) and the order of the sums.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS>
struct ListShape {
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>;
    static constexpr int QC = S::QC;
    // 32 warps (64 registers a thread) for the small specialisations; 16
    // warps give the wide runtime-k one 128 registers.
    static constexpr int NW = (DX > 2 || K1 > 8) ? 16 : 32;
    static constexpr int THREADS = NW * 32;
    static constexpr int RING = kListRing;
    static_assert(QC <= 64, "the term ring holds tiles of up to 64 queries");
    struct Smem {
        int2 ent[NW][32];  // per warp: staged list entries
        unsigned long long work[NW][kNumWork];
        int owner[RING];  // the CTA-local tile number a slot currently serves
        int done[RING];   // queries of that tile finished
        int next;         // next CTA-local query position
    };
    static constexpr size_t SMEM = sizeof(Smem);
};

// Wait until *owner == want (tile slot free), bounded by timeout_ns.
__device__ __forceinline__ bool wait_slot(const int *owner, int want, long long timeout_ns)
{
    const volatile int *o = owner;
    if (*o == want) return true;
    const long long t0 = global_ns();
    while (*o != want) {
        if (global_ns() - t0 > timeout_ns) return false;
        __nanosleep(32);
    }
    return true;
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS>
__global__ void __launch_bounds__(ListShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>::THREADS, 1)
    ksg_list_kernel(const KsgLaunch a, const int n_groups, const int n_chunks, const int chunk_lg)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>;
    using LS = ListShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>;
    constexpr int DS = S::DS, DSP = S::DSP, XW = S::XW, GB = S::GB, QC = S::QC;
    constexpr int NWS = S::NW;  // interleaved sums of the tile kernel
    constexpr int NW = LS::NW, RING = LS::RING;
    constexpr int KH = K1 - 1;  // smallest distances kept (EXACT: exactly k)
    constexpr int kShStage = kTileRows * DSP;
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int SA = IDTX_LIST_SA, SB = IDTX_LIST_SB;  // entries per sub-chunk of the walks
    constexpr int TAIL_A = IDTX_LIST_TAIL_A;  // and after the shared neighbour walk
    const float kInf = CUDART_INF_F;

    extern __shared__ __align__(16) unsigned char l_smem[];
    auto &sm = *reinterpret_cast<typename LS::Smem *>(l_smem);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid < RING) {
        sm.owner[tid] = tid;
        sm.done[tid] = 0;
    }
    if (tid == 0) sm.next = 0;
    for (int i = tid; i < NW * kNumWork; i += LS::THREADS) (&sm.work[0][0])[i] = 0;
    __syncthreads();

    int2 *ent = sm.ent[warp];
    const int2 sentinel = make_int2(0, __float_as_int(CUDART_INF_F));
    const int kk = a.k;
    auto kth = [&](const float(&h)[KH]) { return EXACT ? h[KH - 1] : select_kth<KH>(h, kk - 1); };
    auto sh_row = [&](int64_t j) { return a.sh + (j / kTJ) * kShStage + (j % kTJ) * DSP; };
    const long long t_begin = clock64();

    while (true) {
        // ---------------- take the CTA's next query: tile lt of its stream is
        // tile lt mod 2^chunk_lg of chunk blockIdx.x + (lt >> chunk_lg) *
        // gridDim.x.  Chunks run in super-blocks of GSB groups, query block
        // by query block within a super-block, so the CTAs in flight share a
        // few groups' X rows and a range of queries' lists in L2, while each
        // CTA's warps serve consecutive queries of one group.  Tiles past a
        // group's last one (its last block may be short) are claimed as
        // empty.
        int p = 0;
        if (lane == 0) p = atomicAdd(&sm.next, 1);
        p = __shfl_sync(kFull, p, 0);
        const int lt = p / QC, m = p - lt * QC;
        const int chunk = static_cast<int>(blockIdx.x) + (lt >> chunk_lg) * static_cast<int>(gridDim.x);
        if (chunk >= n_chunks) break;
        const int slot = lt % RING;
        int ok = 1;
        if (lane == 0) ok = wait_slot(&sm.owner[slot], lt, a.timeout_ns) ? 1 : 0;
        ok = __shfl_sync(kFull, ok, 0);
        if (!ok) {
            if (lane == 0) atomicOr(a.err, kErrTimeout);
            break;
        }
        __threadfence_block();
        // (32-bit: n_chunks, the chunk count, fits an int; see the launcher)
        const int n_qb = (a.n_qt + (1 << chunk_lg) - 1) >> chunk_lg;
        const int per_sb = IDTX_LIST_GSB * n_qb;
        const int sb = chunk / per_sb;
        const int g0 = sb * IDTX_LIST_GSB;
        const int gs = n_groups - g0 < IDTX_LIST_GSB ? n_groups - g0 : IDTX_LIST_GSB;
        const int rc = chunk - sb * per_sb;
        const int qblock = rc / gs;
        const int grp = g0 + (rc - qblock * gs);
        const int qt = (qblock << chunk_lg) + (lt & ((1 << chunk_lg) - 1));
        const int64_t qi = static_cast<int64_t>(qt) * QC + m;  // >= n_pad past the last tile
        const int job = grp * GB + lane;
        const bool job_ok = job < a.n_jobs;
        double term = 0.0;

        if (qi < a.n) {
            const float *xg = a.xi + static_cast<int64_t>(grp) * a.n_pad * XW + lane * DX;
            auto x_dist = [&](const float(&xq)[DX], int64_t j) {
                const float *xr = xg + j * XW;
                float dx = fabsf(xq[0] - xr[0]);
#pragma unroll
                for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xq[d] - xr[d]));
                return dx;
            };
            // per-query work counters (warp-uniform)
            unsigned ta = 0, tb = 0, nfa = 0, nfb = 0;
            float xq[DX];
#pragma unroll
            for (int d = 0; d < DX; ++d) xq[d] = xg[qi * XW + d];
            const int4 meta = __ldg(&a.lmeta[qi]);
            const int len_a = meta.x, len_b = meta.y;
            const float r_a = __int_as_float(meta.z), r_b = __int_as_float(meta.w);
            const int2 *la = a.list_a + qi * a.cap_a;
            const int2 *lb = a.list_b + qi * a.cap_b;

            float qc[DS];  // the query's shared coordinates (full-scan fallbacks only)
            bool have_q = false;
            auto load_q = [&]() {
                if (have_q) return;
                const float *qr = sh_row(qi);
#pragma unroll
                for (int d = 0; d < DS; ++d) qc[d] = qr[d];
                have_q = true;
            };

            // ---------------- pass A: the k smallest joint distances
            float h[KH];
#pragma unroll
            for (int t = 0; t < KH; ++t) h[t] = kInf;
            float th = job_ok ? kInf : -1.0f;  // padding jobs never insert
            int walked_a = 0;
            uint32_t amask = 0;  // jobs the shared walk left to finish lane-split
            {
                int2 nxt = len_a > 0 ? __ldg(la + lane) : sentinel;
                for (int e = 0; e < len_a; e += 32) {
                    const int2 cur = nxt;
                    if (e + 32 < len_a) nxt = __ldg(la + e + 32 + lane);
                    __syncwarp();
                    ent[lane] = cur;
                    __syncwarp();
                    int u = 0;
                    for (; u < 32; u += SA) {
                        // Ascending list: once the sub-chunk's first entry is
                        // out of a job's reach, so is everything after it.
                        // When at most TAIL_A jobs are still in reach the
                        // shared walk stops and those finish lane-split below.
                        const uint32_t act =
                            __ballot_sync(kFull, __int_as_float(ent[u].y) < th);
                        if (__popc(act) <= TAIL_A) {
                            amask = act;
                            break;
                        }
                        int jj[SA];
                        float dyz[SA], dd[SA];
#pragma unroll
                        for (int t = 0; t < SA; t += 2) {
                            const int4 q = *reinterpret_cast<const int4 *>(&ent[u + t]);
                            jj[t] = q.x;
                            dyz[t] = __int_as_float(q.y);
                            jj[t + 1] = q.z;
                            dyz[t + 1] = __int_as_float(q.w);
                        }
#pragma unroll
                        for (int t = 0; t < SA; ++t) dd[t] = x_dist(xq, jj[t]);
#pragma unroll
                        for (int t = 0; t < SA; ++t) {
                            const float d = fmaxf(dd[t], dyz[t]);
                            if (d < th) {
                                sorted_insert<KH>(h, d);
                                th = kth(h);
                            }
                        }
                    }
                    walked_a = e + u;
                    if (u < 32) break;
                }
            }
            if (walked_a > len_a) walked_a = len_a;
            // Lane-split finish of the remaining jobs, one at a time: steps of
            // two blocks of 32 entries, one entry per lane and block; the
            // distances below the job's k-th value are inserted smallest first
            // (warp minimum) until the step's last entry is out of reach.
            // my_walked: the prefix of list A this lane's job walked.
            int my_walked = walked_a;
            while (amask) {
                const int f = __ffs(amask) - 1;
                amask &= amask - 1;
                float xf[DX];
#pragma unroll
                for (int d = 0; d < DX; ++d) xf[d] = __shfl_sync(kFull, xq[d], f);
                const float *xgf = xg - lane * DX + f * DX;
                float thf = __shfl_sync(kFull, th, f);
                int pos = walked_a;
                while (pos < len_a) {
                    const int p0 = pos + lane, p1 = pos + 32 + lane;
                    const int2 e0 = p0 < len_a ? __ldg(la + p0) : sentinel;
                    const int2 e1 = p1 < len_a ? __ldg(la + p1) : sentinel;
                    const float y0 = __int_as_float(e0.y), y1 = __int_as_float(e1.y);
                    if (!(__shfl_sync(kFull, y0, 0) < thf)) break;
                    float c0 = kInf, c1 = kInf;
                    if (y0 < thf) {
                        const float *xr = xgf + static_cast<int64_t>(e0.x) * XW;
                        float dx = fabsf(xf[0] - xr[0]);
#pragma unroll
                        for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xf[d] - xr[d]));
                        c0 = fmaxf(dx, y0);
                    }
                    if (y1 < thf) {
                        const float *xr = xgf + static_cast<int64_t>(e1.x) * XW;
                        float dx = fabsf(xf[0] - xr[0]);
#pragma unroll
                        for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xf[d] - xr[d]));
                        c1 = fmaxf(dx, y1);
                    }
                    if (!(c0 < thf)) c0 = kInf;
                    if (!(c1 < thf)) c1 = kInf;
                    while (true) {
                        const float mn = warp_min_nn(fminf(c0, c1));
                        if (!(mn < thf)) break;
                        const uint32_t w0 = __ballot_sync(kFull, c0 == mn);
                        if (w0) {
                            if (lane == __ffs(w0) - 1) c0 = kInf;
                        } else {
                            const uint32_t w1 = __ballot_sync(kFull, c1 == mn);
                            if (lane == __ffs(w1) - 1) c1 = kInf;
                        }
                        if (lane == f) {
                            sorted_insert<KH>(h, mn);
                            th = kth(h);
                        }
                        thf = __shfl_sync(kFull, th, f);
                    }
                    ta += (len_a - pos < 64) ? static_cast<unsigned>(len_a - pos) : 64u;
                    pos += 64;
                    // ascending: if the step's last entry is out of reach, so is the rest
                    if (!(__shfl_sync(kFull, y1, 31) < thf)) break;
                }
                if (lane == f) my_walked = pos < len_a ? pos : len_a;
            }
            // The list ran out before the job's k-th distance dropped to r_A:
            // recompute those jobs over every sample.  For each such job the
            // 32 lanes split the samples, keep their own k smallest, and the
            // warp merges them (repeatedly taking the smallest head).
            const bool fa = job_ok && th > r_a;
            float eps_fix = 0.0f;
            uint32_t fmask = __ballot_sync(kFull, fa);
            if (fmask) load_q();
            nfa = __popc(fmask);
            while (fmask) {
                const int f = __ffs(fmask) - 1;
                fmask &= fmask - 1;
                float xf[DX];
#pragma unroll
                for (int d = 0; d < DX; ++d) xf[d] = __shfl_sync(kFull, xq[d], f);
                const float *xgf = xg - lane * DX + f * DX;
                float hl[KH];
#pragma unroll
                for (int t = 0; t < KH; ++t) hl[t] = kInf;
                float thl = kInf;
                for (int64_t j = lane; j < a.n; j += 32) {
                    const float *row = sh_row(j);
                    float dyz = fabsf(qc[0] - row[0]);
#pragma unroll
                    for (int d = 1; d < DS; ++d) dyz = fmaxf(dyz, fabsf(qc[d] - row[d]));
                    const float *xr = xgf + j * XW;
                    float dx = fabsf(xf[0] - xr[0]);
#pragma unroll
                    for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xf[d] - xr[d]));
                    const float dd = fmaxf(dx, dyz);
                    if (dd < thl && j != qi) {
                        sorted_insert<KH>(hl, dd);
                        thl = kth(hl);
                    }
                }
                float kv = kInf;
                for (int t = 0; t < kk; ++t) {
                    kv = warp_min_nn(hl[0]);
                    const uint32_t who = __ballot_sync(kFull, hl[0] == kv);
                    if (lane == __ffs(who) - 1) {
#pragma unroll
                        for (int mm = 0; mm + 1 < KH; ++mm) hl[mm] = hl[mm + 1];
                        hl[KH - 1] = kInf;
                    }
                }
                if (lane == f) eps_fix = kv;
            }
            const float eps = job_ok ? (fa ? eps_fix : kth(h)) : -1.0f;

            // ---------------- pass B: strict-radius counts
            const bool fb = job_ok && (eps > r_a || eps > r_b);
            int nz = 0, nyz = 0, nxz = 0;
            // Every list A entry below eps lies in the walked prefix (the walk
            // went on until each job's k-th value was at most the next entry).
            if (job_ok && !fb) nyz = list_lower(la, my_walked, eps);
            // The count walk over list B, for every job the entries below its
            // eps (n_z) and those also within eps in X (n_xz).  While more
            // than 16 jobs still need entries the warp walks the list shared,
            // one job per lane (a sub-chunk is skipped by a job whose eps is
            // at most its first entry).  Then the jobs still walking are
            // repacked: with c of them left, each takes 32/M lanes (M the
            // power of two >= c), which split the entries of each staged
            // chunk between them, and at every chunk boundary the warp
            // repacks again once at most M/2 jobs need more -- so no more
            // than half the lanes ever walk for jobs that are done.
            const float ev = (job_ok && !fb) ? eps : 0.0f;
            int walked_b = 0;
            int cf = 0, co = 0;  // staged chunk [cf, cf+32), next entry cf+co
            int2 nxt = len_b > 0 ? __ldg(lb + lane) : sentinel;
            uint32_t rem = 0;  // lanes whose job still needs entries after the shared phase
            for (; cf < len_b; cf += 32) {
                const int2 cur = nxt;
                if (cf + 32 < len_b) nxt = __ldg(lb + cf + 32 + lane);
                __syncwarp();
                ent[lane] = cur;
                __syncwarp();
                int u = 0;
                for (; u < 32; u += SB) {
                    const uint32_t act = __ballot_sync(kFull, ev > __int_as_float(ent[u].y));
                    if (__popc(act) <= IDTX_LIST_REPACK) {
                        rem = act;
                        break;
                    }
                    int jj[SB];
                    float dz[SB], dx[SB];
#pragma unroll
                    for (int t = 0; t < SB; t += 2) {
                        const int4 q = *reinterpret_cast<const int4 *>(&ent[u + t]);
                        jj[t] = q.x;
                        dz[t] = __int_as_float(q.y);
                        jj[t + 1] = q.z;
                        dz[t + 1] = __int_as_float(q.w);
                    }
#pragma unroll
                    for (int t = 0; t < SB; ++t) dx[t] = x_dist(xq, jj[t]);
#pragma unroll
                    for (int t = 0; t < SB; ++t) {
                        const bool pz = dz[t] < eps;
                        nz += pz ? 1 : 0;
                        nxz += (pz && dx[t] < eps) ? 1 : 0;
                    }
                }
                if (u < 32) {
                    co = u;
                    break;
                }
            }
            walked_b = cf + co < len_b ? cf + co : len_b;
            // Repacked phases: M job slots (M a power of two <= 16), slot s on
            // lanes s, s+M, ..., which take the staged chunk's entries r,
            // r + 32/M, ... (r = lane / M), IDTX_LIST_PHASE_STEP per step.
            while (rem) {
                const int c = __popc(rem);
                const int lg = c > 8 ? 4 : (c > 4 ? 3 : (c > 2 ? 2 : (c > 1 ? 1 : 0)));
                const int M = 1 << lg, per = 32 >> lg;
                const int s = lane & (M - 1), r = lane >> lg;
                const bool slot_ok = s < c;
                uint32_t mm = rem;  // the job of slot s: the (s+1)-th lane of rem
                for (int t = 0; t < s && t < c; ++t) mm &= mm - 1;
                const int home = slot_ok ? __ffs(mm) - 1 : lane;
                const float e_home = __shfl_sync(kFull, ev, home);
                const float es = slot_ok ? e_home : 0.0f;
                float xs[DX];
#pragma unroll
                for (int d = 0; d < DX; ++d) xs[d] = __shfl_sync(kFull, xq[d], home);
                const float *xgs = xg + (home - lane) * DX;
                int cz = 0, cx = 0;
                uint32_t still = 0;
                while (true) {
                    for (int u0 = 0; u0 < M; u0 += IDTX_LIST_PHASE_STEP) {
                        constexpr int PS = IDTX_LIST_PHASE_STEP;
                        bool in[PS];
                        float xv[PS][DX];
#pragma unroll
                        for (int t = 0; t < PS; ++t) {
                            const int idx = r + per * (u0 + t);
                            const int2 e = ent[idx & 31];
                            in[t] = u0 + t < M && idx >= co && __int_as_float(e.y) < es;
                            const float *xr = xgs + static_cast<int64_t>(e.x) * XW;
#pragma unroll
                            for (int d = 0; d < DX; ++d) xv[t][d] = in[t] ? xr[d] : xs[d];
                        }
#pragma unroll
                        for (int t = 0; t < PS; ++t) {
                            float dxv = fabsf(xs[0] - xv[t][0]);
#pragma unroll
                            for (int d = 1; d < DX; ++d) dxv = fmaxf(dxv, fabsf(xs[d] - xv[t][d]));
                            cz += in[t] ? 1 : 0;
                            cx += (in[t] && dxv < es) ? 1 : 0;
                        }
                    }
                    tb += static_cast<unsigned>(c * (32 - co));
                    cf += 32;
                    co = 0;
                    still = 0;
                    if (cf >= len_b) break;  // the list is done: so is every job
                    // jobs that need entries of the next chunk (slot lanes 0..M-1)
                    const float dn = __int_as_float(__shfl_sync(kFull, nxt.y, 0));
                    still = __ballot_sync(kFull, r == 0 && es > dn);
                    const int2 cur = nxt;
                    if (cf + 32 < len_b) nxt = __ldg(lb + cf + 32 + lane);
                    __syncwarp();
                    ent[lane] = cur;
                    __syncwarp();
                    if (__popc(still) <= (M >> 1)) break;
                }
                // each slot's total over its lanes, then to the job's lane
                for (int off = M; off < 32; off <<= 1) {
                    cz += __shfl_xor_sync(kFull, cz, off);
                    cx += __shfl_xor_sync(kFull, cx, off);
                }
                const int rank = __popc(rem & ((1u << lane) - 1u));
                const int vz = __shfl_sync(kFull, cz, rank & 31);
                const int vx = __shfl_sync(kFull, cx, rank & 31);
                if ((rem >> lane) & 1u) {
                    nz += vz;
                    nxz += vx;
                }
                rem = __reduce_or_sync(kFull, (r == 0 && ((still >> lane) & 1u)) ? (1u << home) : 0u);
            }
            // Jobs whose eps reaches past a list: counts by a full scan, the
            // 32 lanes splitting the samples of one such job at a time.
            uint32_t bmask = __ballot_sync(kFull, fb);
            if (bmask) load_q();
            nfb = __popc(bmask);
            while (bmask) {
                const int f = __ffs(bmask) - 1;
                bmask &= bmask - 1;
                float xf[DX];
#pragma unroll
                for (int d = 0; d < DX; ++d) xf[d] = __shfl_sync(kFull, xq[d], f);
                const float ef = __shfl_sync(kFull, eps, f);
                const float *xgf = xg - lane * DX + f * DX;
                int cz = 0, cyz = 0, cxz = 0;
                for (int64_t j = lane; j < a.n; j += 32) {
                    const float *row = sh_row(j);
                    float dz = fabsf(qc[0] - row[0]);
#pragma unroll
                    for (int d = 1; d < DZ; ++d) dz = fmaxf(dz, fabsf(qc[d] - row[d]));
                    float dyz = dz;
#pragma unroll
                    for (int d = DZ; d < DS; ++d) dyz = fmaxf(dyz, fabsf(qc[d] - row[d]));
                    const float *xr = xgf + j * XW;
                    float dx = fabsf(xf[0] - xr[0]);
#pragma unroll
                    for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xf[d] - xr[d]));
                    const bool self = j == qi;
                    const bool pz = dz < ef && !self;
                    cz += pz ? 1 : 0;
                    cyz += (dyz < ef && !self) ? 1 : 0;
                    cxz += (pz && dx < ef) ? 1 : 0;
                }
                cz = __reduce_add_sync(kFull, cz);
                cyz = __reduce_add_sync(kFull, cyz);
                cxz = __reduce_add_sync(kFull, cxz);
                if (lane == f) {
                    nz = cz;
                    nyz = cyz;
                    nxz = cxz;
                }
            }
            if (job_ok) {
                term = a.psi[nz + 1] - a.psi[nxz + 1] - a.psi[nyz + 1];
                const int64_t orig = a.order ? static_cast<int64_t>(a.order[qi]) : qi;
                if (a.eps_out) a.eps_out[static_cast<int64_t>(job) * a.n + orig] = eps;
                if (a.cnt_out) {
                    int32_t *co = a.cnt_out + static_cast<int64_t>(job) * 3 * a.n;
                    co[orig] = nxz;
                    co[a.n + orig] = nyz;
                    co[2 * a.n + orig] = nz;
                }
            }
            const int snz = __reduce_add_sync(kFull, job_ok ? nz : 0);
            const int snyz = __reduce_add_sync(kFull, job_ok ? nyz : 0);
            if (lane == 0) {
                unsigned long long *w = sm.work[warp];
                w[8] += static_cast<unsigned>(snz);
                w[9] += static_cast<unsigned>(snyz);
                w[0] += static_cast<unsigned>(walked_a);
                w[1] += static_cast<unsigned>(walked_b);
                w[2] += static_cast<unsigned long long>(nfa) * static_cast<unsigned long long>(a.n - 1);
                w[3] += static_cast<unsigned long long>(nfb) * static_cast<unsigned long long>(a.n - 1);
                w[4] += nfa + nfb;
                w[6] += tb;
                w[7] += ta;
            }
        }

        // ---------------- the term goes to the tile's slot; the warp that
        // finishes the tile's last query sums it in ksg_fused_kernel's order
        // (NWS sums over the queries m = w, w + NWS, ..., then their sum in
        // order of w), writes the partial and frees the slot.
        double *ring = a.ring + (static_cast<int64_t>(blockIdx.x) * RING + slot) * QC * 32;
        __stcg(ring + m * 32 + lane, term);
        __threadfence_block();
        __syncwarp();
        int prev = 0;
        if (lane == 0) prev = atomicAdd(&sm.done[slot], 1);
        prev = __shfl_sync(kFull, prev, 0);
        if (prev == QC - 1) {
            __threadfence_block();
            const int64_t q0 = static_cast<int64_t>(qt) * QC;
            double s = 0.0;
#pragma unroll 1
            for (int w = 0; w < NWS; ++w) {
                double tsum = 0.0;
                for (int mm = w; mm < QC; mm += NWS) {
                    if (q0 + mm >= a.n) continue;
                    tsum += __ldcg(ring + mm * 32 + lane);
                }
                s += tsum;
            }
            if (job_ok && qt < a.n_qt) a.partial[static_cast<int64_t>(job) * a.n_qt + qt] = s;
            __syncwarp();
            if (lane == 0) {
                sm.done[slot] = 0;
                __threadfence_block();
                *reinterpret_cast<volatile int *>(&sm.owner[slot]) = lt + RING;
            }
        }
    }

    if (lane == 0) sm.work[warp][5] += static_cast<unsigned long long>(clock64() - t_begin);
    __syncthreads();
    if (a.work && tid < kNumWork) {
        unsigned long long s = 0;
        for (int w = 0; w < NW; ++w) s += sm.work[w][tid];
        atomicAdd(&a.work[tid], s);
    }
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
cudaError_t launch_ksg_list(const KsgLaunch &a, int n_groups, cudaStream_t stream)
{
    using LS = ListShape<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    auto kern = ksg_list_kernel<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    // Per device: the dynamic shared memory, a carveout that leaves the rest
    // of the SM's memory to L1, and the SM count (one CTA per SM).
    static DeviceOnce setup;
    static int n_sms[kMaxDevices];
    cudaError_t e = once_per_device(setup, [&](int d) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(LS::SMEM));
        if (r == cudaSuccess) {
            int smem_sm = 0;
            r = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, d);
            if (r == cudaSuccess && smem_sm > 0) {
                const int pct = static_cast<int>((LS::SMEM + 1024) * 100 / smem_sm) + 1;
                r = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         pct < 100 ? pct : 100);
            }
        }
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&n_sms[d], cudaDevAttrMultiProcessorCount, d);
        return r;
    });
    if (e != cudaSuccess) return e;
    const int64_t tiles = static_cast<int64_t>(a.n_qt) * n_groups;
    if (tiles <= 0) return cudaSuccess;  // set-up only
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int chunk_lg = 0;  // the largest chunk (up to IDTX_LIST_CHUNK) giving every SM two chunks
    while ((2 << chunk_lg) <= IDTX_LIST_CHUNK && (tiles >> (chunk_lg + 1)) >= 2 * n_sms[dev])
        ++chunk_lg;
    // every group's query tiles in blocks of 2^chunk_lg (the last block may be short)
    const int64_t chunks = static_cast<int64_t>(n_groups) * ((a.n_qt + (1 << chunk_lg) - 1) >> chunk_lg);
    if (chunks > 0x3fffffff) return cudaErrorInvalidValue;  // the kernel's chunk arithmetic is 32-bit
    int64_t grid = chunks < n_sms[dev] ? chunks : n_sms[dev];
    if (grid > kListRingCtas) grid = kListRingCtas;
    kern<<<static_cast<unsigned>(grid), LS::THREADS, LS::SMEM, stream>>>(
        a, n_groups, static_cast<int>(chunks), chunk_lg);
    return cudaGetLastError();
}

// One compiled specialisation: the tile kernel (ksg_kernel.cuh), its
// persistent form, and the list kernel, all with the same launch shape so
// that their digamma partial sums agree bit for bit; and the plain schedule
// (ksg_plain.cuh) of the same dimension bucket.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
KsgVariant make_variant()
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    return KsgVariant{DX, DY, DZ, K1, EXACT ? 1 : 0, S::GB, S::DSP, S::QC,
                      &launch_ksg<DX, DY, DZ, K1, EXACT, QC, NWARPS>,
                      &launch_ksg_table<DX, DY, DZ, K1, EXACT, QC, NWARPS>,
                      &launch_ksg_list<DX, DY, DZ, K1, EXACT, QC, NWARPS>,
                      &launch_ksg_plain<DX, DY, DZ, K1, EXACT, QC, NWARPS>};
}

}  // namespace idtx
