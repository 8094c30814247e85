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
//   list A: every j != i with d_YZ(i,j) < r_A(i), ascending by (d_YZ, j),
//   list B: every j != i with d_Z(i,j)  < r_B(i), ascending by (d_Z, j),
// at most cap_a / cap_b entries, r_A and r_B chosen so.  Per (query, job):
//   pass A: eps_i = k-th smallest of max(d_X, d_YZ) over j != i.  Walking
//     list A in order, an entry whose d_YZ is at least the current k-th value
//     cannot enter (the joint distance is at least d_YZ), nor can any later
//     one, so the walk stops there.  If the list runs out while the k-th
//     value is still above r_A, an unlisted sample might enter: that job is
//     recomputed by a full scan.
//   pass B: n_yz = #{list A entries with d_YZ < eps} (binary search), n_z and
//     n_xz from a walk over the list B entries with d_Z < eps, using
//     max(d_X, d_Z) < eps <=> d_X < eps and d_Z < eps.  Both are exact when
//     eps <= r_A and eps <= r_B (every sample closer than eps is listed);
//     otherwise the job's counts come from a full scan.
// Every distance is formed from the same fp32 differences and maxima as in
// the definition, so eps and the counts are exact, and the digamma terms are
// summed in the same order as ksg_fused_kernel's: both kernels give
// bit-identical estimates and either may serve a call.
//
// Design (GB300).  A CTA takes QC queries of one group of 32 jobs, one job
// per lane; its warps take queries one at a time from a shared counter.  A
// walk reads its list 32 entries at a time with one coalesced load (the next
// chunk is prefetched), stages them in the warp's shared buffer and consumes
// them in sub-chunks: broadcast 16-byte reads give two entries each, and the
// X values of the 32 jobs at each entry's sample -- one 128-byte row of xi --
// are loaded for the whole sub-chunk back to back, so many gathers are in
// flight per warp.  The walks are warp-uniform (a warp stops when every
// lane's job is done), so lanes never diverge around the loads.  Nothing is staged in shared memory beyond the
// per-query digamma terms, so several CTAs share an SM and its L1 keeps the
// xi rows that neighbouring queries (samples are in Morton order) share.
// There are no waits: every loop is bounded by a list length or by N.
#pragma once

#include "ksg_kernel.cuh"

// List entries per sub-chunk of the neighbour-pass and count-pass walks
// (even divisors of 32; compile-time knobs, the defaults are the tuned values).
#ifndef IDTX_LIST_SA
#define IDTX_LIST_SA 16
#endif
#ifndef IDTX_LIST_SB
#define IDTX_LIST_SB 16
#endif
// Warps per CTA of the list kernel, minimum resident CTAs per SM asked of the
// compiler (0: none), and job groups per block of the launch order (CTAs of
// the same query tile for GBLK consecutive groups run back to back, so a
// query's lists are read from L2 while its groups' X rows stay resident).
#ifndef IDTX_LIST_NW
#define IDTX_LIST_NW 4
#endif
// Jobs of a warp whose count walk goes on past the others' (the largest
// eps) and is finished with the lanes splitting its entries.
#ifndef IDTX_LIST_TAIL
#define IDTX_LIST_TAIL 2
#endif
#ifndef IDTX_LIST_TAIL_A
#define IDTX_LIST_TAIL_A 2
#endif
#ifndef IDTX_LIST_MINB
#define IDTX_LIST_MINB 0
#endif
#ifndef IDTX_LIST_GBLK
#define IDTX_LIST_GBLK 32
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

// QCTA, NWARPS: the tile kernel's launch shape, which fixes the partial-sum
// layout (one partial per QCTA queries) and the order of its sums (NWARPS
// interleaved per-warp sums); LNW: this kernel's own warps per CTA.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS, int LNW>
__device__ __forceinline__ void ksg_list_cta(const KsgLaunch &a, const int qt, const int grp)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QCTA, NWARPS>;
    constexpr int DS = S::DS, DSP = S::DSP, XW = S::XW, GB = S::GB, QC = S::QC;
    constexpr int NWS = S::NW;  // interleaved sums of the tile kernel
    constexpr int NW = LNW;
    constexpr int KH = K1 - 1;  // smallest distances kept (EXACT: exactly k)
    constexpr int kShStage = kTileRows * DSP;
    constexpr unsigned kFull = 0xffffffffu;
    const float kInf = CUDART_INF_F;

    constexpr int SA = IDTX_LIST_SA, SB = IDTX_LIST_SB;  // entries per sub-chunk of the walks
    constexpr int TAIL = IDTX_LIST_TAIL;  // jobs finished after the warp's shared count walk
    constexpr int TAIL_A = IDTX_LIST_TAIL_A;  // and after its shared neighbour walk
    __shared__ double s_term[QC][GB];  // digamma term of (query, job)
    __shared__ double s_red[NWS][GB];
    __shared__ __align__(16) int2 s_ent[NW][32];  // per warp: staged list entries
    __shared__ int s_next;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t q0 = static_cast<int64_t>(qt) * QC;
    const int qv = static_cast<int>(a.n - q0 < QC ? a.n - q0 : QC);
    const int job = grp * GB + lane;
    const bool job_ok = job < a.n_jobs;
    const float *xg = a.xi + static_cast<int64_t>(grp) * a.n_pad * XW + lane * DX;
    int2 *ent = s_ent[warp];
    const int2 sentinel = make_int2(0, __float_as_int(CUDART_INF_F));
    if (qv <= 0) {
        if (tid < GB && job_ok) a.partial[static_cast<int64_t>(job) * a.n_qt + qt] = 0.0;
        return;
    }
    if (tid == 0) s_next = 0;
    __syncthreads();

    const int kk = a.k;
    auto kth = [&](const float(&h)[KH]) { return EXACT ? h[KH - 1] : select_kth<KH>(h, kk - 1); };
    auto sh_row = [&](int64_t j) { return a.sh + (j / kTJ) * kShStage + (j % kTJ) * DSP; };
    auto x_dist = [&](const float(&xq)[DX], int64_t j) {
        const float *xr = xg + j * XW;
        float dx = fabsf(xq[0] - xr[0]);
#pragma unroll
        for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xq[d] - xr[d]));
        return dx;
    };

    unsigned long long walk_a = 0, walk_b = 0, brute_a = 0, brute_b = 0, fallbacks = 0;  // per warp
    unsigned long long tail_b = 0;  // (job, entry) pairs of the count walks' tails
    unsigned long long tail_a = 0;  // (job, entry) pairs of the neighbour walks' tails
    const long long t_begin = clock64();

    while (true) {
        int m = 0;
        if (lane == 0) m = atomicAdd(&s_next, 1);
        m = __shfl_sync(kFull, m, 0);
        if (m >= qv) break;
        const int64_t qi = q0 + m;
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
        // The list is read 32 entries at a time (one coalesced load, the next
        // chunk prefetched), staged in the warp's shared buffer and consumed
        // in sub-chunks of SA entries whose X rows are loaded back to back.
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
                    // Ascending list: once the sub-chunk's first entry is out
                    // of a job's reach, so is everything after it.  When at
                    // most TAIL_A jobs are still in reach the shared walk
                    // stops and those finish lane-split below.
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
                        const int4 p = *reinterpret_cast<const int4 *>(&ent[u + t]);
                        jj[t] = p.x;
                        dyz[t] = __int_as_float(p.y);
                        jj[t + 1] = p.z;
                        dyz[t + 1] = __int_as_float(p.w);
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
        walk_a += walked_a;
        // Lane-split finish of the remaining jobs, one at a time: blocks of 32
        // entries, one per lane; the distances below the job's k-th value are
        // inserted smallest first (warp minimum), until a block starts out
        // of reach.  my_walked: the prefix of list A this lane's job walked.
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
            for (; pos < len_a; pos += 32) {
                // pos is a multiple of 16, so the block may end past the written
                // sentinels: lanes beyond the list take a sentinel
                const int2 en = pos + lane < len_a ? __ldg(la + pos + lane) : sentinel;
                const float dyz = __int_as_float(en.y);
                if (!(__shfl_sync(kFull, dyz, 0) < thf)) break;
                const float *xr = xgf + static_cast<int64_t>(en.x) * XW;
                float dx = fabsf(xf[0] - xr[0]);
#pragma unroll
                for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xf[d] - xr[d]));
                float cand = fmaxf(dx, dyz);
                if (!(cand < thf)) cand = kInf;
                while (true) {
                    const float mn = warp_min(cand);
                    if (!(mn < thf)) break;
                    const uint32_t who = __ballot_sync(kFull, cand == mn);
                    if (lane == __ffs(who) - 1) cand = kInf;
                    if (lane == f) {
                        sorted_insert<KH>(h, mn);
                        th = kth(h);
                    }
                    thf = __shfl_sync(kFull, th, f);
                }
                tail_a += 32;
            }
            if (lane == f) my_walked = pos < len_a ? pos : len_a;
        }
        // The list ran out before the job's k-th distance dropped to r_A:
        // recompute those jobs over every sample.  For each such job the 32
        // lanes split the samples, keep their own k smallest, and the warp
        // merges them (repeatedly taking the smallest head).
        const bool fa = job_ok && th > r_a;
        float eps_fix = 0.0f;
        uint32_t fmask = __ballot_sync(kFull, fa);
        if (fmask) {
            load_q();
            fallbacks += __popc(fmask);
        }
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
                kv = warp_min(hl[0]);
                const uint32_t who = __ballot_sync(kFull, hl[0] == kv);
                if (lane == __ffs(who) - 1) {
#pragma unroll
                    for (int m = 0; m + 1 < KH; ++m) hl[m] = hl[m + 1];
                    hl[KH - 1] = kInf;
                }
            }
            if (lane == f) eps_fix = kv;
            brute_a += a.n - 1;
        }
        const float eps = job_ok ? (fa ? eps_fix : kth(h)) : -1.0f;

        // ---------------- pass B: strict-radius counts
        const bool fb = job_ok && (eps > r_a || eps > r_b);
        int nz = 0, nyz = 0, nxz = 0;
        // Every list A entry below eps lies in the walked prefix (the walk
        // went on until each job's k-th value was at most the next entry).
        if (job_ok && !fb) nyz = list_lower(la, my_walked, eps);
        // The warp walks list B up to the (TAIL+1)-th largest eps of the jobs
        // it serves (ascending, so the walk stops at the first entry at or
        // beyond it); the at most TAIL jobs with a larger eps -- the long
        // tail of the walk -- finish afterwards one at a time, the 32 lanes
        // splitting their remaining entries.  n_z is the number of entries
        // below the job's eps (binary search).
        const float ev = (job_ok && !fb) ? eps : -1.0f;
        float emax;
        {
            float cur = ev;
#pragma unroll 1
            for (int t = 0; t < TAIL; ++t) {
                const float mx = warp_max(cur);
                const uint32_t who = __ballot_sync(kFull, cur == mx);
                if (lane == __ffs(who) - 1) cur = -1.0f;
            }
            emax = warp_max(cur);
        }
        const bool tail = ev > emax;
        int walked_b = 0;
        {
            int2 nxt = len_b > 0 ? __ldg(lb + lane) : sentinel;
            for (int f = 0; f < len_b; f += 32) {
                const int2 cur = nxt;
                if (f + 32 < len_b) nxt = __ldg(lb + f + 32 + lane);
                __syncwarp();
                ent[lane] = cur;
                __syncwarp();
                int u = 0;
                for (; u < 32; u += SB) {
                    if (!(__int_as_float(ent[u].y) < emax)) break;
                    int jj[SB];
                    float dz[SB], dx[SB];
#pragma unroll
                    for (int t = 0; t < SB; t += 2) {
                        const int4 p = *reinterpret_cast<const int4 *>(&ent[u + t]);
                        jj[t] = p.x;
                        dz[t] = __int_as_float(p.y);
                        jj[t + 1] = p.z;
                        dz[t + 1] = __int_as_float(p.w);
                    }
#pragma unroll
                    for (int t = 0; t < SB; ++t) dx[t] = x_dist(xq, jj[t]);
#pragma unroll
                    for (int t = 0; t < SB; ++t) nxz += (dz[t] < eps && dx[t] < eps) ? 1 : 0;
                }
                walked_b = f + u;
                if (u < 32) break;
            }
        }
        if (walked_b > len_b) walked_b = len_b;
        walk_b += walked_b;
        if (job_ok && !fb && !tail) nz = list_lower(lb, walked_b, eps);
        uint32_t tmask = __ballot_sync(kFull, tail);
        while (tmask) {
            const int f = __ffs(tmask) - 1;
            tmask &= tmask - 1;
            const float ef = __shfl_sync(kFull, eps, f);
            float xf[DX];
#pragma unroll
            for (int d = 0; d < DX; ++d) xf[d] = __shfl_sync(kFull, xq[d], f);
            const float *xgf = xg - lane * DX + f * DX;
            // every entry below `end` has d_Z < ef; those before walked_b are counted
            const int end = list_lower(lb, len_b, ef);
            int cnt = 0;
#pragma unroll 4
            for (int e = walked_b + lane; e < end; e += 32) {
                const int j = __ldg(&lb[e].x);
                const float *xr = xgf + static_cast<int64_t>(j) * XW;
                float dx = fabsf(xf[0] - xr[0]);
#pragma unroll
                for (int d = 1; d < DX; ++d) dx = fmaxf(dx, fabsf(xf[d] - xr[d]));
                cnt += dx < ef ? 1 : 0;
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(kFull, cnt, off);
            if (lane == f) {
                nxz += cnt;
                nz = end;
            }
            tail_b += end > walked_b ? end - walked_b : 0;
        }
        // Jobs whose eps reaches past a list: counts by a full scan, the 32
        // lanes splitting the samples of one such job at a time.
        uint32_t bmask = __ballot_sync(kFull, fb);
        if (bmask) {
            load_q();
            fallbacks += __popc(bmask);
        }
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
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                cz += __shfl_xor_sync(kFull, cz, off);
                cyz += __shfl_xor_sync(kFull, cyz, off);
                cxz += __shfl_xor_sync(kFull, cxz, off);
            }
            if (lane == f) {
                nz = cz;
                nyz = cyz;
                nxz = cxz;
            }
            brute_b += a.n - 1;
        }
        if (job_ok) {
            s_term[m][lane] = a.psi[nz + 1] - a.psi[nxz + 1] - a.psi[nyz + 1];
            const int64_t orig = a.order ? static_cast<int64_t>(a.order[qi]) : qi;
            if (a.eps_out) a.eps_out[static_cast<int64_t>(job) * a.n + orig] = eps;
            if (a.cnt_out) {
                int32_t *co = a.cnt_out + static_cast<int64_t>(job) * 3 * a.n;
                co[orig] = nxz;
                co[a.n + orig] = nyz;
                co[2 * a.n + orig] = nz;
            }
        }
    }
    __syncthreads();

    // ---------------- digamma sums in ksg_fused_kernel's order: NWS sums
    // over the queries m = w, w + NWS, ..., then their sum in order of w
    for (int w = warp; w < NWS; w += NW) {
        double tsum = 0.0;
        for (int m = w; m < QC; m += NWS) {
            const int64_t qi = q0 + m;
            if (qi >= a.n || !job_ok) continue;
            tsum += s_term[m][lane];
        }
        s_red[w][lane] = tsum;
    }
    if (a.work && lane == 0) {
        atomicAdd(&a.work[0], walk_a);
        atomicAdd(&a.work[1], walk_b);
        atomicAdd(&a.work[2], brute_a);
        atomicAdd(&a.work[3], brute_b);
        atomicAdd(&a.work[4], fallbacks);
        atomicAdd(&a.work[6], tail_b);
        atomicAdd(&a.work[7], tail_a);
        atomicAdd(&a.work[5], static_cast<unsigned long long>(clock64() - t_begin));
    }
    __syncthreads();
    if (tid < GB && job_ok) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NWS; ++w) s += s_red[w][tid];
        a.partial[static_cast<int64_t>(job) * a.n_qt + qt] = s;
    }
}

// Block b of the launch order: blocks of GBLK job groups; within a block the
// CTAs of one query tile for its groups are consecutive.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QCTA, int NWARPS, int LNW>
__global__ void __launch_bounds__(LNW * 32, IDTX_LIST_MINB)
    ksg_list_kernel(const KsgLaunch a, const int n_groups)
{
    const int64_t id = blockIdx.x;
    const int64_t per_blk = static_cast<int64_t>(a.n_qt) * IDTX_LIST_GBLK;
    const int gb = static_cast<int>(id / per_blk);
    const int64_t rem = id - gb * per_blk;
    const int left = n_groups - gb * IDTX_LIST_GBLK;
    const int gcount = left < IDTX_LIST_GBLK ? left : IDTX_LIST_GBLK;
    const int qt = static_cast<int>(rem / gcount);
    const int grp = gb * IDTX_LIST_GBLK + static_cast<int>(rem - static_cast<int64_t>(qt) * gcount);
    ksg_list_cta<DX, DY, DZ, K1, EXACT, QCTA, NWARPS, LNW>(a, qt, grp);
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
cudaError_t launch_ksg_list(const KsgLaunch &a, int n_groups, cudaStream_t stream)
{
    constexpr int LNW = IDTX_LIST_NW;
    const int64_t blocks = static_cast<int64_t>(a.n_qt) * n_groups;
    if (blocks <= 0) return cudaSuccess;
    ksg_list_kernel<DX, DY, DZ, K1, EXACT, QC, NWARPS, LNW>
        <<<static_cast<unsigned>(blocks), LNW * 32, 0, stream>>>(a, n_groups);
    return cudaGetLastError();
}

// One compiled specialisation: the tile kernel (ksg_kernel.cuh), its
// persistent form, and the list kernel, all with the same launch shape so
// that their digamma partial sums agree bit for bit.
template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
KsgVariant make_variant()
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    return KsgVariant{DX, DY, DZ, K1, EXACT ? 1 : 0, S::GB, S::DSP, S::QC,
                      &launch_ksg<DX, DY, DZ, K1, EXACT, QC, NWARPS>,
                      &launch_ksg_table<DX, DY, DZ, K1, EXACT, QC, NWARPS>,
                      &launch_ksg_list<DX, DY, DZ, K1, EXACT, QC, NWARPS>};
}

}  // namespace idtx
