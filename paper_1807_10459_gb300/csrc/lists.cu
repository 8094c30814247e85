// lists.cu -- per-query sorted neighbour lists in the shared (Y,Z) and Z
// subspaces, the preparation step of ksg_list_kernel (ksg_list.cuh).
//
// For every query i (sorted sample position) and every other sample j that
// may belong to a list (whole tiles that cannot are skipped: see the
// kernel), the max-norm distances d_Z(i,j) over the z columns and d_YZ(i,j)
// over the z and y columns of sh are formed exactly as in the estimator's
// definition (fp32 |a-b| and maxima).  List A holds every j != i with
// d_YZ < r_A(i), list B every j != i with d_Z < r_B(i), each ascending by
// distance (equal distances in any order); r_A, r_B are the largest
// histogram-bin edges for which the lists fit their capacities (+inf when
// every sample fits).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include <cub/block/block_radix_sort.cuh>

#include "ksg_common.cuh"

namespace idtx {

namespace {

constexpr int kLThreads = 256;
constexpr int kBins = 4096;          // bins on bits 30..19 of a non-negative float
constexpr int kBinShift = 19;
constexpr int kBinsPerThread = kBins / kLThreads;

// Digit width of the block radix sorts: 7 passes over a 32-bit key instead
// of CUB's default 8 (measured on GB300: 1.82 against 1.97 ms for 9995
// queries, lists of 2048 and 4096; 6 bits spills).
constexpr int kSortRadixBits = 5;

// Largest tile-visit bitmap (32-bit words): calls with more tiles visit all.
constexpr int kMaxVisitWords = 1024;
// Tile pruning runs for calls of at least kPruneMinTiles tiles whose lists
// hold at most an eighth of the samples: otherwise its per-query set-up (two
// histogram clears, bounds of every tile, two ranking scans) costs more than
// it saves (measured on GB300: N = 1000 lost 7 %; the greedy step's build,
// N = 9995 with lists of 2048 and 4096, 0.15 ms; N = 99850 with lists of
// 512 and 1024 was built 1.8x faster).
constexpr int kPruneMinTiles = 64;
constexpr int kPruneMaxListShare = 8;  // lists of at most n / 8 entries

constexpr int kMaxRow4 = 5;  // float4 columns of a row of sh: dsp <= 20 (dz' <= 16, dy <= 4)
constexpr int kUnrollJ = 4;  // samples a thread has in flight per step of a distance pass

// Fold float4 column c of a row into the running maxima of d_Z (the first
// dzb columns) and d_YZ (the first dsb): the estimator's fp32 |a-b| and maxima.
__device__ __forceinline__ void fold4(const float4 q, const float4 r, int c, int dzb, int dsb,
                                      float &mz, float &my)
{
    const float a[4] = {fabsf(q.x - r.x), fabsf(q.y - r.y), fabsf(q.z - r.z), fabsf(q.w - r.w)};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int d = 4 * c + e;
        if (d < dzb) mz = fmaxf(mz, a[e]);
        if (d < dsb) my = fmaxf(my, a[e]);
    }
}

// First bin b with (count of bins <= b) > cap, or kBins if the total fits.
// All threads of the block call it; the result is returned to every thread.
__device__ int cut_bin(const int *hist, int cap, int *s_part, int *s_cut)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int local = 0;
    for (int b = 0; b < kBinsPerThread; ++b) local += hist[tid * kBinsPerThread + b];
    // inclusive scan over threads
    int inc = local;
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += v;
    }
    if (lane == 31) s_part[warp] = inc;
    if (tid == 0) *s_cut = kBins;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += s_part[w];
    int cum = before + inc - local;  // count in bins before this thread's range
    if (cum <= cap && cum + local > cap) {
        for (int b = 0; b < kBinsPerThread; ++b) {
            cum += hist[tid * kBinsPerThread + b];
            if (cum > cap) {
                *s_cut = tid * kBinsPerThread + b;
                break;
            }
        }
    }
    __syncthreads();
    const int r = *s_cut;
    __syncthreads();
    return r;
}

// Sort the n collected (distance bits, sample) pairs of one list ascending by
// distance and write them, then +inf sentinels up to a multiple of 32 (at
// most cap), to out.  Ties may land in any order: nothing downstream depends
// on the order of equal distances.  Every key is below `bound` (the bits of
// the list's cut, a non-negative float), so only its low 32 - clz(bound)
// bits can differ and the sort passes over those alone; the padding keys
// (all ones) stay above every real key in those bits.  The pairs are first
// taken into registers, so the sort's scratch may overlay the collection
// buffers (tmp); all threads of the block call it.
template <int ITEMS>
__device__ void sort_and_store(const uint32_t *keys, const int32_t *vals, int n, int cap,
                               uint32_t bound, void *tmp, int2 *out)
{
    using Sort = cub::BlockRadixSort<uint32_t, kLThreads, ITEMS, int32_t, kSortRadixBits>;
    uint32_t k[ITEMS];
    int32_t v[ITEMS];
    const int t0 = threadIdx.x * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int at = t0 + i;
        k[i] = at < n ? keys[at] : 0xFFFFFFFFu;
        v[i] = at < n ? vals[at] : 0;
    }
    __syncthreads();  // the collection buffers may now be overwritten
    const int end_bit = max(1, 32 - __clz(bound));
    Sort(*reinterpret_cast<typename Sort::TempStorage *>(tmp)).Sort(k, v, 0, end_bit);
    const int end = min(cap, (n + 31) & ~31);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int at = t0 + i;
        if (at < end)
            out[at] = at < n ? make_int2(v[i], (int)k[i]) : make_int2(0, __float_as_int(INFINITY));
    }
    __syncthreads();
}

template <int ITEMS>
constexpr size_t sort_tmp_bytes()
{
    return sizeof(typename cub::BlockRadixSort<uint32_t, kLThreads, ITEMS, int32_t, kSortRadixBits>::TempStorage);
}

// One block per query.  Dynamic shared memory: the two histograms, later
// overlaid by the collected keys and samples of both lists, later by the
// sort's scratch (build_smem bytes), then at visit_off the tile-visit bitmap
// and its per-word prefix counts.
// IA, IB: sort items per thread (kLThreads * IA >= cap_a, kLThreads * IB >=
// cap_b).
//
// Tile pruning.  Rows kTJ and kTJ+1 of every tile of sh hold its samples'
// per-dimension minimum and maximum.  For the query, a tile's box gap G (the
// largest over dimensions of the distance from the query to the box, 0
// inside) bounds its samples' distances from below and its far corner F
// (the largest over dimensions of the query's distance to the farther face)
// from above, in the subspaces Z and (Y,Z), both in the definition's fp32
// arithmetic (rounding is monotone, so the bounds hold for the computed
// distances).  Summing tile sizes by F gives a radius R within which more
// than cap samples lie: the list's cut is at most R, so the histogram pass
// needs only the tiles with G < R (it is exact below R).  The collecting
// pass needs only the tiles with G below the cut.
template <int IA, int IB>
__global__ void __launch_bounds__(kLThreads, 3)
    k_build_lists(const float *sh, int dsp, int dzb, int dsb, int64_t n, int cap_a, int cap_b,
                  int2 *list_a, int2 *list_b, int4 *meta, int visit_off)
{
    extern __shared__ __align__(16) unsigned char l_smem[];
    __shared__ int s_part[kLThreads / 32];
    __shared__ int s_cut;
    __shared__ int s_cnt[2];
    __shared__ int s_nvis;
    int *hist_a = reinterpret_cast<int *>(l_smem);
    int *hist_b = hist_a + kBins;
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x;
    const int nc = dsp / 4;  // float4 columns per row
    auto row4 = [&](int64_t j) {
        return reinterpret_cast<const float4 *>(sh + ((j / kTJ) * kTileRows + (j % kTJ)) * dsp);
    };
    float4 q4[kMaxRow4];
    {
        const float4 *qr = row4(i);
#pragma unroll
        for (int c = 0; c < kMaxRow4; ++c) q4[c] = c < nc ? qr[c] : make_float4(0, 0, 0, 0);
    }
    const int warp = tid >> 5;
    const int n_tiles = (int)((n + kTJ - 1) / kTJ);
    const int vwords = (n_tiles + 31) / 32;
    const bool prune = vwords <= kMaxVisitWords && n_tiles >= kPruneMinTiles &&
                       (int64_t)max(cap_a, cap_b) * kPruneMaxListShare <= n;
    uint32_t *visit = reinterpret_cast<uint32_t *>(l_smem + visit_off);
    // Box gap and far-corner bounds of tile t in Z and (Y,Z).
    auto tile_bounds = [&](int t, float &gz, float &gyz, float &fz, float &fyz) {
        const float4 *lo = reinterpret_cast<const float4 *>(sh + ((int64_t)t * kTileRows + kTJ) * dsp);
        const float4 *hi = lo + nc;
        gz = gyz = fz = fyz = 0.0f;
#pragma unroll
        for (int c = 0; c < kMaxRow4; ++c) {
            if (c < nc) {
                const float4 a4 = lo[c], b4 = hi[c], q = q4[c];
                const float qa[4] = {q.x, q.y, q.z, q.w}, la[4] = {a4.x, a4.y, a4.z, a4.w},
                            ha[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int d = 4 * c + e;
                    const float g = fmaxf(fmaxf(la[e] - qa[e], qa[e] - ha[e]), 0.0f);
                    const float f = fmaxf(fabsf(qa[e] - la[e]), fabsf(qa[e] - ha[e]));
                    if (d < dzb) {
                        gz = fmaxf(gz, g);
                        fz = fmaxf(fz, f);
                    }
                    if (d < dsb) {
                        gyz = fmaxf(gyz, g);
                        fyz = fmaxf(fyz, f);
                    }
                }
            }
        }
    };
    // Bit t of the visit bitmap: tile t has G < lim in either subspace.
    auto mark_tiles = [&](float lim_a, float lim_b) {
        for (int w = warp; w < vwords; w += kLThreads / 32) {
            const int t = w * 32 + (tid & 31);
            bool vis = false;
            if (t < n_tiles) {
                float gz, gyz, fz, fyz;
                tile_bounds(t, gz, gyz, fz, fyz);
                vis = gyz < lim_a || gz < lim_b;
            }
            const uint32_t bits = __ballot_sync(0xffffffffu, vis);
            if ((tid & 31) == 0) visit[w] = bits;
        }
    };
    // The visited tiles are taken by the warps in turn (the visited tile of
    // rank k by warp k mod 8); vpre[w] counts the visited tiles in the
    // bitmap's words before w.
    int *vpre = reinterpret_cast<int *>(visit + vwords);
    auto rank_tiles = [&]() {  // all threads; the bitmap written and synced before
        if (warp == 0) {
            const int lane = tid & 31;
            const int per = (vwords + 31) / 32;
            const int w0 = lane * per, w1 = min(w0 + per, vwords);
            int sum = 0;
            for (int w = w0; w < w1; ++w) sum += __popc(visit[w]);
            int inc = sum;
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += v;
            }
            int run = inc - sum;
            for (int w = w0; w < w1; ++w) {
                vpre[w] = run;
                run += __popc(visit[w]);
            }
            if (lane == 31) s_nvis = inc;
        }
        __syncthreads();
    };
    // The tile of rank k (all tiles in order when not pruning); wp: the
    // bitmap word to search from (a warp's ranks only grow).
    auto tile_of = [&](int k, int &wp) -> int {
        if (!prune) return k;
        while (wp + 1 < vwords && vpre[wp + 1] <= k) ++wp;
        return wp * 32 + (int)__fns(visit[wp], 0, k - vpre[wp] + 1);
    };
    constexpr int kSegs = kTJ / 32;  // 32-sample segments per tile
    // Distances of samples j[u] = tile t's segment s0 + u, this lane's
    // sample (kUnrollJ segments, their rows loaded back to back); the query
    // itself and samples past the tile or n get +inf (and read the query's
    // own row, an L1 hit).
    auto dists_tile = [&](int t, int s0, int64_t (&j)[kUnrollJ], float (&dz)[kUnrollJ],
                          float (&dyz)[kUnrollJ]) {
        const float4 *r[kUnrollJ];
        bool ok[kUnrollJ];
#pragma unroll
        for (int u = 0; u < kUnrollJ; ++u) {
            j[u] = (int64_t)t * kTJ + (s0 + u) * 32 + (tid & 31);
            ok[u] = s0 + u < kSegs && j[u] < n && j[u] != i;
            r[u] = row4(ok[u] ? j[u] : i);
            dz[u] = dyz[u] = 0.0f;
        }
#pragma unroll
        for (int c = 0; c < kMaxRow4; ++c) {
            if (c < nc) {
                float4 v[kUnrollJ];
#pragma unroll
                for (int u = 0; u < kUnrollJ; ++u) v[u] = r[u][c];
#pragma unroll
                for (int u = 0; u < kUnrollJ; ++u) fold4(q4[c], v[u], c, dzb, dsb, dz[u], dyz[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnrollJ; ++u)
            if (!ok[u]) dz[u] = dyz[u] = INFINITY;
    };
    constexpr int kWarps = kLThreads / 32;

    // The radii R: tile sizes summed into the histograms by far corner.
    // Bins hold bits 30..19 of a non-negative float, so the upper edge of
    // bin b is the float with bits (b + 1) << 19; from bin 4079 on that is
    // +inf or past it.
    auto upper_edge = [](int b) {
        return b + 1 >= (0x7F800000 >> kBinShift) ? INFINITY : __uint_as_float((unsigned)(b + 1) << kBinShift);
    };
    if (prune) {
        for (int b = tid; b < 2 * kBins; b += kLThreads) hist_a[b] = 0;
        __syncthreads();
        for (int t = tid; t < n_tiles; t += kLThreads) {
            float gz, gyz, fz, fyz;
            tile_bounds(t, gz, gyz, fz, fyz);
            const int64_t left = n - (int64_t)t * kTJ;
            const int size = left < kTJ ? (int)left : kTJ;
            atomicAdd(&hist_a[__float_as_uint(fyz) >> kBinShift], size);
            atomicAdd(&hist_b[__float_as_uint(fz) >> kBinShift], size);
        }
        __syncthreads();
        // more than cap + 1 samples (the query among them) within the bin's upper edge
        const int fa = cut_bin(hist_a, cap_a + 1, s_part, &s_cut);
        const int fb = cut_bin(hist_b, cap_b + 1, s_part, &s_cut);
        mark_tiles(fa >= kBins ? INFINITY : upper_edge(fa), fb >= kBins ? INFINITY : upper_edge(fb));
    }
    for (int b = tid; b < 2 * kBins; b += kLThreads) hist_a[b] = 0;
    __syncthreads();
    if (prune) rank_tiles();
    {
        const int n_iter = prune ? s_nvis : n_tiles;
        int wp = 0;
        for (int k = warp; k < n_iter; k += kWarps) {
            const int t = tile_of(k, wp);
            for (int s0 = 0; s0 < kSegs; s0 += kUnrollJ) {
                int64_t j[kUnrollJ];
                float dz[kUnrollJ], dyz[kUnrollJ];
                dists_tile(t, s0, j, dz, dyz);
#pragma unroll
                for (int u = 0; u < kUnrollJ; ++u) {
                    if (dz[u] == INFINITY) continue;  // the query itself or past n
                    atomicAdd(&hist_a[__float_as_uint(dyz[u]) >> kBinShift], 1);
                    atomicAdd(&hist_b[__float_as_uint(dz[u]) >> kBinShift], 1);
                }
            }
        }
    }
    __syncthreads();
    const int cut_a = cut_bin(hist_a, cap_a, s_part, &s_cut);
    const int cut_b = cut_bin(hist_b, cap_b, s_part, &s_cut);
    const float r_a = cut_a >= kBins ? INFINITY : __uint_as_float((unsigned)cut_a << kBinShift);
    const float r_b = cut_b >= kBins ? INFINITY : __uint_as_float((unsigned)cut_b << kBinShift);
    if (prune) {
        mark_tiles(r_a, r_b);  // the histogram pass is done with the bitmap (cut_bin syncs)
        __syncthreads();
        rank_tiles();
    }

    // Collect the samples below the cuts (in order of arrival; a warp claims
    // the slots of all its qualifying lanes with one atomic per list).
    uint32_t *key_a = reinterpret_cast<uint32_t *>(l_smem);
    int32_t *val_a = reinterpret_cast<int32_t *>(key_a + kLThreads * IA);
    uint32_t *key_b = reinterpret_cast<uint32_t *>(val_a + kLThreads * IA);
    int32_t *val_b = reinterpret_cast<int32_t *>(key_b + kLThreads * IB);
    if (tid < 2) s_cnt[tid] = 0;
    __syncthreads();  // histograms are dead from here on
    const int lane = tid & 31;
    const uint32_t below = (1u << lane) - 1u;
    {
        const int n_iter = prune ? s_nvis : n_tiles;
        int wp = 0;
        for (int k = warp; k < n_iter; k += kWarps) {  // whole warps iterate
            const int t = tile_of(k, wp);
            for (int s0 = 0; s0 < kSegs; s0 += kUnrollJ) {
                int64_t j[kUnrollJ];
                float dz[kUnrollJ], dyz[kUnrollJ];
                dists_tile(t, s0, j, dz, dyz);
#pragma unroll
                for (int u = 0; u < kUnrollJ; ++u) {
                    const bool in_a = dyz[u] < r_a, in_b = dz[u] < r_b;
                    const uint32_t ma = __ballot_sync(0xffffffffu, in_a);
                    const uint32_t mb = __ballot_sync(0xffffffffu, in_b);
                    int base_a = 0, base_b = 0;
                    if (lane == 0) {
                        if (ma) base_a = atomicAdd(&s_cnt[0], __popc(ma));
                        if (mb) base_b = atomicAdd(&s_cnt[1], __popc(mb));
                    }
                    base_a = __shfl_sync(0xffffffffu, base_a, 0);
                    base_b = __shfl_sync(0xffffffffu, base_b, 0);
                    if (in_a) {
                        const int at = base_a + __popc(ma & below);
                        if (at < cap_a) {
                            key_a[at] = __float_as_uint(dyz[u]);
                            val_a[at] = (int32_t)j[u];
                        }
                    }
                    if (in_b) {
                        const int at = base_b + __popc(mb & below);
                        if (at < cap_b) {
                            key_b[at] = __float_as_uint(dz[u]);
                            val_b[at] = (int32_t)j[u];
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    const int na = min(s_cnt[0], cap_a), nb = min(s_cnt[1], cap_b);
    // List B first: its pairs go to registers, then its scratch overlays
    // list B's buffers (list A's stay intact below them).
    sort_and_store<IB>(key_b, val_b, nb, cap_b, __float_as_uint(r_b), key_b, list_b + i * cap_b);
    sort_and_store<IA>(key_a, val_a, na, cap_a, __float_as_uint(r_a), key_a, list_a + i * cap_a);
    if (tid == 0) meta[i] = make_int4(na, nb, __float_as_int(r_a), __float_as_int(r_b));
}

// Items per thread covering a capacity (a power of two, at least 1).
int items_for(int cap)
{
    int it = 1;
    while (it * kLThreads < cap) it <<= 1;
    return it;
}

// Shared memory of k_build_lists<ia, ib>: the histograms, or the collected
// pairs of both lists, or list A's pairs plus list B's sort scratch,
// whichever is largest.
size_t build_smem(int ia, int ib, size_t tmp_b, size_t tmp_a)
{
    const size_t hist = 2 * (size_t)kBins * sizeof(int);
    const size_t pairs_a = (size_t)kLThreads * ia * 8, pairs_b = (size_t)kLThreads * ib * 8;
    size_t m = hist;
    m = std::max(m, pairs_a + pairs_b);
    m = std::max(m, pairs_a + tmp_b);
    m = std::max(m, tmp_a);
    return (m + 15) & ~size_t(15);
}

template <int IA, int IB>
cudaError_t launch_build(const float *sh, int dsp, int dzb, int dsb, int64_t n, int cap_a,
                         int cap_b, int2 *list_a, int2 *list_b, int4 *meta, cudaStream_t st)
{
    static DeviceOnce attr;  // the attribute is per function and device
    const size_t main = build_smem(IA, IB, sort_tmp_bytes<IB>(), sort_tmp_bytes<IA>());
    cudaError_t e = once_per_device(attr, [&](int) {
        return cudaFuncSetAttribute(k_build_lists<IA, IB>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(main + 2 * kMaxVisitWords * sizeof(uint32_t)));
    });
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    const int64_t vwords = ((n + kTJ - 1) / kTJ + 31) / 32;
    const size_t smem =
        main + (vwords <= kMaxVisitWords ? 2 * (size_t)vwords * sizeof(uint32_t) : 0);
    k_build_lists<IA, IB><<<(unsigned)n, kLThreads, smem, st>>>(
        sh, dsp, dzb, dsb, n, cap_a, cap_b, list_a, list_b, meta, (int)main);
    return cudaGetLastError();
}

}  // namespace

cudaError_t build_lists(const float *sh, int dsp, int dzb, int dsb, int64_t n, int cap_a,
                        int cap_b, int2 *list_a, int2 *list_b, int4 *meta, cudaStream_t st)
{
    // One instantiation per size class s: list A up to 128 s entries, list B
    // up to 256 s (s = 2, 4, 8, 16).
    int s = std::max(items_for(cap_b), 2 * items_for(cap_a));
    s = std::max(s, 2);
    if (n <= 0) {  // set-up only: every instantiation's attribute (outside captures)
        cudaError_t e = launch_build<1, 2>(sh, dsp, dzb, dsb, 0, 0, 0, nullptr, nullptr, nullptr, st);
        if (e == cudaSuccess) e = launch_build<2, 4>(sh, dsp, dzb, dsb, 0, 0, 0, nullptr, nullptr, nullptr, st);
        if (e == cudaSuccess) e = launch_build<4, 8>(sh, dsp, dzb, dsb, 0, 0, 0, nullptr, nullptr, nullptr, st);
        if (e == cudaSuccess) e = launch_build<8, 16>(sh, dsp, dzb, dsb, 0, 0, 0, nullptr, nullptr, nullptr, st);
        return e;
    }
    switch (s) {
    case 2:
        return launch_build<1, 2>(sh, dsp, dzb, dsb, n, cap_a, cap_b, list_a, list_b, meta, st);
    case 4:
        return launch_build<2, 4>(sh, dsp, dzb, dsb, n, cap_a, cap_b, list_a, list_b, meta, st);
    case 8:
        return launch_build<4, 8>(sh, dsp, dzb, dsb, n, cap_a, cap_b, list_a, list_b, meta, st);
    default:
        return launch_build<8, 16>(sh, dsp, dzb, dsb, n, cap_a, cap_b, list_a, list_b, meta, st);
    }
}

}  // namespace idtx
