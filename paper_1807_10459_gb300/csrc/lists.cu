// lists.cu -- per-query sorted neighbour lists in the shared (Y,Z) and Z
// subspaces, the preparation step of ksg_list_kernel (ksg_list.cuh).
//
// For every query i (sorted sample position) and every other sample j, the
// max-norm distances d_Z(i,j) over the z columns and d_YZ(i,j) over the z and
// y columns of sh are formed exactly as in the estimator's definition (fp32
// |a-b| and maxima).  List A holds every j != i with d_YZ < r_A(i), list B
// every j != i with d_Z < r_B(i), each ascending by (distance, j); r_A, r_B
// are the largest histogram-bin edges for which the lists fit their
// capacities (+inf when every sample fits).
#include <cuda_runtime.h>

#include <cstdint>

#include "ksg_common.cuh"

namespace idtx {

namespace {

constexpr int kLThreads = 256;
constexpr int kBins = 4096;          // bins on bits 30..19 of a non-negative float
constexpr int kBinShift = 19;
constexpr int kBinsPerThread = kBins / kLThreads;

__device__ __forceinline__ void dists(const float *q, const float *row, int dzb, int dsb,
                                      float &dz, float &dyz)
{
    float m = 0.0f;
    for (int d = 0; d < dzb; ++d) m = fmaxf(m, fabsf(q[d] - row[d]));
    dz = m;
    for (int d = dzb; d < dsb; ++d) m = fmaxf(m, fabsf(q[d] - row[d]));
    dyz = m;
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

// Ascending bitonic sort of keys[0..p), p a power of two.
__device__ void bitonic_sort(unsigned long long *keys, int p)
{
    for (int size = 2; size <= p; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (p >> 1); t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const unsigned long long x = keys[lo], y = keys[hi];
                if ((x > y) == asc) {
                    keys[lo] = y;
                    keys[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int pow2_at_least(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// One block per query.  Dynamic shared memory: max(2 * kBins ints,
// (pow2(cap_a) + pow2(cap_b)) keys); the key arrays reuse the histograms.
__global__ void __launch_bounds__(kLThreads)
    k_build_lists(const float *sh, int dsp, int dzb, int dsb, int64_t n, int cap_a, int cap_b,
                  int2 *list_a, int2 *list_b, int4 *meta)
{
    extern __shared__ __align__(16) unsigned char l_smem[];
    __shared__ float s_q[32];
    __shared__ int s_part[kLThreads / 32];
    __shared__ int s_cut;
    __shared__ int s_cnt[2];
    int *hist_a = reinterpret_cast<int *>(l_smem);
    int *hist_b = hist_a + kBins;
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x;
    auto row_of = [&](int64_t j) { return sh + ((j / kTJ) * kTileRows + (j % kTJ)) * dsp; };

    if (tid < dsb) s_q[tid] = row_of(i)[tid];
    for (int b = tid; b < 2 * kBins; b += kLThreads) hist_a[b] = 0;
    __syncthreads();
    for (int64_t j = tid; j < n; j += kLThreads) {
        if (j == i) continue;
        float dz, dyz;
        dists(s_q, row_of(j), dzb, dsb, dz, dyz);
        atomicAdd(&hist_a[__float_as_uint(dyz) >> kBinShift], 1);
        atomicAdd(&hist_b[__float_as_uint(dz) >> kBinShift], 1);
    }
    __syncthreads();
    const int cut_a = cut_bin(hist_a, cap_a, s_part, &s_cut);
    const int cut_b = cut_bin(hist_b, cap_b, s_part, &s_cut);
    const float r_a = cut_a >= kBins ? INFINITY : __uint_as_float((unsigned)cut_a << kBinShift);
    const float r_b = cut_b >= kBins ? INFINITY : __uint_as_float((unsigned)cut_b << kBinShift);

    // Collect the samples below the cuts (order of arrival), then sort.
    const int pa = pow2_at_least(cap_a);
    unsigned long long *keys_a = reinterpret_cast<unsigned long long *>(l_smem);
    unsigned long long *keys_b = keys_a + pa;
    if (tid < 2) s_cnt[tid] = 0;
    __syncthreads();  // histograms are dead from here on
    for (int64_t j = tid; j < n; j += kLThreads) {
        if (j == i) continue;
        float dz, dyz;
        dists(s_q, row_of(j), dzb, dsb, dz, dyz);
        if (dyz < r_a) {
            const int at = atomicAdd(&s_cnt[0], 1);
            if (at < cap_a) keys_a[at] = ((unsigned long long)__float_as_uint(dyz) << 32) | (uint32_t)j;
        }
        if (dz < r_b) {
            const int at = atomicAdd(&s_cnt[1], 1);
            if (at < cap_b) keys_b[at] = ((unsigned long long)__float_as_uint(dz) << 32) | (uint32_t)j;
        }
    }
    __syncthreads();
    const int na = min(s_cnt[0], cap_a), nb = min(s_cnt[1], cap_b);
    const int p_a = pow2_at_least(max(na, 1)), p_b = pow2_at_least(max(nb, 1));
    for (int t = na + tid; t < p_a; t += kLThreads) keys_a[t] = ~0ull;
    for (int t = nb + tid; t < p_b; t += kLThreads) keys_b[t] = ~0ull;
    __syncthreads();
    bitonic_sort(keys_a, p_a);
    bitonic_sort(keys_b, p_b);

    // Entries, then +inf sentinels up to a multiple of 32 (the walks read 32
    // entries at a time; capacities are multiples of 32).
    const int2 sentinel = make_int2(0, __float_as_int(INFINITY));
    int2 *la = list_a + i * cap_a;
    int2 *lb = list_b + i * cap_b;
    const int end_a = min(cap_a, (na + 31) & ~31), end_b = min(cap_b, (nb + 31) & ~31);
    for (int t = tid; t < end_a; t += kLThreads)
        la[t] = t < na ? make_int2((int)(uint32_t)keys_a[t], (int)(keys_a[t] >> 32)) : sentinel;
    for (int t = tid; t < end_b; t += kLThreads)
        lb[t] = t < nb ? make_int2((int)(uint32_t)keys_b[t], (int)(keys_b[t] >> 32)) : sentinel;
    if (tid == 0)
        meta[i] = make_int4(na, nb, __float_as_int(r_a), __float_as_int(r_b));
}

}  // namespace

size_t list_smem_bytes(int cap_a, int cap_b)
{
    auto p2 = [](int v) {
        int p = 1;
        while (p < v) p <<= 1;
        return p;
    };
    const size_t keys = (size_t)(p2(cap_a) + p2(cap_b)) * sizeof(unsigned long long);
    const size_t hist = 2 * (size_t)kBins * sizeof(int);
    return keys > hist ? keys : hist;
}

cudaError_t build_lists(const float *sh, int dsp, int dzb, int dsb, int64_t n, int cap_a,
                        int cap_b, int2 *list_a, int2 *list_b, int4 *meta, cudaStream_t st)
{
    static bool attr_set = false;  // per process; the attribute is per function
    const size_t smem = list_smem_bytes(kMaxListA, kMaxListB);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_build_lists,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (n <= 0) return cudaSuccess;
    k_build_lists<<<(unsigned)n, kLThreads, list_smem_bytes(cap_a, cap_b), st>>>(
        sh, dsp, dzb, dsb, n, cap_a, cap_b, list_a, list_b, meta);
    return cudaGetLastError();
}

}  // namespace idtx
