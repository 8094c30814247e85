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
// Design (GB300, one CTA = 128 queries x GB jobs, one query per thread):
//   * All jobs of a group share Y and Z (a surrogate only permutes X, and the
//     candidates of one greedy step differ only in X).  The Y/Z distance of a
//     (query, reference) pair is computed once per thread and reused by the GB
//     jobs the thread holds in registers.
//   * Pass A keeps, per job, the k+1 smallest joint distances in a sorted
//     register array.  The sample itself is never skipped: its own distance 0
//     occupies one slot, so the (k+1)-th smallest including it is the k-th
//     smallest over j != i.  A job can only change when the shared distance is
//     below the largest current k-th distance of the thread's jobs, so the
//     per-job work runs behind one compare on that bound.
//   * Pass B counts with the same tiles; the pair (i,i) is counted when
//     eps_i > 0 and is subtracted at the end.  The per-job work runs only when
//     the Z distance is below the largest eps of the thread's jobs, because
//     every counted pair has d_Z < eps.
//   * Reference tiles (128 samples of sh and of xi) are staged into shared
//     memory by 1-D TMA bulk copies (cp.async.bulk) completing on an mbarrier,
//     double-buffered; both passes stream the same tiles.  Every mbarrier
//     wait is bounded by %globaltimer; on expiry the CTA records kErrTimeout,
//     waits (bounded) for its own copies in flight and exits without output.
//   * Padding samples (j >= n) are +inf in every column, so they never enter
//     a heap or a count; padding queries (i >= n) compute on zeros and are
//     masked out of all outputs.
#pragma once

#include <cstdint>
#include <math_constants.h>

#include "ksg_common.cuh"

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

// Reference row jj of a staged sh tile (DSP floats, float4 aligned).
template <int DSP>
__device__ __forceinline__ void load_row(const float *rs, int jj, float (&r)[DSP])
{
#pragma unroll
    for (int m = 0; m < DSP / 4; ++m) {
        const float4 v = reinterpret_cast<const float4 *>(rs + jj * DSP)[m];
        r[4 * m + 0] = v.x;
        r[4 * m + 1] = v.y;
        r[4 * m + 2] = v.z;
        r[4 * m + 3] = v.w;
    }
}

// X values of the GB jobs at reference jj of a staged xi tile.
template <int XW>
__device__ __forceinline__ void load_xrow(const float *rx, int jj, float (&xv)[XW])
{
#pragma unroll
    for (int m = 0; m < XW / 4; ++m) {
        const float4 v = reinterpret_cast<const float4 *>(rx + jj * XW)[m];
        xv[4 * m + 0] = v.x;
        xv[4 * m + 1] = v.y;
        xv[4 * m + 2] = v.z;
        xv[4 * m + 3] = v.w;
    }
}

// 0xffffffff if a < b else 0 (IEEE compare; false for NaN).
__device__ __forceinline__ uint32_t lt_mask(float a, float b)
{
    uint32_t r;
    asm("set.lt.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

// Bit jj of (lo | hi << 64) is set iff the max-norm distance over the first
// ND coordinates between the query and reference jj of the tile is < bound.
template <int ND, int DSP>
__device__ __forceinline__ void tile_mask(const float *rs, const float *q, float bound,
                                          uint64_t &lo, uint64_t &hi)
{
    uint32_t w[kTJ / 32];
#pragma unroll
    for (int word = 0; word < kTJ / 32; ++word) {
        uint32_t m = 0;
#pragma unroll 8
        for (int b = 31; b >= 0; --b) {
            float r[DSP];
            load_row<DSP>(rs, word * 32 + b, r);
            float d = fabsf(q[0] - r[0]);
#pragma unroll
            for (int t = 1; t < ND; ++t) d = fmaxf(d, fabsf(q[t] - r[t]));
            m = m + m - lt_mask(d, bound);  // shift in one bit: 2m + (d < bound)
        }
        w[word] = m;
    }
    static_assert(kTJ == 128, "two 64-bit masks per tile");
    lo = (uint64_t)w[0] | ((uint64_t)w[1] << 32);
    hi = (uint64_t)w[2] | ((uint64_t)w[3] << 32);
}

// Pop the lowest set reference index of (lo, hi).
__device__ __forceinline__ int next_ref(uint64_t &lo, uint64_t &hi)
{
    const bool use_lo = lo != 0;
    const uint64_t m = use_lo ? lo : hi;
    const int jj = (__ffsll((long long)m) - 1) + (use_lo ? 0 : 64);
    const uint64_t rest = m & (m - 1);
    if (use_lo)
        lo = rest;
    else
        hi = rest;
    return jj;
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int GB>
struct KsgShape {
    static constexpr int DS = DZ + DY;
    static constexpr int DSP = (DS + 3) & ~3;
    static constexpr int XW = GB * DX;
    static constexpr size_t SMEM_SH = 2ull * kTJ * DSP * sizeof(float);
    static constexpr size_t SMEM_X = 2ull * kTJ * XW * sizeof(float);
    static constexpr size_t SMEM = SMEM_SH + SMEM_X + 2 * sizeof(uint64_t);
    static_assert(XW % 4 == 0, "x tile rows must be whole float4s");
};

template <int DX, int DY, int DZ, int K1, bool EXACT, int GB>
__global__ void __launch_bounds__(kTQ) ksg_fused_kernel(const KsgLaunch a)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, GB>;
    constexpr int DS = S::DS;
    constexpr int DSP = S::DSP;
    constexpr int XW = S::XW;
    constexpr int NW = kTQ / 32;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_sh = reinterpret_cast<float *>(smem_raw);
    float *s_x = reinterpret_cast<float *>(smem_raw + S::SMEM_SH);
    uint64_t *s_bar = reinterpret_cast<uint64_t *>(smem_raw + S::SMEM_SH + S::SMEM_X);
    __shared__ int s_abort;
    __shared__ double s_red[NW][GB];

    const int tid = threadIdx.x;
    const int qt = blockIdx.x;
    const int grp = blockIdx.y;
    const int64_t i = static_cast<int64_t>(qt) * kTQ + tid;
    const bool valid = i < a.n;
    const int n_tiles = static_cast<int>(a.n_pad / kTJ);
    const float *xi_grp = a.xi + static_cast<int64_t>(grp) * a.n_pad * XW;

    // The query's own coordinates (zeros for padding queries).
    float q[DS];
#pragma unroll
    for (int d = 0; d < DS; ++d) q[d] = valid ? a.sh[i * DSP + d] : 0.0f;
    float xq[GB][DX];
#pragma unroll
    for (int g = 0; g < GB; ++g)
#pragma unroll
        for (int d = 0; d < DX; ++d) xq[g][d] = valid ? xi_grp[i * XW + g * DX + d] : 0.0f;

    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int total = 2 * n_tiles;  // pass A tiles, then pass B tiles
    constexpr uint32_t kShBytes = kTJ * DSP * sizeof(float);
    constexpr uint32_t kXBytes = kTJ * XW * sizeof(float);
    int issued = 0;
    auto issue = [&](int it) {
        const int tile = it < n_tiles ? it : it - n_tiles;
        const int st = it & 1;
        mbar_arrive_expect_tx(&s_bar[st], kShBytes + kXBytes);
        tma_bulk_load(s_sh + st * kTJ * DSP, a.sh + static_cast<int64_t>(tile) * kTJ * DSP,
                      kShBytes, &s_bar[st]);
        tma_bulk_load(s_x + st * kTJ * XW, xi_grp + static_cast<int64_t>(tile) * kTJ * XW, kXBytes,
                      &s_bar[st]);
    };
    if (tid == 0) {
        issue(0);
        if (total > 1) issue(1);
    }
    issued = total > 1 ? 2 : 1;

    // Wait for the tile of iteration `it`; false (and the CTA-wide abort flag)
    // when the bounded wait ran out.
    auto wait_tile = [&](int it) {
        if (!mbar_wait_bounded(&s_bar[it & 1], static_cast<uint32_t>((it >> 1) & 1),
                               a.timeout_ns)) {
            s_abort = 1;
            atomicOr(a.err, kErrTimeout);
        }
    };
    // After the CTA finished reading iteration `it`'s stage: refill it.
    auto release_tile = [&](int it) {
        if (tid == 0 && it + 2 < total) {
            fence_proxy_async_smem();
            issue(it + 2);
        }
        if (it + 2 < total) ++issued;
    };

    int it = 0;
    float e[GB];
    {
        // ---------------- pass A: per job the k+1 smallest joint distances, ascending
        float h[GB][K1];
#pragma unroll
        for (int g = 0; g < GB; ++g)
#pragma unroll
            for (int m = 0; m < K1; ++m) h[g][m] = CUDART_INF_F;
        float kth[GB];
#pragma unroll
        for (int g = 0; g < GB; ++g) kth[g] = CUDART_INF_F;
        float bound = CUDART_INF_F;  // >= every job's current threshold

        for (; it < n_tiles; ++it) {
            wait_tile(it);
            const float *rs = s_sh + (it & 1) * kTJ * DSP;
            const float *rx = s_x + (it & 1) * kTJ * XW;
            // Phase 1: which references of the tile pass the shared bound.
            uint64_t lo, hi;
            tile_mask<DS, DSP>(rs, q, bound, lo, hi);
            // Phase 2: this thread's passing references only (warps iterate
            // max-over-lanes times instead of union-over-lanes).
            while (lo | hi) {
                const int jj = next_ref(lo, hi);
                float r[DSP];
                load_row<DSP>(rs, jj, r);
                float dyz = fabsf(q[0] - r[0]);
#pragma unroll
                for (int d = 1; d < DS; ++d) dyz = fmaxf(dyz, fabsf(q[d] - r[d]));
                float xv[XW];
                load_xrow<XW>(rx, jj, xv);
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    float dxg = fabsf(xq[g][0] - xv[g * DX]);
#pragma unroll
                    for (int d = 1; d < DX; ++d) dxg = fmaxf(dxg, fabsf(xq[g][d] - xv[g * DX + d]));
                    const float dd = fmaxf(dxg, dyz);
                    const float th = EXACT ? h[g][K1 - 1] : kth[g];
                    if (dd < th) {
                        sorted_insert<K1>(h[g], dd);
                        if (!EXACT) kth[g] = select_kth<K1>(h[g], a.k);
                    }
                }
            }
            float bb = EXACT ? h[0][K1 - 1] : kth[0];
#pragma unroll
            for (int g = 1; g < GB; ++g) bb = fmaxf(bb, EXACT ? h[g][K1 - 1] : kth[g]);
            bound = bb;
            __syncthreads();
            if (s_abort) break;
            release_tile(it);
        }
#pragma unroll
        for (int g = 0; g < GB; ++g) e[g] = EXACT ? h[g][K1 - 1] : kth[g];
    }

    int cxz[GB], cyz[GB], cz[GB];
    if (!s_abort) {
        // ---------------- pass B: strict-radius counts in the subspaces
        float bound = 0.0f;
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            bound = fmaxf(bound, e[g]);
            cxz[g] = 0;
            cyz[g] = 0;
            cz[g] = 0;
        }
        for (; it < total; ++it) {
            wait_tile(it);
            const float *rs = s_sh + (it & 1) * kTJ * DSP;
            const float *rx = s_x + (it & 1) * kTJ * XW;
            uint64_t lo, hi;
            tile_mask<DZ, DSP>(rs, q, bound, lo, hi);  // Z distance < max eps
            while (lo | hi) {
                const int jj = next_ref(lo, hi);
                float r[DSP];
                load_row<DSP>(rs, jj, r);
                float dz = fabsf(q[0] - r[0]);
#pragma unroll
                for (int d = 1; d < DZ; ++d) dz = fmaxf(dz, fabsf(q[d] - r[d]));
                float dyz = dz;
#pragma unroll
                for (int d = DZ; d < DS; ++d) dyz = fmaxf(dyz, fabsf(q[d] - r[d]));
                float xv[XW];
                load_xrow<XW>(rx, jj, xv);
#pragma unroll
                for (int g = 0; g < GB; ++g) {
                    float dxg = fabsf(xq[g][0] - xv[g * DX]);
#pragma unroll
                    for (int d = 1; d < DX; ++d) dxg = fmaxf(dxg, fabsf(xq[g][d] - xv[g * DX + d]));
                    cz[g] += dz < e[g] ? 1 : 0;
                    cyz[g] += dyz < e[g] ? 1 : 0;
                    cxz[g] += fmaxf(dxg, dz) < e[g] ? 1 : 0;
                }
            }
            __syncthreads();
            if (s_abort) break;
            release_tile(it);
        }
    }

    if (s_abort) {
        // Wait (bounded) for this CTA's copies still in flight, then leave.
        if (tid == 0)
            for (int u = it; u < issued; ++u)
                (void)mbar_wait_bounded(&s_bar[u & 1], static_cast<uint32_t>((u >> 1) & 1),
                                        a.timeout_ns);
        __syncthreads();
        return;
    }

    // ---------------- epilogue: self pair, outputs, digamma terms
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int g = 0; g < GB; ++g) {
        const int self = e[g] > 0.0f ? 1 : 0;
        const int nxz = cxz[g] - self, nyz = cyz[g] - self, nz = cz[g] - self;
        const int job = grp * GB + g;
        double t = 0.0;
        if (valid && job < a.n_jobs) {
            t = a.psi[nz + 1] - a.psi[nxz + 1] - a.psi[nyz + 1];
            if (a.eps_out) a.eps_out[static_cast<int64_t>(job) * a.n + i] = e[g];
            if (a.cnt_out) {
                int32_t *c = a.cnt_out + static_cast<int64_t>(job) * 3 * a.n;
                c[i] = nxz;
                c[a.n + i] = nyz;
                c[2 * a.n + i] = nz;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) s_red[warp][g] = t;
    }
    __syncthreads();
    if (tid < GB) {
        const int job = grp * GB + tid;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += s_red[w][tid];
        if (job < a.n_jobs) a.partial[static_cast<int64_t>(job) * a.n_qt + qt] = s;
    }
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int GB>
cudaError_t launch_ksg(const KsgLaunch &a, int n_groups, cudaStream_t stream)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, GB>;
    auto kern = ksg_fused_kernel<DX, DY, DZ, K1, EXACT, GB>;
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(S::SMEM));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid(static_cast<unsigned>(a.n_qt), static_cast<unsigned>(n_groups));
    kern<<<grid, kTQ, S::SMEM, stream>>>(a);
    return cudaGetLastError();
}

template <int DX, int DY, int DZ, int K1, bool EXACT, int GB>
KsgVariant make_variant()
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, GB>;
    return KsgVariant{DX, DY, DZ, K1, EXACT ? 1 : 0, GB, S::DSP,
                      &launch_ksg<DX, DY, DZ, K1, EXACT, GB>};
}

}  // namespace idtx
