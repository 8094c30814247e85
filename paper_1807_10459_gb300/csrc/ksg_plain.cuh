// ksg_plain.cuh -- the "plain" schedule: one estimate per launch.
//
// The reference point that batching is measured against: the KSG estimate
// (KSG algorithm 1, conditional form; the estimator named in the IDTxl
// paper's Summary) of ONE job by brute force, with no sharing between
// estimates, no sample ordering and no pruning.  A warp serves one query;
// its 32 lanes split the reference samples (lane l takes j = l, l + 32, ...),
// each keeping its own k+1 smallest joint distances (the query itself, at
// distance 0, included), and the warp merges them by repeated minima, so the
// (k+1)-th smallest is eps_i.  A second sweep counts the strict-radius
// neighbours in the subspaces, the self pair removed.  A CTA of 8 warps
// serves 8 consecutive queries and writes their digamma terms' sum, in warp
// order, as one partial; k_finalize sums the partials in order.  Distances
// are the definition's fp32 |a - b| and maxima, so eps and the counts equal
// the other kernels'; only the order of the fp64 sum differs (estimates
// agree within rounding).
#pragma once

#include "ksg_kernel.cuh"

namespace idtx {

constexpr int kPlainWarps = kPlainQueriesPerPartial;  // queries per CTA of the plain schedule

// sh: the group's shared-coordinate tiles (DZ z columns, then DY y columns,
// rows of DSP floats); xj: this job's X values [n_pad][DX]; partial: this
// job's [n_pad / kPlainWarps] partial sums; eps (nullable): this job's [n]
// eps_i; cnt (nullable): this job's [3][n] n_xz, n_yz, n_z.
template <int DX, int DY, int DZ, int K1, bool EXACT, int DSP>
__global__ void __launch_bounds__(kPlainWarps * 32)
    k_ksg_plain(const float *sh, const float *xj, int64_t n, int k, const double *psi,
                double *partial, float *eps, int32_t *cnt)
{
    constexpr int DS = DZ + DY;
    constexpr int KH = K1;  // the k+1 smallest including the query (EXACT: exactly)
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ double s_t[kPlainWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = blockIdx.x * static_cast<int64_t>(kPlainWarps) + warp;
    auto row = [&](int64_t j) { return sh + ((j / kTJ) * kTileRows + (j % kTJ)) * DSP; };
    double term = 0.0;
    if (i < n) {
        float q[DS], xq[DX];
        const float *qr = row(i);
#pragma unroll
        for (int d = 0; d < DS; ++d) q[d] = qr[d];
#pragma unroll
        for (int d = 0; d < DX; ++d) xq[d] = xj[i * DX + d];
        // subspace distances of reference j: Z, then (Y,Z), then (X,Z) and joint
        auto dist = [&](int64_t j, float &dz, float &dyz, float &dxz, float &dj) {
            const float *r = row(j);
            float mz = 0.0f;
#pragma unroll
            for (int d = 0; d < DZ; ++d) mz = fmaxf(mz, fabsf(q[d] - r[d]));
            float my = mz;
#pragma unroll
            for (int d = DZ; d < DS; ++d) my = fmaxf(my, fabsf(q[d] - r[d]));
            float mx = 0.0f;
#pragma unroll
            for (int d = 0; d < DX; ++d) mx = fmaxf(mx, fabsf(xq[d] - xj[j * DX + d]));
            dz = mz;
            dyz = my;
            dxz = fmaxf(mx, mz);
            dj = fmaxf(mx, my);
        };
        float h[KH];
#pragma unroll
        for (int t = 0; t < KH; ++t) h[t] = CUDART_INF_F;
        float th = CUDART_INF_F;
        for (int64_t j = lane; j < n; j += 32) {
            float dz, dyz, dxz, dj;
            dist(j, dz, dyz, dxz, dj);
            if (dj < th) {
                sorted_insert<KH>(h, dj);
                th = EXACT ? h[KH - 1] : select_kth<KH>(h, k);
            }
        }
        // the (k+1)-th smallest over the warp: take the warp minimum k+1 times
        float e = 0.0f;
        for (int t = 0; t <= k; ++t) {
            e = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(h[0])));
            const uint32_t who = __ballot_sync(kFull, h[0] == e);
            if (lane == __ffs(who) - 1) {
#pragma unroll
                for (int m = 0; m + 1 < KH; ++m) h[m] = h[m + 1];
                h[KH - 1] = CUDART_INF_F;
            }
        }
        int cz = 0, cyz = 0, cxz = 0;
        for (int64_t j = lane; j < n; j += 32) {
            float dz, dyz, dxz, dj;
            dist(j, dz, dyz, dxz, dj);
            cz += dz < e ? 1 : 0;
            cyz += dyz < e ? 1 : 0;
            cxz += dxz < e ? 1 : 0;
        }
        cz = __reduce_add_sync(kFull, cz);
        cyz = __reduce_add_sync(kFull, cyz);
        cxz = __reduce_add_sync(kFull, cxz);
        const int self = e > 0.0f ? 1 : 0;
        term = psi[cz - self + 1] - psi[cxz - self + 1] - psi[cyz - self + 1];
        if (lane == 0) {
            if (eps) eps[i] = e;
            if (cnt) {
                cnt[i] = cxz - self;
                cnt[n + i] = cyz - self;
                cnt[2 * n + i] = cz - self;
            }
        }
    }
    if (lane == 0) s_t[warp] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kPlainWarps; ++w) s += s_t[w];
        partial[blockIdx.x] = s;
    }
}

// One CTA per kPlainWarps queries of the n_pad (a multiple of kTJ) padded
// ones, so that every partial of the job is written (0 past n).
template <int DX, int DY, int DZ, int K1, bool EXACT, int QC, int NWARPS>
cudaError_t launch_ksg_plain(const float *sh, const float *xj, const double *psi, int64_t n,
                             int64_t n_pad, int k, double *partial, float *eps, int32_t *cnt,
                             cudaStream_t stream)
{
    using S = KsgShape<DX, DY, DZ, K1, EXACT, QC, NWARPS>;
    const int64_t blocks = n_pad / kPlainWarps;
    if (blocks <= 0) return cudaSuccess;
    k_ksg_plain<DX, DY, DZ, K1, EXACT, S::DSP>
        <<<static_cast<unsigned>(blocks), kPlainWarps * 32, 0, stream>>>(sh, xj, n, k, psi,
                                                                         partial, eps, cnt);
    return cudaGetLastError();
}

}  // namespace idtx
