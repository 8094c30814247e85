// ksg_common.cuh -- internal declarations shared by the library's translation units.
//
// Layouts in device memory (all fp32 unless stated):
//   sh   [n_pad][dsp]        "shared" coordinates of every sample, the same for all
//                            jobs of a group: DZ z-dimensions, then DY y-dimensions,
//                            then unused padding up to dsp (a multiple of 4).
//                            Missing z/y dimensions of a bucket are 0; rows
//                            j >= n (padding samples) are +inf in every column.
//   xi   [n_groups][n_pad][GB*DX]
//                            per-job X values, GB jobs interleaved per sample:
//                            element (j, g, d) = X_job[d][pi_job(j)], +inf for j >= n.
//   psi  [n_max+1] fp64      digamma at the integers 1..n_max (index 0 unused).
//   partial [n_jobs][n_qt] fp64  per query tile sums of the digamma terms.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace idtx {

constexpr int kTQ = 128;  // queries per CTA (one per thread)
constexpr int kTJ = 128;  // reference samples per staged tile

// Device error word bits.
enum : int {
    kErrNonFinite = 1,  // NaN/Inf in an input column
    kErrTimeout = 2,    // a bounded mbarrier wait ran out
    kErrInternal = 4,   // an internal check failed
};

struct KsgLaunch {
    const float *sh;
    const float *xi;
    const double *psi;
    double *partial;
    float *eps_out;      // nullable, [n_jobs][n]
    int32_t *cnt_out;    // nullable, [n_jobs][3][n]: n_xz, n_yz, n_z
    int *err;
    int64_t n, n_pad;
    int n_jobs, n_qt, k;
    long long timeout_ns;
};

typedef cudaError_t (*KsgLaunchFn)(const KsgLaunch &, int n_groups, cudaStream_t);

// One compiled specialisation of the fused estimator kernel.
struct KsgVariant {
    int dx, dy, dz;   // bucket dimensions (inputs are zero-padded up to them)
    int k1;           // heap length (k+1 when exact, else an upper bound)
    int exact;        // 1: only k == k1-1
    int gb;           // jobs per CTA
    int dsp;          // floats per row of sh
    KsgLaunchFn fn;
};

// Registries filled by the instantiation units.
int ksg_variants_d11(KsgVariant *out);
int ksg_variants_d12(KsgVariant *out);
int ksg_variants_d21(KsgVariant *out);
int ksg_variants_d22(KsgVariant *out);
int ksg_variants_generic(KsgVariant *out);

}  // namespace idtx
