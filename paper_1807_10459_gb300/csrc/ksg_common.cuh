// ksg_common.cuh -- internal declarations shared by the library's translation units.
//
// Layouts in device memory (all fp32 unless stated):
//   sh   [n_tiles][kTJ+2][dsp]  "shared" coordinates of every sample, the same for
//                            all jobs of a group, in tiles of kTJ samples: rows
//                            0..kTJ-1 hold DZ z-dimensions, then DY y-dimensions,
//                            then unused padding up to dsp (a multiple of 4);
//                            row kTJ holds the tile's per-dimension minimum and
//                            row kTJ+1 its maximum over its real samples.
//                            Missing z/y dimensions of a bucket are 0; samples
//                            j >= n (padding) are +inf in every column.
//   Samples are stored in the order `order` (sorted position m holds original
//   sample order[m]); without a sort order is the identity.
//   xi   [n_groups][n_pad][GB*DX]
//                            per-job X values, GB jobs interleaved per sample:
//                            element (j, g, d) = X_job[d][pi_job(j)], +inf for j >= n.
//   psi  [n_max+1] fp64      digamma at the integers 1..n_max (index 0 unused).
//   partial [n_jobs][n_qt] fp64  per query tile sums of the digamma terms.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace idtx {

#ifndef IDTX_TILE
#define IDTX_TILE 128
#endif
constexpr int kTJ = IDTX_TILE;  // reference samples per staged tile (a multiple of 32)
constexpr int kTQ = kTJ;        // sample padding granularity

// Device error word bits.
enum : int {
    kErrNonFinite = 1,  // NaN/Inf in an input column
    kErrTimeout = 2,    // a bounded mbarrier wait ran out
    kErrInternal = 4,   // an internal check failed
};

constexpr int kTileRows = kTJ + 2;  // samples + bounding box rows

// Work counters written by the fused kernel (per launch, summed over CTAs):
//   [0] (query, reference) pairs scanned by the neighbour pass,
//   [1] pairs that passed its shared bound (per-job work done),
//   [2] pairs scanned by the count pass, [3] pairs that passed its bound,
//   [4] SM clock cycles warps spent waiting for staged tiles, [5] cycles warps
//   spent in the kernel (both summed over warps).
// The list kernel (ksg_list.cuh) writes, per (query, group of jobs):
//   [0] list A entries walked, [1] list B entries walked, [2] / [3] samples
//   scanned by pass-A / pass-B full-scan fallbacks, [4] fallbacks taken,
//   [5] cycles as above, [6] (job, entry) pairs of the count walk's repacked
//   phases, [7] (job, entry) pairs of the neighbour walk's lane-split tails,
//   [8] / [9] the sums of n_z / n_yz over (query, job): the list entries a
//   walk that visited exactly the entries each job needs would touch.
constexpr int kNumWork = 10;

// Capacities of the per-query neighbour lists (entries; multiples of 32).
constexpr int kMaxListA = 2048;  // by d_YZ
constexpr int kMaxListB = 4096;  // by d_Z

// The list kernel's ring of per-query digamma terms (ksg_list.cuh), in global
// scratch after the lists: per CTA, kListRing query tiles of up to 64
// queries x 32 jobs (fp64).  The kernel runs at most kListRingCtas CTAs.
#ifndef IDTX_LIST_RING
#define IDTX_LIST_RING 8
#endif
constexpr int kListRing = IDTX_LIST_RING;
constexpr int kListRingCtas = 192;
constexpr size_t kListRingBytes = (size_t)kListRingCtas * kListRing * 64 * 32 * sizeof(double);

struct KsgLaunch {
    const float *sh;
    const float *xi;
    const double *psi;
    double *partial;
    float *eps_out;      // nullable, [n_jobs][n] in original sample order
    int32_t *cnt_out;    // nullable, [n_jobs][3][n]: n_xz, n_yz, n_z, original order
    const int32_t *order;  // nullable: original index of sorted position m
    unsigned long long *work;  // nullable, [kNumWork]
    int *err;
    int64_t n, n_pad;
    int n_jobs, n_qt, k;
    long long timeout_ns;
    // list kernel only (ksg_list.cuh): per query i, list_a[i * cap_a ..] and
    // list_b[i * cap_b ..] entries (sorted sample j, distance bits) and
    // lmeta[i] = (len_a, len_b, bits of r_a, bits of r_b)
    const int2 *list_a;
    const int2 *list_b;
    const int4 *lmeta;
    double *ring;  // kListRingBytes of scratch for the list kernel's term ring
    int cap_a, cap_b;
};

typedef cudaError_t (*KsgLaunchFn)(const KsgLaunch &, int n_groups, cudaStream_t);

// One estimate of one job by the plain schedule (ksg_plain.cuh): sh the
// group's tiles, xj the job's X values [n_pad][dx bucket], partial the job's
// n_pad / 8 partial sums.
typedef cudaError_t (*KsgPlainFn)(const float *sh, const float *xj, const double *psi, int64_t n,
                                  int64_t n_pad, int k, double *partial, float *eps,
                                  int32_t *cnt, cudaStream_t);
constexpr int kPlainQueriesPerPartial = 8;

// Several problems of one kernel variant in one persistent launch.  Task t
// (0 <= t < n_tasks) belongs to the problem p with start[p] <= t < start[p+1];
// its local index l = t - start[p] is query tile l % n_qt of job group
// l / n_qt.  CTAs take tasks in order from *next (zero before the launch).
struct KsgTable {
    const KsgLaunch *probs;  // device [n_probs]
    const int64_t *start;    // device [n_probs + 1]
    int *next;               // device counter
    int n_probs;
    int64_t n_tasks;
};

typedef cudaError_t (*KsgTableFn)(const KsgTable &, cudaStream_t);

// One compiled specialisation of the fused estimator kernel.
struct KsgVariant {
    int dx, dy, dz;   // bucket dimensions (inputs are zero-padded up to them)
    int k1;           // heap length (k+1 when exact, else an upper bound)
    int exact;        // 1: only k == k1-1
    int gb;           // jobs per CTA (one per lane)
    int dsp;          // floats per row of sh
    int qc;           // queries per CTA
    KsgLaunchFn fn;
    KsgTableFn fn_table;  // persistent multi-problem form
    KsgLaunchFn fn_list;  // the same estimates over sorted neighbour lists
    KsgPlainFn fn_plain;  // one estimate per launch (the plain schedule)
};

// Per-query sorted neighbour lists of a group prepared into sh (lists.cu):
// z columns [0, dzb), y columns [dzb, dsb) of rows of dsp floats.
cudaError_t build_lists(const float *sh, int dsp, int dzb, int dsb, int64_t n, int cap_a,
                        int cap_b, int2 *list_a, int2 *list_b, int4 *meta, cudaStream_t st);

// Radix sort of (key, index) pairs on the low end_bit key bits (sort.cu).
// With tmp == nullptr only sets tmp_bytes.
cudaError_t sort_pairs_u32(void *tmp, size_t &tmp_bytes, const uint32_t *keys_in,
                           uint32_t *keys_out, const int32_t *vals_in, int32_t *vals_out, int n,
                           int end_bit, cudaStream_t stream);

// Learned-screen network kernels (screen.cu).  A work area holds the batch
// activations (B rows), the gradient and the bf16 copy of the parameters.
struct MlpWork {
    float *xn, *z1, *a1, *z2, *a2, *d2, *d1, *y, *dy, *grad;
    __nv_bfloat16 *wbf;
};
size_t mlp_work_floats(int B);
void mlp_work_carve(float *base, int B, MlpWork *w);
cudaError_t mlp_round(const float *params, MlpWork &w, cudaStream_t st);
cudaError_t mlp_forward(const float *params, MlpWork &w, const float *feats,
                        const int32_t *order, int64_t start, int B, const float *mean,
                        const float *scale, cudaStream_t st);
cudaError_t mlp_loss(MlpWork &w, const float *targets, const int32_t *order, int64_t start, int B,
                     float dy_scale, float quantile, bool want_dy, double *loss_acc,
                     cudaStream_t st);
cudaError_t mlp_backward(MlpWork &w, int B, bool accumulate, cudaStream_t st);
cudaError_t mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr,
                     cudaStream_t st);

// One-time set-up per device (kernel attributes, occupancy, SM count).
// Function attributes and device properties belong to a device, so a process
// that uses several GPUs needs the set-up once on each; the mutex serialises
// host threads.  A failed set-up is retried by the next call.
constexpr int kMaxDevices = 64;
struct DeviceOnce {
    std::mutex mu;
    bool done[kMaxDevices] = {};
};

// Runs f(device) on the current device unless it already succeeded there.
template <typename F>
cudaError_t once_per_device(DeviceOnce &o, F &&f)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(o.mu);
    if (o.done[dev]) return cudaSuccess;
    e = f(dev);
    if (e == cudaSuccess) o.done[dev] = true;
    return e;
}

// Registries filled by the instantiation units.
int ksg_variants_d11(KsgVariant *out);
int ksg_variants_d12(KsgVariant *out);
int ksg_variants_d21(KsgVariant *out);
int ksg_variants_d22(KsgVariant *out);
int ksg_variants_generic(KsgVariant *out);

}  // namespace idtx
