// probe.cu -- measured instruction-issue rates of the device, the peak the
// list kernel's roofline figure is taken against.
//
// The estimator path is a comparison workload (max-norm distances, strict
// compares, counts): no tensor-core contraction and, per the kernels' DRAM
// counters, far from the HBM bound.  Its roofline is instruction issue on
// the CUDA cores.  Each probe kernel runs one instruction class (or the
// count pass's mix) in eight independent register chains per thread at full
// occupancy, with no memory traffic inside the timed loop, and reports
// lane-operations per SM per clock and per second.
#include <cuda_runtime.h>

#include <cstdint>

#include "idtx.h"

namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeCtasPerSm = 2;
constexpr int kUnroll = 4;  // iterations of the 8-chain body per loop trip

// One probe.  Every step of a chain reads the current value of the next
// chain, so the assembler can neither fold a chain into fewer operations
// (as it would a chain of adds of one loop-invariant value) nor hoist a
// compare out of the loop.  OP 0: a_c = a_c + a_{c+1} (FADD); 1: a_c =
// max(a_c, a_{c+1}) (FMNMX); 2: a_c = a_c + a_{c+1}, n_c += (a_c < e) (FADD,
// FSETP and a predicated add: 3 operations); 3: n_c = n_c + n_{c+1} (IADD);
// 4: the count pass's step per (job, entry) with x_v = a_c and d_z = a_{c+1}:
// d = x_q - x_v; p = d_z < e; q = |d| < e and p; n_z += p; n_xz += q;
// a_c = d (subtract, absolute value, two compares, two adds: 6 operations).
template <int OP>
__global__ void __launch_bounds__(kProbeThreads)
    k_probe(int iters, unsigned long long *cycles, int *sink)
{
    float a[8];
    int n[8], m[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
        n[c] = static_cast<int>(threadIdx.x) + c;
        m[c] = c;
    }
    const float e = 0.5f, xq = 0.75f;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int nb = (c + 1) & 7;
                if (OP == 0) {
                    asm volatile("add.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(a[nb]));
                } else if (OP == 1) {
                    asm volatile("max.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(a[nb]));
                } else if (OP == 2) {
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tadd.f32 %1, %1, %2;\n\tsetp.lt.f32 p, %1, %3;\n\t"
                        "@p add.s32 %0, %0, 1;\n\t}"
                        : "+r"(n[c]), "+f"(a[c])
                        : "f"(a[nb]), "f"(e));
                } else if (OP == 3) {
                    asm volatile("add.s32 %0, %0, %1;" : "+r"(n[c]) : "r"(n[nb]));
                } else {
                    asm volatile(
                        "{\n\t.reg .pred p, q;\n\t.reg .f32 d;\n\t"
                        "sub.f32 d, %3, %2;\n\t"
                        "setp.lt.f32 p, %4, %5;\n\t"
                        "abs.f32 %2, d;\n\t"
                        "setp.lt.and.f32 q, %2, %5, p;\n\t"
                        "@p add.s32 %0, %0, 1;\n\t"
                        "@q add.s32 %1, %1, 1;\n\t"
                        "mov.f32 %2, d;\n\t}"
                        : "+r"(n[c]), "+r"(m[c]), "+f"(a[c])
                        : "f"(xq), "f"(a[nb]), "f"(e));
                }
            }
        }
    }
    const long long t1 = clock64();
    int acc = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc += n[c] + m[c] + __float_as_int(a[c]);
    if (acc == 0x7fffffff) sink[0] = acc;  // keeps the chains live
    if (threadIdx.x == 0) atomicAdd(cycles, static_cast<unsigned long long>(t1 - t0));
}

template <int OP>
int run_probe(int n_sms, int iters, cudaEvent_t e0, cudaEvent_t e1, unsigned long long *d_cyc,
              int *d_sink, double *ms_out, double *cycles_per_cta)
{
    const int grid = n_sms * kProbeCtasPerSm;
    if (cudaMemset(d_cyc, 0, sizeof(unsigned long long)) != cudaSuccess) return 1;
    k_probe<OP><<<grid, kProbeThreads>>>(iters / 8, d_cyc, d_sink);  // warm-up
    if (cudaMemset(d_cyc, 0, sizeof(unsigned long long)) != cudaSuccess) return 1;
    if (cudaEventRecord(e0) != cudaSuccess) return 1;
    k_probe<OP><<<grid, kProbeThreads>>>(iters, d_cyc, d_sink);
    if (cudaEventRecord(e1) != cudaSuccess) return 1;
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return 1;
    unsigned long long cyc = 0;
    if (cudaMemcpy(&cyc, d_cyc, sizeof(cyc), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    *ms_out = ms;
    *cycles_per_cta = static_cast<double>(cyc) / grid;
    return 0;
}

}  // namespace

extern "C" int idtx_probe_issue_rates(int device, idtx_issue_rates *out)
{
    if (!out) return IDTX_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return IDTX_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return IDTX_EINVAL;
    int rc = IDTX_OK;
    int n_sms = 0;
    unsigned long long *d_cyc = nullptr;
    int *d_sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&d_cyc, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&d_sink, sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = IDTX_ECUDA;
    const int iters = 4096;
    // lane-operations per thread of one probe: iters * unroll * 8 chains * ops
    const double per_thread = static_cast<double>(iters) * kUnroll * 8;
    const double threads = static_cast<double>(n_sms) * kProbeCtasPerSm * kProbeThreads;
    double ms[5] = {}, cyc[5] = {};
    if (rc == IDTX_OK &&
        (run_probe<0>(n_sms, iters, e0, e1, d_cyc, d_sink, &ms[0], &cyc[0]) ||
         run_probe<1>(n_sms, iters, e0, e1, d_cyc, d_sink, &ms[1], &cyc[1]) ||
         run_probe<2>(n_sms, iters, e0, e1, d_cyc, d_sink, &ms[2], &cyc[2]) ||
         run_probe<3>(n_sms, iters, e0, e1, d_cyc, d_sink, &ms[3], &cyc[3]) ||
         run_probe<4>(n_sms, iters, e0, e1, d_cyc, d_sink, &ms[4], &cyc[4])))
        rc = IDTX_ECUDA;
    if (rc == IDTX_OK) {
        // operations per chain step: 1 for the single-instruction classes, 3
        // for add, compare and consuming add, 6 for the count-pass step
        const double ops[5] = {1.0, 1.0, 3.0, 1.0, 6.0};
        double *per_clk[5] = {&out->fadd_per_sm_clk, &out->fmnmx_per_sm_clk,
                              &out->fsetp_add_per_sm_clk, &out->iadd_per_sm_clk,
                              &out->count_mix_per_sm_clk};
        double *per_s[5] = {&out->fadd_per_s, &out->fmnmx_per_s, &out->fsetp_add_per_s,
                            &out->iadd_per_s, &out->count_mix_per_s};
        for (int i = 0; i < 5; ++i) {
            const double lane_ops = per_thread * ops[i] * threads;
            *per_s[i] = lane_ops / (ms[i] * 1e-3);
            // a CTA's own clock count spans the whole launch (one wave)
            *per_clk[i] = lane_ops / (cyc[i] * n_sms);
        }
        out->sm_clock_mhz = cyc[4] / (ms[4] * 1e-3) * 1e-6;
        out->n_sms = n_sms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_cyc) cudaFree(d_cyc);
    if (d_sink) cudaFree(d_sink);
    cudaSetDevice(prev);
    return rc;
}
