// shuffle.cuh -- surrogate permutations: the Fisher-Yates (Durstenfeld)
// shuffle driven by SplitMix64, one warp per permutation, bit for bit the
// sequential definition.
//
// The permutation of slot `slot` of n samples: the row starts as the
// identity; for step s = 0 .. n-2, with i = n-1-s,
//   r   = mix64(base + (s+1) * gamma),   base = seed ^ mix64(stream)
//   j   = hi64(r * (i+1))                (uniform on 0..i)
//   swap a[i], a[j].
// The steps are sequential, but steps on disjoint positions commute: the
// warp draws the next 32 steps in parallel (lane t takes step s0 + t) and
// performs at once the longest prefix of them in which no step draws the
// same j as an earlier one or has its position i drawn by an earlier one (an
// earlier step cannot touch a later one's j, since j <= i), then continues
// after that prefix.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace idtx {

constexpr uint64_t kSplitMixGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    // SplitMix64 output function (Steele, Lea & Flood 2014).
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Any n: the row shuffled in place in global memory (int32, loads and stores
// through L2), 64-bit step arithmetic.  perm[slot * n .. +n).
__global__ void __launch_bounds__(32)
    k_fisher_yates(int32_t *perm, const uint64_t *streams, const uint64_t *seeds, int64_t n)
{
    constexpr unsigned kFull = 0xffffffffu;
    const int slot = blockIdx.x;
    const int lane = threadIdx.x;
    int32_t *a = perm + (int64_t)slot * n;
    for (int64_t i = lane; i < n; i += 32) __stcg(a + i, (int32_t)i);
    __syncwarp();
    const uint64_t base = seeds[slot] ^ mix64(streams[slot]);
    const uint32_t below = (1u << lane) - 1u;
    int64_t s0 = 0;
    while (s0 < n - 1) {
        const int64_t s = s0 + lane;
        const bool valid = s < n - 1;
        const int64_t i = n - 1 - s;
        int64_t j = 0;
        if (valid) {
            const uint64_t r = mix64(base + (uint64_t)(s + 1) * kSplitMixGamma);
            j = (int64_t)__umul64hi(r, (uint64_t)(i + 1));
        }
        const uint32_t live = __ballot_sync(kFull, valid);
        // same j as an earlier lane
        const uint32_t same = __match_any_sync(kFull, valid ? (int)j : -1 - lane);
        const uint32_t dup = __ballot_sync(kFull, valid && (same & below) != 0);
        // position i drawn by an earlier lane: lane a marks lane n-1-s0-j_a
        const int64_t b = n - 1 - s0 - j;
        const uint32_t hit =
            __reduce_or_sync(kFull, (valid && b > lane && b < 32) ? (1u << (int)b) : 0u);
        const uint32_t bad = (dup | hit) & live;
        const int run = bad ? __ffs(bad) - 1 : __popc(live);
        if (lane < run) {
            const int32_t x = __ldcg(a + i), y = __ldcg(a + j);
            __stcg(a + i, y);
            __stcg(a + j, x);
        }
        __syncwarp();
        s0 += run;
    }
}

// Layouts of k_shuffle_smem's row in shared memory, by row length.
enum ShuffleMode : int {
    kShufPosFlag = 0,  // n <= 32768: uint16_t entries, flags in their top bits
    kShufBitmap = 1,   // n <= 65536: uint16_t entries, then an n-bit flag bitmap
    kShufWide = 2,     // n <= kWideMaxN: the low 16 bits of the entries, then a
                       // bitmap of their bit 16, then the flag bitmap
};
constexpr int kPosFlagMaxN = 32768;
constexpr int kWideMaxN = 102400;  // 230400 bytes: within 227 KB of shared memory

// Dynamic shared memory of k_shuffle_smem<MODE> for rows of n samples.
__host__ __device__ constexpr int shuffle_smem_bytes(int n, int mode)
{
    return mode == kShufPosFlag
               ? ((2 * n + 3) & ~3)
               : ((2 * n + 15) & ~15) + (mode == kShufWide ? 2 : 1) * ((n + 31) / 32) * 4;
}

// The layout for a row of n samples (-1: too long for shared memory).
__host__ __device__ constexpr int shuffle_mode(int64_t n)
{
    return n <= kPosFlagMaxN ? kShufPosFlag
                             : (n <= 65536 ? kShufBitmap : (n <= kWideMaxN ? kShufWide : -1));
}

// n <= kWideMaxN: the row in dynamic shared memory (layout MODE, above),
// 32-bit step arithmetic.  Each lane keeps the draws of steps s0 + lane and
// s0 + 32 + lane, so SplitMix64 runs a round ahead of the conflict test, and
// a round's swaps (loads, then stores) bracket the next round's test.  With
// `order`, the row is written composed with it: perm[slot][j] = pi(order[j]),
// so that a consumer indexing samples in that order reads the row in
// sequence.
//
// Equal draws.  Each lane sets a flag bit for its position j with an atomic
// OR, and of any lanes with equal draws all but the first to arrive find
// the bit already set.  A flagged lane is treated as a conflict: that cuts
// the prefix at a flagged lane of every equal pair, which may be the earlier
// lane of the pair (the prefix is then shorter than it could be, never
// wrong; when that lane is the round's first it runs alone).  The order in
// which the hardware serves a warp's atomics is not relied on.  The flags
// are cleared before the round's swaps store.  The flag of position j is
// the top bit of entry j itself in kShufPosFlag (every entry leaves that bit
// free), else bit j of the flag bitmap.  Measured on GB300, 9447 rows of
// 9995 written composed: 0.62 ms, against 0.79 ms with a 4096-bit bitmap
// indexed by j mod 4096 (whose flags needed an exact match.any to confirm),
// 1.05 ms with match.any in every round and 0.97 ms with one ballot per bit
// of j; match.any has 373 cycles of latency there.
template <int MODE>
__global__ void __launch_bounds__(32)
    k_shuffle_smem(int32_t *perm, const uint64_t *streams, const uint64_t *seeds, int n,
                   const int32_t *order)
{
    constexpr bool POS_FLAG = MODE == kShufPosFlag;
    extern __shared__ __align__(16) unsigned char fy_smem[];
    uint16_t *fy_row = reinterpret_cast<uint16_t *>(fy_smem);
    const int words = (n + 31) / 32;
    uint32_t *hib = reinterpret_cast<uint32_t *>(fy_smem + ((2 * n + 15) & ~15));
    uint32_t *bitmap = MODE == kShufWide ? hib + words : hib;
    constexpr unsigned kFull = 0xffffffffu;
    const int slot = blockIdx.x;
    const int lane = threadIdx.x;
    // entry p of the row; kShufWide keeps bit 16 in hib (set with atomics:
    // a round's lanes write distinct entries that may share a word)
    auto read = [&](uint32_t p) -> uint32_t {
        uint32_t v = fy_row[p];
        if (MODE == kShufWide) v |= ((hib[p >> 5] >> (p & 31u)) & 1u) << 16;
        return v;
    };
    auto write = [&](uint32_t p, uint32_t v) {
        fy_row[p] = (uint16_t)v;
        if (MODE == kShufWide) {
            const uint32_t b = 1u << (p & 31u);
            if (v >> 16)
                atomicOr(&hib[p >> 5], b);
            else
                atomicAnd(&hib[p >> 5], ~b);
        }
    };
    for (int i = lane; i < n; i += 32) fy_row[i] = (uint16_t)i;
    if (MODE == kShufWide)
        for (int w = lane; w < words; w += 32) hib[w] = w * 32 >= 65536 ? 0xffffffffu : 0u;
    if (!POS_FLAG)
        for (int w = lane; w < words; w += 32) bitmap[w] = 0u;
    __syncwarp();
    const uint64_t base = seeds[slot] ^ mix64(streams[slot]);
    auto draw = [&](int s) { return mix64(base + (uint64_t)(s + 1) * kSplitMixGamma); };
    const int last = n - 1;  // steps 0 .. last-1
    uint64_t r_a = draw(lane), r_b = draw(32 + lane);
    // The test of the round starting at step s0 with draws r_a: each lane's
    // position i and draw j, and the length of the conflict-free prefix.
    auto test = [&](int s0, uint32_t &i, uint32_t &j) -> int {
        const int s = s0 + lane;
        const bool valid = s < last;
        i = (uint32_t)(last - s);
        // j = hi64(r * (i+1)) from 32-bit halves (i+1 < 2^32):
        // hi64(r m) = (hi32(r) m + hi32(lo32(r) m)) >> 32, no carry out
        const uint32_t m = i + 1u;
        const uint64_t ph = (uint64_t)(uint32_t)(r_a >> 32) * m;
        const uint32_t pl = __umulhi((uint32_t)r_a, m);
        j = valid ? (uint32_t)((ph + pl) >> 32) : 0u;
        const uint32_t live = __ballot_sync(kFull, valid);
        uint32_t *word = POS_FLAG ? reinterpret_cast<uint32_t *>(fy_row) + (j >> 1)
                                  : bitmap + (j >> 5);
        const uint32_t bit = POS_FLAG ? 0x8000u << ((j & 1u) * 16) : 1u << (j & 31u);
        const uint32_t old = valid ? atomicOr(word, bit) : 0u;
        __syncwarp();  // every lane's OR is done before any flag is cleared
        if (valid) {
            if (POS_FLAG)
                atomicAnd(word, ~bit);
            else
                *word = 0u;
        }
        __syncwarp();
        const uint32_t dup = __ballot_sync(kFull, (old & bit) != 0);
        // position i of lane b = last - s0 - b is drawn by an earlier lane
        const int b = (last - s0) - (int)j;
        const uint32_t hit =
            __reduce_or_sync(kFull, (valid && b > lane && b < 32) ? (1u << b) : 0u);
        const uint32_t bad = (dup | hit) & live;
        // Lane 0 never conflicts (no earlier lane), but its flag is set when
        // a later equal draw's atomic was served first: it then runs alone.
        // Every round so advances by at least one step.
        return bad ? max(1, __ffs(bad) - 1) : __popc(live);
    };
    int s0 = 0;
    uint32_t i = 0, j = 0;
    int run = last > 0 ? test(0, i, j) : 0;
    while (run > 0) {
        uint32_t x = 0, y = 0;
        if (lane < run) {
            x = read(i);
            y = read(j);
        }
        if (POS_FLAG) __syncwarp();  // the loads are done before the next test flags
        // slide the window by run steps and test the next round
        const int src = (lane + run) & 31;
        const bool from_a = lane + run < 32;
        const uint64_t sa = __shfl_sync(kFull, r_a, src);
        const uint64_t sb = __shfl_sync(kFull, r_b, src);
        const int s0n = s0 + run;
        const uint64_t fresh = draw(s0n + 32 + lane);
        r_a = from_a ? sa : sb;
        r_b = from_a ? sb : fresh;
        uint32_t in = 0, jn = 0;
        const int run_n = s0n < last ? test(s0n, in, jn) : 0;
        if (lane < run) {
            write(i, y);
            write(j, x);
        }
        __syncwarp();
        s0 = s0n;
        i = in;
        j = jn;
        run = run_n;
    }
    int32_t *out = perm + (int64_t)slot * n;
    if (order) {
        // kBatch loads of the order in flight per lane before their lookups
        constexpr int kBatch = 8;
        for (int t0 = 0; t0 < n; t0 += 32 * kBatch) {
            int o[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int t = t0 + u * 32 + lane;
                o[u] = t < n ? __ldg(order + t) : 0;
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int t = t0 + u * 32 + lane;
                if (t < n) out[t] = (int32_t)read((uint32_t)o[u]);
            }
        }
    } else {
        for (int t = lane; t < n; t += 32) out[t] = (int32_t)read((uint32_t)t);
    }
}

}  // namespace idtx
