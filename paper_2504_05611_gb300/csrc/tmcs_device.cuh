// Device primitives shared by the sampling kernels (tmcs_sample.cu,
// tmcs_flow.cu): the Philox4x32-10 generator and the gap count of the
// sampling specification, wall-clock time for bounded waits, and
// shared-memory counters.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "tmcs_internal.h"

namespace tmcs {

constexpr uint64_t kWaitNs = 2000000000ull;  // bounded device-side waits: 2 s of wall time

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products (multipliers 0xD2511F53, 0xCD9E8D57) whose high
// halves are XORed with the other two counter words and the round key; the
// key is bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t n0 = uint32_t(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = uint32_t(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = uint32_t(p1);
        c2 = n2;
        c3 = uint32_t(p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Philox4x32-10 of counter (j, c1, c2, c3) for a stream whose words c1, c2,
// c3 are fixed: round 1 of every call shares the product of c2 and the
// words derived from it, so a stream computes them once (philox_stream) and
// each call starts from round 2's inputs. Same output as philox4x32_10.
struct PhiloxStream {
    uint32_t a0;  // round-1 output word 0: hi(M1 c2) ^ c1 ^ k0
    uint32_t a1;  // round-1 output word 1: lo(M1 c2)
    uint32_t a3;  // c3 ^ k1 (XORed with hi(M0 j) to give round-1 word 2)
};

__device__ __forceinline__ PhiloxStream philox_stream(uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                      uint32_t k1) {
    const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
    PhiloxStream s;
    s.a0 = uint32_t(p1 >> 32) ^ c1 ^ k0;
    s.a1 = uint32_t(p1);
    s.a3 = c3 ^ k1;
    return s;
}

__device__ __forceinline__ uint4 philox_call(const PhiloxStream &s, uint32_t j, uint32_t k0, uint32_t k1) {
    const uint64_t p0 = uint64_t(0xD2511F53u) * j;
    uint32_t c0 = s.a0, c1 = s.a1, c2 = uint32_t(p0 >> 32) ^ s.a3, c3 = uint32_t(p0);
#pragma unroll
    for (int r = 1; r < 10; r++) {
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
        const uint64_t q0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t q1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t n0 = uint32_t(q1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = uint32_t(q0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = uint32_t(q1);
        c2 = n2;
        c3 = uint32_t(q0);
    }
    return make_uint4(c0, c1, c2, c3);
}

// Gap of the sampling specification: G = #{g in 1..4096 : w < T[g]} for the
// non-increasing table T (T + i holds T[i+1]). A float estimate of
// log((w+1) 2^-32) / log(1-p) lands within one step of the count; the two
// loops then move it to the exact count by comparing against the table, so
// the result never depends on the estimate's rounding.
__device__ __forceinline__ int gap_count(const uint32_t *__restrict__ T, float inv_log2, uint32_t w) {
    const float lg = __log2f(__uint2float_rn(w) + 1.0f) - 32.0f;
    const float est = lg * inv_log2;
    int g = est >= float(kGapLen) ? int(kGapLen) : (est > 0.0f ? int(est) : 0);
    // both neighbours of the estimate at once (T[kGapLen] is in bounds and
    // used only below kGapLen); the loops run only when the estimate is off
    const uint32_t at = __ldg(T + g), below = __ldg(T + (g > 0 ? g - 1 : 0));
    if (g < int(kGapLen) && w < at) {
        g++;
        while (g < int(kGapLen) && w < __ldg(T + g)) g++;
    } else if (g > 0 && w >= below) {
        g--;
        while (g > 0 && w >= __ldg(T + g - 1)) g--;
    }
    return g;
}

// gap_count on a table in shared memory (SMT) or global memory.
template <bool SMT>
__device__ __forceinline__ int gap_count_t(const uint32_t *__restrict__ T, float inv_log2, uint32_t w) {
    if constexpr (!SMT) return gap_count(T, inv_log2, w);
    const float lg = __log2f(__uint2float_rn(w) + 1.0f) - 32.0f;
    const float est = lg * inv_log2;
    int g = est >= float(kGapLen) ? int(kGapLen) : (est > 0.0f ? int(est) : 0);
    // both neighbours of the estimate at once (a table row has more than
    // kGapLen + 1 words, so T[kGapLen] is in bounds; it is used only below
    // kGapLen); the correction loops run only when the estimate is off
    const uint32_t at = T[g], below = T[g > 0 ? g - 1 : 0];
    if (g < int(kGapLen) && w < at) {
        g++;
        while (g < int(kGapLen) && w < T[g]) g++;
    } else if (g > 0 && w >= below) {
        g--;
        while (g > 0 && w >= T[g - 1]) g--;
    }
    return g;
}

// gap_count_t with a cheaper estimate and an early exit: est = log2(w | 1)
// * inv_log2 + c32 (c32 = -32 inv_log2, so est ~ log(w 2^-32) / log(1-p));
// two table reads show whether the estimate g is the count (w < T[g] and
// w >= T[g+1], T + i holding T[i+1]); only lanes where it is not walk to the
// exact count. Same result as gap_count_t for every w.
template <bool SMT>
__device__ __forceinline__ int gap_count_est(const uint32_t *__restrict__ T, float inv_log2, float c32, uint32_t w) {
    auto ld = [&](int i) -> uint32_t {
        if constexpr (SMT) return T[i];
        else return __ldg(T + i);
    };
    const float est = fmaf(__log2f(__uint2float_rn(w | 1u)), inv_log2, c32);
    int g = min(max(__float2int_rz(est), 0), int(kGapLen));
    const uint32_t a = ld(max(g, 1) - 1), b = ld(min(g, int(kGapLen) - 1));
    const bool ge = g == 0 || w < a;              // count >= g
    const bool gt = g < int(kGapLen) && w < b;    // count >= g + 1
    if (ge && !gt) return g;
    if (gt) {
        g++;
        while (g < int(kGapLen) && w < ld(g)) g++;
    } else {
        g--;
        while (g > 0 && w >= ld(g - 1)) g--;
    }
    return g;
}

// Gap count with a single table read, for tables with |inv_log2| below
// kNearInv (p above about 2.1e-5). The count is floor(x) clamped to
// [0, kGapLen] for the real x = (log2(w + 1) - 32) / log2(1 - p), since
// w < floor(2^32 (1-p)^g) holds exactly when g <= x; the host's rounding of
// the table moves that boundary only where x lies within 1e-9 of an integer.
// est = fma(log2f(w + 1), inv_log2, c32) with c32 = -32 inv_log2 (exact in
// float) differs from x by at most
//   |inv| (|log2 error| + 32 * 2^-24) + |x| 2^-24
// where the log2 error is at most 2^-17 + 2^-22.6 (CUDA documents __log2f to
// 2 ulp of a result below 32, or 2^-22.6 absolute on [0.5, 2]; w + 1 is
// formed with two float roundings): below 0.32 + 2.5e-4 for |inv| < 32768.
// So with m = rint(est) the count is m or m - 1, and one comparison with
// T[m] decides (clamping m to [1, kGapLen] keeps the answer right at both
// ends). Same result as gap_count_t for every w of such a table.
constexpr float kNearInv = 32768.0f;

// gap_count_near on the table whose word T[g - 1] sits at tab[base1 + g]
// (base1 = the table's first word index minus one, modulo 2^32), so a
// caller walking many draws of one table forms the base once.
template <bool SMT>
__device__ __forceinline__ int gap_count_near_at(const uint32_t *__restrict__ tab, uint32_t base1, float inv_log2,
                                                 float c32, uint32_t w) {
    const float est = fmaf(__log2f(__uint2float_rn(w) + 1.0f), inv_log2, c32);
    const int m = min(max(__float2int_rn(est), 1), int(kGapLen));
    const uint32_t i = base1 + uint32_t(m);
    uint32_t t;
    if constexpr (SMT) t = tab[i];
    else t = __ldg(tab + i);
    return w < t ? m : m - 1;
}

template <bool SMT>
__device__ __forceinline__ int gap_count_near(const uint32_t *__restrict__ T, float inv_log2, float c32, uint32_t w) {
    return gap_count_near_at<SMT>(T, 0xFFFFFFFFu, inv_log2, c32, w);
}

// The count by one table read where the table allows it, else by the log
// estimate with neighbour loops (per lane: lanes of one warp may differ).
template <bool SMT>
__device__ __forceinline__ int gap_count_fast(const uint32_t *__restrict__ T, float inv_log2, uint32_t w) {
    if (fabsf(inv_log2) < kNearInv) return gap_count_near<SMT>(T, inv_log2, -32.0f * inv_log2, w);
    return gap_count_t<SMT>(T, inv_log2, w);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_shared_volatile(const uint32_t *p) {
    return *reinterpret_cast<const volatile uint32_t *>(p);
}

// Shared-memory accesses with acquire / release ordering at CTA scope (the
// walker/applier hand-offs of the decoupled kernel): cheaper than a full
// fence next to a relaxed access.
__device__ __forceinline__ uint32_t shared_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t ld_acquire_shared(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(shared_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_shared64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.cta.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(shared_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_shared(uint32_t *p, uint32_t v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(shared_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_shared64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.cta.shared::cta.u64 [%0], %1;" ::"r"(shared_addr(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_shared(uint32_t *p, uint32_t v) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(shared_addr(p)), "r"(v) : "memory");
}

// Warp-aggregated shared counter: the calling lane's index among all lanes
// that call together (one atomic per warp).
__device__ __forceinline__ uint32_t grab_index(uint32_t *ctr) {
    const uint32_t mask = __activemask();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t leader = uint32_t(__ffs(mask)) - 1u;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(ctr, uint32_t(__popc(mask)));
    base = __shfl_sync(mask, base, int(leader));
    return base + uint32_t(__popc(mask & ((1u << lane) - 1u)));
}

// 64-bit warp-aggregated counter: the calling lane's index among all lanes
// that call together (one atomic per warp).
__device__ __forceinline__ uint64_t grab_index64(unsigned long long *ctr) {
    const uint32_t mask = __activemask();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t leader = uint32_t(__ffs(mask)) - 1u;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, int(leader));
    return uint64_t(base) + uint64_t(__popc(mask & ((1u << lane) - 1u)));
}

// Pauli indices a noise kind draws from uniformly (PAULI_CHANNEL_1 uses its
// thresholds instead).
__device__ __forceinline__ uint32_t npauli_of(uint32_t kind) {
    return kind == N_DEP2 ? 15u : kind == N_DEP1 ? 3u : 1u;
}

}  // namespace tmcs
