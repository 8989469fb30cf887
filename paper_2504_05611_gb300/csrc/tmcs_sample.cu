// CUDA side of libtmcs (sm_103a): device copies of compiled programs, the
// frame-layer kernel, and the sampling entry points.
//
// Execution model. One CTA owns K consecutive 64-shot chunks (a tile) and
// keeps every live frame component and record of those shots resident in
// shared memory as K uint64 words per slot. It runs the compiled program one
// layer at a time (barrier in between):
//   - clear / XOR / copy layers: one thread per (update, chunk word);
//   - noise layers: one thread per (64-unit segment, chunk); the thread walks
//     that segment's Philox4x32-10 event stream (geometric gaps located in
//     the L1-resident gap table) and XORs each event's Pauli into the frame
//     words of its target (Methods "Simulation" noise channels);
//   - detector layers: one thread per (detector, chunk) XORs its record slots
//     and writes the 64-shot word straight to HBM, detector-major, so
//     consecutive threads store consecutive words of one detector row;
//   - observable layers accumulate into slots written at the end.
// The sampling specification (counter layout, gap tables, Pauli decoding)
// is identical to the CPU oracle's, so outputs match it bit for bit.
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tmcs_device.cuh"
#include "tmcs_internal.h"

namespace tmcs {

// ------------------------------------------------------------ device code

struct KernelArgs {
    const Layer *layers;
    const uint32_t *args;
    const NoiseDesc *noise;
    const uint32_t *tables;
    uint32_t *status;      // device status word (bit 0: a bounded wait expired)
    uint32_t n_layers;
    uint32_t n_slots;
    uint32_t max_window_segs;  // event buffer holds max_window_segs * K units
    uint32_t group_warps;      // frame_kernel_w: warps per chunk group
    uint32_t key0, key1;
    uint32_t first_chunk;  // global chunk of output column 0
    uint64_t n_cols;       // output columns (chunks) of this call
    uint64_t last_mask;    // valid-shot mask of the last column
    uint64_t *det;
    uint64_t *obs;
    // single-fault mode (tmcs_fault_signatures): noise ops inject one fault
    // per lane instead of sampling; lane l of output column c carries fault
    // fault_first + 64 c + l
    const uint64_t *fault_base;
    uint64_t fault_first;
    uint32_t fault_mode;
};

// Buffered events of one (segment, chunk) of a noise op: up to kEvCap events
// as (position in segment: 12 bits | Pauli index << 12); if the walk had more,
// it resumes at draw cont_d from position cont_pos when the op is applied.
struct EvUnit {
    uint16_t ev[kEvCap];
    uint16_t n;
    uint16_t cont_d;  // 0xFFFF: walk complete
    int16_t cont_pos;
    uint16_t pad;
};
static_assert(sizeof(EvUnit) == 24, "EvUnit layout");


// ---- PTX wrappers: mbarrier + bulk asynchronous copy (TMA, 1-D)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase `parity` of `bar`; gives up after kWaitNs of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() - t0 > kWaitNs) return false;
    return true;
}
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void xor_bit(uint64_t *F, uint32_t slot, uint32_t K, int k, unsigned long long bit) {
    if (slot != kDeadSlot) atomicXor(reinterpret_cast<unsigned long long *>(&F[slot * K + k]), bit);
}

// One event of a noise op: Pauli index pk applied to the live frame
// components of the unit's target(s) in lane pos % 64 of chunk word k.
template <int K>
__device__ __forceinline__ void apply_event(uint64_t *F, const uint32_t *__restrict__ tg, uint32_t kind,
                                            uint32_t s, int pos, uint32_t pk, int k) {
    const uint32_t unit = s * kSegUnits + uint32_t(pos >> 6);
    const unsigned long long bit = 1ull << (pos & 63);
    if (kind == N_DEP2) {
        const uint32_t c0 = __ldg(tg + 2 * unit), c1 = __ldg(tg + 2 * unit + 1);
        const uint32_t pa = pk >> 2, pb = pk & 3u;
        if (pa & 1u) xor_bit(F, c0 & 0xFFFFu, K, k, bit);
        if (pa & 2u) xor_bit(F, c0 >> 16, K, k, bit);
        if (pb & 1u) xor_bit(F, c1 & 0xFFFFu, K, k, bit);
        if (pb & 2u) xor_bit(F, c1 >> 16, K, k, bit);
    } else {
        const uint32_t c0 = __ldg(tg + unit);
        const uint32_t pa = kind == N_XERR ? 1u : kind == N_ZERR ? 2u : pk;  // DEPOLARIZE1, PAULI_CHANNEL_1: pk
        if (pa & 1u) xor_bit(F, c0 & 0xFFFFu, K, k, bit);
        if (pa & 2u) xor_bit(F, c0 >> 16, K, k, bit);
    }
}

// Pauli index (x = bit 0, z = bit 1) of an event from its Pauli word.
__device__ __forceinline__ uint32_t pauli_index(const NoiseDesc &nd, uint32_t npauli, uint32_t wp) {
    if (nd.kind == N_PC1) return wp < nd.t1 ? 1u : wp < nd.t2 ? 3u : 2u;
    return 1u + __umulhi(wp, npauli);
}

// Walks draws d = d0, d0+1, ... of one (segment, chunk) stream from position
// pos. With buf != nullptr, events are stored until kEvCap are held (then the
// resume point is recorded); with buf == nullptr they are applied to F.
template <int K>
__device__ __forceinline__ void walk_segment(const NoiseDesc &nd, const uint32_t *__restrict__ T, float inv,
                                             uint32_t s, uint32_t chunk, uint32_t key0, uint32_t key1,
                                             uint32_t d0, int pos, EvUnit *buf, uint64_t *F,
                                             const uint32_t *__restrict__ tg, int k) {
    const int n_trials = 64 * int(min(kSegUnits, nd.n_units - s * kSegUnits));
    const uint32_t npauli = npauli_of(nd.kind);
    uint32_t n = 0;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (uint32_t d = d0;; d++) {
        if (d == d0 || (d & 1u) == 0) w = philox4x32_10(d >> 1, chunk, nd.op_index, s, key0, key1);
        const uint32_t wg = (d & 1u) ? w.z : w.x;
        const uint32_t wp = (d & 1u) ? w.w : w.y;
        const int prev = pos;
        pos += 1 + gap_count_fast<false>(T, inv, wg);
        if (pos >= n_trials) break;
        const uint32_t pk = pauli_index(nd, npauli, wp);
        if (buf) {
            if (n == kEvCap) {
                buf->cont_d = uint16_t(d);
                buf->cont_pos = int16_t(prev);
                buf->n = uint16_t(n);
                return;
            }
            buf->ev[n++] = uint16_t(uint32_t(pos) | (pk << 12));
            prefetch_l1(tg + (nd.kind == N_DEP2 ? 2u : 1u) * (s * kSegUnits + uint32_t(pos >> 6)));
        } else {
            apply_event<K>(F, tg, nd.kind, s, pos, pk, k);
        }
    }
    if (buf) {
        buf->n = uint16_t(n);
        buf->cont_d = 0xFFFFu;
    }
}

// Single-fault mode: every lane of the tile whose fault index falls in this
// noise op's range gets exactly that fault (target unit, Pauli index 1..KP).
template <int K>
__device__ __forceinline__ void inject_faults(uint64_t *F, const KernelArgs &P, uint32_t desc, uint64_t col0,
                                              int nvalid, uint32_t tid, uint32_t nthreads) {
    const NoiseDesc nd = P.noise[desc];
    const uint64_t fb = P.fault_base[desc];
    const uint32_t KP = nd.kind == N_DEP2 ? 15u : (nd.kind == N_DEP1 || nd.kind == N_PC1) ? 3u : 1u;
    const uint64_t fe = fb + uint64_t(nd.n_units) * KP;
    const uint32_t *tg = P.args + nd.tgt_off;
    for (uint32_t i = tid; i < uint32_t(nvalid) * 64u; i += nthreads) {
        const int k = int(i / 64u);
        const uint32_t lane = i % 64u;
        const uint64_t f = P.fault_first + 64ull * (col0 + uint64_t(k)) + lane;
        if (f < fb || f >= fe) continue;
        const uint64_t idx = f - fb;
        const uint32_t unit = uint32_t(idx / KP), pk = uint32_t(idx % KP) + 1u;
        apply_event<K>(F, tg, nd.kind, unit / kSegUnits, int((unit % kSegUnits) * 64u + lane), pk, k);
    }
}

// Runs the whole program for one tile of K chunks starting at output column col0.
//
// Update layers give each thread whole ops: an op's K chunk words of a slot
// are contiguous, so one item moves KV vectors (128-bit when K >= 2). Ops
// are unrolled by U so a thread keeps U*KV independent loads in flight.
template <int K>
__device__ __forceinline__ void run_tile(const KernelArgs P, uint64_t *F, uint32_t *stage0, uint32_t *stage1,
                                         EvUnit *evbuf, uint64_t *bars, int *abort_flag, uint64_t col0,
                                         uint32_t (&parity)[2]) {
    constexpr int V = K >= 2 ? 2 : 1;  // 64-bit words per vector
    constexpr int KV = K / V;          // vectors per slot
    constexpr int U = KV >= 4 ? 1 : 4 / KV;  // ops per unrolled step
    using VecT = typename std::conditional<V == 2, ulonglong2, unsigned long long>::type;
    VecT *Fv = reinterpret_cast<VecT *>(F);
    const uint64_t rem = P.n_cols - col0;
    const int nvalid = rem < uint64_t(K) ? int(rem) : K;
    const uint32_t chunk0 = P.first_chunk + uint32_t(col0);
    const uint32_t T_ = blockDim.x, tid = threadIdx.x;

    auto issue = [&](uint32_t L) {
        if (tid == 0 && L < P.n_layers) {
            const Layer ly = P.layers[L];
            if (ly.nwords) {
                uint32_t *dst = (L & 1u) ? stage1 : stage0;
                fence_proxy_async();
                mbar_arrive_expect_tx(&bars[L & 1u], ly.nwords * 4u);
                bulk_copy_g2s(dst, P.args + ly.off, ly.nwords * 4u, &bars[L & 1u]);
            }
        }
    };
    issue(0);
    for (uint32_t L = 0; L < P.n_layers; L++) {
        const Layer ly = P.layers[L];
        issue(L + 1);
        const uint32_t *st = (L & 1u) ? stage1 : stage0;
        bool ready = true;
        if (ly.nwords) {
            ready = mbar_wait_bounded(&bars[L & 1u], parity[L & 1u]);
            parity[L & 1u] ^= 1u;
            if (!ready) *abort_flag = 1;
        }
        if (ready) {
            switch (ly.kind) {
            case L_ZERO: {
                VecT z;
                if constexpr (V == 2) z = make_ulonglong2(0ull, 0ull); else z = 0ull;
                for (uint32_t i = tid; i < ly.count; i += T_) {
                    VecT *d = Fv + st[i] * KV;
#pragma unroll
                    for (int v = 0; v < KV; v++) d[v] = z;
                }
                break;
            }
            case L_XOR:
            case L_COPY: {
                const uint32_t n = ly.count;
                const bool is_xor = ly.kind == L_XOR;
                for (uint32_t i0 = tid; i0 < n; i0 += U * T_) {
                    uint32_t dsl[U], ssl[U];
                    bool ok[U];
#pragma unroll
                    for (int r = 0; r < U; r++) {
                        const uint32_t i = i0 + uint32_t(r) * T_;
                        ok[r] = i < n;
                        const uint32_t w = ok[r] ? st[i] : 0u;
                        dsl[r] = (w & 0xFFFFu) * KV;
                        ssl[r] = (w >> 16) * KV;
                    }
                    VecT a[U][KV], b[U][KV];
#pragma unroll
                    for (int r = 0; r < U; r++)
                        if (ok[r]) {
#pragma unroll
                            for (int v = 0; v < KV; v++) {
                                b[r][v] = Fv[ssl[r] + v];
                                if (is_xor) a[r][v] = Fv[dsl[r] + v];
                            }
                        }
#pragma unroll
                    for (int r = 0; r < U; r++)
                        if (ok[r]) {
#pragma unroll
                            for (int v = 0; v < KV; v++) {
                                if constexpr (V == 2) {
                                    Fv[dsl[r] + v] = is_xor ? make_ulonglong2(a[r][v].x ^ b[r][v].x, a[r][v].y ^ b[r][v].y)
                                                            : b[r][v];
                                } else {
                                    Fv[dsl[r] + v] = is_xor ? (a[r][v] ^ b[r][v]) : b[r][v];
                                }
                            }
                        }
                }
                break;
            }
            case L_NGEN: {
                const uint32_t units = P.fault_mode ? 0u : ly.aux2 * K;
                for (uint32_t u = tid; u < units; u += T_) {
                    const uint32_t ws = u / K;
                    const int k = int(u % K);
                    uint32_t di = ly.aux, base = 0;
                    uint32_t nseg = P.noise[di].n_seg;
                    while (ws >= base + nseg) {
                        base += nseg;
                        nseg = P.noise[++di].n_seg;
                    }
                    EvUnit *E = evbuf + u;
                    if (k >= nvalid) {
                        E->n = 0;
                        E->cont_d = 0xFFFFu;
                        continue;
                    }
                    const NoiseDesc nd = P.noise[di];
                    const uint32_t *Tt = P.tables + size_t(nd.table) * kTableWords;
                    const float inv = __uint_as_float(__ldg(Tt + kGapLen));
                    walk_segment<K>(nd, Tt, inv, ws - base, chunk0 + uint32_t(k), P.key0, P.key1, 0u, -1, E,
                                    nullptr, P.args + nd.tgt_off, k);
                }
                break;
            }
            case L_NAPPLY: {
                if (P.fault_mode) {
                    inject_faults<K>(F, P, ly.aux, col0, nvalid, tid, T_);
                    break;
                }
                const NoiseDesc nd = P.noise[ly.aux];
                const uint32_t *tg = P.args + nd.tgt_off;
                const uint32_t items = nd.n_seg * K * kEvCap;
                for (uint32_t i = tid; i < items; i += T_) {
                    const uint32_t uu = i / kEvCap, e = i % kEvCap;
                    const uint32_t s = uu / K;
                    const int k = int(uu % K);
                    if (k >= nvalid) continue;
                    const EvUnit *E = evbuf + (ly.aux2 + s) * K + uint32_t(k);
                    if (e < E->n) {
                        const uint32_t v = E->ev[e];
                        apply_event<K>(F, tg, nd.kind, s, int(v & 0xFFFu), v >> 12, k);
                    }
                    if (e == 0 && E->cont_d != 0xFFFFu) {
                        const uint32_t *Tt = P.tables + size_t(nd.table) * kTableWords;
                        const float inv = __uint_as_float(__ldg(Tt + kGapLen));
                        walk_segment<K>(nd, Tt, inv, s, chunk0 + uint32_t(k), P.key0, P.key1, E->cont_d,
                                        E->cont_pos, nullptr, F, tg, k);
                    }
                }
                break;
            }
            case L_DET: {
                for (uint32_t d = tid; d < ly.count; d += T_) {
                    const uint32_t lo = st[d], hi = st[d + 1];
                    VecT v[KV];
#pragma unroll
                    for (int q = 0; q < KV; q++) {
                        if constexpr (V == 2) v[q] = make_ulonglong2(0ull, 0ull); else v[q] = 0ull;
                    }
                    for (uint32_t t = lo; t < hi; t++) {
                        const VecT *x = Fv + st[t] * KV;
#pragma unroll
                        for (int q = 0; q < KV; q++) {
                            if constexpr (V == 2) {
                                const VecT y = x[q];
                                v[q].x ^= y.x;
                                v[q].y ^= y.y;
                            } else {
                                v[q] ^= x[q];
                            }
                        }
                    }
                    uint64_t *out = P.det + uint64_t(ly.aux + d) * P.n_cols + col0;
                    const bool full = nvalid == K && col0 + K != P.n_cols;
                    if (full && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
#pragma unroll
                        for (int q = 0; q < KV; q++) reinterpret_cast<VecT *>(out)[q] = v[q];
                    } else {
#pragma unroll
                        for (int q = 0; q < KV; q++) {
#pragma unroll
                            for (int h = 0; h < V; h++) {
                                const int k = q * V + h;
                                uint64_t w;
                                if constexpr (V == 2) w = h ? v[q].y : v[q].x; else w = v[q];
                                if (k < nvalid)
                                    out[k] = (col0 + uint64_t(k) == P.n_cols - 1) ? (w & P.last_mask) : w;
                            }
                        }
                    }
                }
                break;
            }
            case L_OBS: {
                const uint32_t n = ly.count * K;
                for (uint32_t i = tid; i < n; i += T_) {
                    const uint32_t d = i / K;
                    const int k = int(i % K);
                    const uint32_t b = st[d], e = st[d + 1];
                    uint64_t v = 0;
                    for (uint32_t t = b + 1; t < e; t++) v ^= F[st[t] * K + k];
                    F[st[b] * K + k] ^= v;
                }
                break;
            }
            case L_OBSOUT: {
                const uint32_t n = ly.count * K;
                for (uint32_t i = tid; i < n; i += T_) {
                    const uint32_t o = i / K;
                    const int k = int(i % K);
                    if (k >= nvalid) continue;
                    uint64_t v = F[st[o] * K + k];
                    const uint64_t col = col0 + uint64_t(k);
                    if (col == P.n_cols - 1) v &= P.last_mask;
                    P.obs[uint64_t(o) * P.n_cols + col] = v;
                }
                break;
            }
            case L_GAUGE: {
                // slot ^= gauge word of (op, target u, chunk): Philox at
                // counter (u / 2, chunk, op, 2^31); even u takes w0 | w1 << 32,
                // odd u takes w2 | w3 << 32
                const uint32_t n = ly.count * K;
                for (uint32_t i = tid; i < n; i += T_) {
                    const uint32_t g = i / K;
                    const int k = int(i % K);
                    if (k >= nvalid) continue;
                    const uint32_t slot = st[3 * g], op = st[3 * g + 1], u = st[3 * g + 2];
                    const uint4 w = philox4x32_10(u >> 1, chunk0 + uint32_t(k), op, 0x80000000u, P.key0, P.key1);
                    const uint64_t word = (u & 1u) ? (uint64_t(w.z) | (uint64_t(w.w) << 32))
                                                   : (uint64_t(w.x) | (uint64_t(w.y) << 32));
                    F[slot * K + k] ^= word;
                }
                break;
            }
            case L_RECOUT: {
                // record r = reference bit XOR frame bit, one row per record
                const uint32_t n = ly.count * K;
                for (uint32_t i = tid; i < n; i += T_) {
                    const uint32_t g = i / K;
                    const int k = int(i % K);
                    if (k >= nvalid) continue;
                    const uint32_t w0 = st[2 * g], r = st[2 * g + 1];
                    uint64_t v = F[(w0 & 0x7FFFFFFFu) * K + k];
                    if (w0 >> 31) v = ~v;
                    const uint64_t col = col0 + uint64_t(k);
                    if (col == P.n_cols - 1) v &= P.last_mask;
                    P.det[uint64_t(r) * P.n_cols + col] = v;
                }
                break;
            }
            default:
                break;
            }
        }
        __syncthreads();
        if (*abort_flag) {
            // a staging copy never arrived: wait (bounded) for the one still in
            // flight, record the failure and leave together
            if (tid == 0) {
                if (L + 1 < P.n_layers && P.layers[L + 1].nwords)
                    mbar_wait_bounded(&bars[(L + 1) & 1u], parity[(L + 1) & 1u]);
                atomicOr(P.status, 1u);
            }
            return;
        }
    }
}

template <int K>
__global__ void __launch_bounds__(512) frame_kernel(const KernelArgs P) {
    extern __shared__ __align__(128) uint64_t smem[];
    uint64_t *F = smem;
    uint8_t *base = reinterpret_cast<uint8_t *>(smem) + ((size_t(P.n_slots) * K * 8 + 127) & ~size_t(127));
    uint32_t *stage0 = reinterpret_cast<uint32_t *>(base);
    uint32_t *stage1 = stage0 + kStageWords;
    EvUnit *evbuf = reinterpret_cast<EvUnit *>(stage1 + kStageWords);
    // same layout as kernel_smem_bytes(n_slots, max_window_segs, K)
    uint64_t *bars = reinterpret_cast<uint64_t *>(evbuf + size_t(P.max_window_segs) * K);
    int *abort_flag = reinterpret_cast<int *>(bars + 2);
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    run_tile<K>(P, F, stage0, stage1, evbuf, bars, abort_flag, uint64_t(blockIdx.x) * K, parity);
}

// ---------------------------------------------------------------------------
// Event-signature kernel: samples the same noise streams as the frame kernels
// and, instead of running the Clifford layers, XORs each event's precomputed
// output list (the XOR of its generators' lists) into a shared-memory ring of
// detector words. Bit-identical to the frame kernels because detector flips
// are linear in the events (see tmcs_signature.cpp).
//
// A CTA owns K chunks at a time (persistent over tiles). Per step it walks
// the step's (segment, chunk) streams, one per thread, applying events with
// 32-bit shared atomics (lanes 0-31 in the low word, 32-63 in the high word),
// then writes and clears the detectors that the step finalised. Observables
// accumulate in a small array written once per tile.

struct SigArgs {
    const NoiseDesc *noise;   // tgt_off = the descriptor's first event slot
    const uint32_t *tables;
    const uint4 *item_rec;    // per item: op index, segment, first event slot, kind | table << 3 | (units-1) << 16 | desc << 22
    const uint4 *steps;       // SigStep: item_begin, item_end, flush_lo, flush_hi
    const uint32_t *ev_ent;   // two words per event slot (see SigProgram), then the overflow lists
    uint32_t n_steps;
    uint32_t window_mask;     // ring size - 1 (power of two)
    uint32_t n_obs;
    uint32_t queue_cap;       // events the shared queue holds
    uint32_t smem_tables;     // gap tables copied to shared memory (0, or all of them)
    uint32_t stage_items;     // shared staging buffer for a step's item records (0: read them from global)
    uint32_t key0, key1;
    uint32_t first_chunk;
    uint64_t n_cols, last_mask, n_tiles;
    uint64_t *det;
    uint64_t *obs;
    // pipelined kernel only
    uint32_t lag;             // steps in flight (> 0)
    uint32_t n_items;         // item records of the schedule
    uint32_t n_det;           // detectors (tile T's ring offset is T * n_det)
    uint32_t vec_out;         // det is 16-byte aligned and n_cols even: 16-byte output stores
    uint32_t *status;         // device status word (bit 0: a bounded wait expired)
    uint32_t stall_flush;     // testing: the flusher waits for one stream more than step 0 has
                              // (a count nothing reaches), so its bounded wait expires
};

// Draws of one (segment, chunk) stream from its start; sink(pos, pauli) per
// event, in stream order (the sampling specification's walk).
template <class Sink>
__device__ __forceinline__ void walk_stream(const NoiseDesc &nd, const uint32_t *__restrict__ T, float inv,
                                            uint32_t s, uint32_t chunk, uint32_t key0, uint32_t key1,
                                            Sink &&sink) {
    const int n_trials = 64 * int(min(kSegUnits, nd.n_units - s * kSegUnits));
    const uint32_t npauli = npauli_of(nd.kind);
    int pos = -1;
    uint4 w = make_uint4(0, 0, 0, 0);
    for (uint32_t d = 0;; d++) {
        if ((d & 1u) == 0) w = philox4x32_10(d >> 1, chunk, nd.op_index, s, key0, key1);
        const uint32_t wg = (d & 1u) ? w.z : w.x;
        const uint32_t wp = (d & 1u) ? w.w : w.y;
        pos += 1 + gap_count_fast<false>(T, inv, wg);
        if (pos >= n_trials) break;
        sink(pos, pauli_index(nd, npauli, wp));
    }
}

// Queued events: event slot index (low word), and lane | chunk k << 6 (4
// bits, K <= 16) | ring offset << 16 | observable buffer << 30 (high word;
// the last two are zero in the barrier kernel; bits 10-15 are not read here). A thread
// applies up to N at once, all N slot loads issued before any is used so
// their latencies overlap.
template <int N>
__device__ __forceinline__ void sig_apply_events(const SigArgs &A, const uint64_t (&q)[N], int n, uint64_t *ring,
                                                 uint64_t *oacc, int K) {
    uint2 v[N];
#pragma unroll
    for (int j = 0; j < N; j++)
        v[j] = j < n ? __ldg(reinterpret_cast<const uint2 *>(A.ev_ent) + uint32_t(q[j])) : make_uint2(kEvNone, kEvNone);
#pragma unroll
    for (int j = 0; j < N; j++) {
        if (v[j].x == kEvNone) continue;
        const uint32_t hi = uint32_t(q[j] >> 32);
        const uint32_t lane = hi & 63u, k = (hi >> 6) & 15u;
        const uint32_t roff = (hi >> 16) & 0x3FFFu;
        // the observable accumulators follow the ring in shared memory, so
        // an entry becomes one word row: detector d at (d + roff) mod W,
        // observable o of buffer b at W + b * n_obs + o
        unsigned int *ring32 = reinterpret_cast<unsigned int *>(ring + k) + (lane >> 5);
        const uint32_t obase = A.window_mask + 1u + ((hi >> 30) & 1u) * A.n_obs;
        const uint32_t bit = 1u << (lane & 31u);
        auto put = [&](uint32_t w) {
            const uint32_t idx = w & 0x1FFFFFFFu;
            const uint32_t row = (w & (1u << 29)) ? obase + idx : ((idx + roff) & A.window_mask);
            atomicXor(ring32 + size_t(row) * 2 * K, bit);
        };
        if (v[j].x & kEvOverflow) {
            const uint32_t *ov = A.ev_ent + (v[j].x & ~kEvOverflow);
            for (uint32_t x = 0; x < v[j].y; x++) put(__ldg(ov + x));
        } else {
            put(v[j].x);
            if (v[j].y != kEvNone) put(v[j].y);
        }
    }
}


// Applies the n events of a warp's queue slice, converged: lane l takes
// events l, l + 32, ... N at a time. Called by all 32 lanes.
template <int N = 4>
__device__ __forceinline__ void sig_warp_apply(const SigArgs &A, const uint64_t *wq, uint32_t n, uint64_t *ring,
                                               uint64_t *oacc, int K) {
    __syncwarp();
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t e0 = lane; e0 < n; e0 += 32u * N) {
        uint64_t qb[N];
        int nb = 0;
#pragma unroll
        for (int j = 0; j < N; j++) {
            const uint32_t e = e0 + 32u * uint32_t(j);
            qb[j] = e < n ? wq[e] : 0ull;
            nb += e < n ? 1 : 0;
        }
        sig_apply_events<N>(A, qb, nb, ring, oacc, K);
    }
    __syncwarp();
}

// events a lane applies at once when a warp's queue slice fills during the
// walk (the walk's state stays live across it)
#ifndef TMCS_WALK_APPLY
#define TMCS_WALK_APPLY 2
#endif
constexpr int kWalkApply = TMCS_WALK_APPLY;

// Walk phase of one step for one warp: every lane holds one (segment, chunk)
// stream and runs one Philox call (two draws) of it per iteration; a lane
// whose stream ends takes the next from the step's counter, so the warp stays
// converged on the generator. Events go to the warp's own queue slice at
// offsets from a ballot (no atomics); when the slice would overflow, the
// warp first applies it together and starts it again. Returns the number of
// queued events.
// tabs: the gap tables, in shared memory when SMT.
template <bool SMT>
__device__ __forceinline__ uint32_t sig_walk(const SigArgs &A, const uint4 st, uint32_t n, uint32_t nvalid,
                                             uint32_t chunk0, const uint32_t *tabs, const uint4 *sitems,
                                             uint64_t *wq, uint32_t wcap, uint32_t *s_next, uint64_t *ring,
                                             uint64_t *oacc, int K) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t qn = 0;  // events in the slice (warp-uniform)
    bool have = false, exhausted = false;
    uint32_t call = 0, seg = 0, op = 0, kind = 0, chunk = 0, ubase = 0, tag = 0, t1 = 0, t2 = 0, npauli = 1, kp = 1;
    int pos = -1, n_trials = 0;
    const uint32_t *Tt = tabs;
    float inv = 0.f;
    for (;;) {
        if (!have && !exhausted) {
            const uint32_t i = grab_index(s_next);
            exhausted = i >= n;
            if (i < n) {
                const uint32_t il = i / nvalid;
                const uint32_t k = i % nvalid;
                const uint4 rec = sitems ? sitems[il] : __ldg(A.item_rec + st.x + il);
                kind = rec.w & 7u;
                Tt = tabs + size_t((rec.w >> 3) & 0x1FFFu) * kTableWords;
                inv = __uint_as_float(Tt[kGapLen]);
                seg = rec.y;
                op = rec.x;
                if (kind == N_PC1) {
                    t1 = A.noise[rec.w >> 22].t1;
                    t2 = A.noise[rec.w >> 22].t2;
                }
                npauli = npauli_of(kind);
                kp = sig_paulis(kind);
                chunk = chunk0 + k;
                ubase = rec.z;
                tag = k << 6;
                n_trials = 64 * int(((rec.w >> 16) & 63u) + 1u);
                call = 0;
                pos = -1;
                have = true;
            }
        }
        if (!__any_sync(0xFFFFFFFFu, have)) break;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (have) w = philox4x32_10(call, chunk, op, seg, A.key0, A.key1);
        call++;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            bool ev = false;
            uint64_t q = 0;
            if (have) {
                const uint32_t wg = h ? w.z : w.x, wp = h ? w.w : w.y;
                pos += 1 + gap_count_fast<SMT>(Tt, inv, wg);
                if (pos >= n_trials) {
                    have = false;
                } else {
                    const uint32_t pk = kind == N_PC1 ? (wp < t1 ? 1u : wp < t2 ? 3u : 2u)
                                                      : 1u + __umulhi(wp, npauli);
                    q = uint64_t(ubase + uint32_t(pos >> 6) * kp + (pk - 1u)) | (uint64_t(tag | uint32_t(pos & 63)) << 32);
                    ev = true;
                }
            }
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, ev);
            if (m) {
                const uint32_t c = uint32_t(__popc(m));
                if (qn + c > wcap) {
                    // slice full: the warp applies it together (slot loads
                    // overlapped) and starts it again
                    sig_warp_apply<kWalkApply>(A, wq, qn, ring, oacc, K);
                    qn = 0;
                }
                if (ev) wq[qn + uint32_t(__popc(m & lt))] = q;
                qn += c;
            }
        }
    }
    return qn;
}

// Shared-memory regions of one circuit's layout (same order and sizes as
// sig_smem_bytes): detector ring, observables (padded to 16 bytes), gap
// tables, staged item records, event queue.
struct SigSmem {
    uint64_t *ring, *oacc;
    uint32_t *stab;
    uint4 *sitems_buf;
    uint64_t *queue;
};

__device__ __forceinline__ SigSmem sig_layout(uint64_t *smem, const SigArgs &A, int K) {
    SigSmem S;
    const size_t W = size_t(A.window_mask) + 1;
    S.ring = smem;
    S.oacc = smem + W * K;
    S.stab = reinterpret_cast<uint32_t *>(smem + (((W + A.n_obs) * K + 1) & ~size_t(1)));
    S.sitems_buf = reinterpret_cast<uint4 *>(S.stab + size_t(A.smem_tables) * kTableWords);
    S.queue = reinterpret_cast<uint64_t *>(S.sitems_buf + A.stage_items);
    return S;
}

// Clears the ring and observables and loads the gap tables of circuit A
// (all threads; ends with a barrier).
template <int K>
__device__ __forceinline__ void sig_setup(const SigArgs &A, const SigSmem &S) {
    const uint32_t T_ = blockDim.x, tid = threadIdx.x;
    const uint32_t W = A.window_mask + 1u;
    for (uint32_t i = tid; i < (W + A.n_obs) * K; i += T_) S.ring[i] = 0ull;
    for (uint32_t i = tid; i < A.smem_tables * kTableWords; i += T_) S.stab[i] = __ldg(A.tables + i);
    __syncthreads();
}

// One tile of K chunks, all threads. Per step: (1) every warp walks
// (segment, chunk) streams taken from a shared counter and queues its events
// in its own slice of the queue; (2) every warp applies its slice; (3) after
// a barrier the step's final detectors are written out and cleared. Leaves
// the ring, the observables and the counter clean for the next tile.
template <int K>
__device__ __forceinline__ void sig_tile(const SigArgs &A, const SigSmem &S, uint64_t tile, uint32_t *s_next) {
    const uint32_t T_ = blockDim.x, tid = threadIdx.x;
    const uint32_t W = A.window_mask + 1u;
    const uint32_t wcap = A.queue_cap / (T_ >> 5);  // queue slice per warp
    const uint4 *sitems = A.stage_items ? S.sitems_buf : nullptr;
    const uint64_t col0 = tile * K;
    const uint64_t rem = A.n_cols - col0;
    const int nvalid = rem < uint64_t(K) ? int(rem) : K;
    const uint32_t chunk0 = A.first_chunk + uint32_t(col0);
    if (A.stage_items) {
        const uint4 s0 = __ldg(A.steps);
        for (uint32_t i = tid; i < s0.y - s0.x; i += T_) S.sitems_buf[i] = __ldg(A.item_rec + s0.x + i);
        __syncthreads();
    }
    for (uint32_t si = 0; si < A.n_steps; si++) {
        const uint4 st = __ldg(A.steps + si);
        const uint32_t n = (st.y - st.x) * uint32_t(nvalid);
        uint64_t *wq = S.queue + size_t(tid >> 5) * wcap;
        const uint32_t left =
            A.smem_tables
                ? sig_walk<true>(A, st, n, uint32_t(nvalid), chunk0, S.stab, sitems, wq, wcap, s_next, S.ring, S.oacc, K)
                : sig_walk<false>(A, st, n, uint32_t(nvalid), chunk0, A.tables, sitems, wq, wcap, s_next, S.ring,
                                  S.oacc, K);
        sig_warp_apply(A, wq, left, S.ring, S.oacc, K);
        __syncthreads();
        if (tid == 0) *s_next = 0;
        const uint32_t nf = (st.w - st.z) * K;
        for (uint32_t i = tid; i < nf; i += T_) {
            const uint32_t d = st.z + i / K;
            const int k = int(i % K);
            if (k >= nvalid) continue;
            uint64_t v = 0ull;
            if (d - st.z < W) {
                uint64_t *r = S.ring + size_t(d & A.window_mask) * K + k;
                v = *r;
                *r = 0ull;
            }
            const uint64_t col = col0 + uint64_t(k);
            if (col == A.n_cols - 1) v &= A.last_mask;
            __stcs(reinterpret_cast<unsigned long long *>(A.det + uint64_t(d) * A.n_cols + col), v);
        }
        if (A.stage_items && si + 1 < A.n_steps) {
            const uint4 s1 = __ldg(A.steps + si + 1);
            for (uint32_t i = tid; i < s1.y - s1.x; i += T_) S.sitems_buf[i] = __ldg(A.item_rec + s1.x + i);
        }
        __syncthreads();
    }
    for (uint32_t i = tid; i < A.n_obs * K; i += T_) {
        const uint32_t o = i / K;
        const int k = int(i % K);
        uint64_t v = S.oacc[i];
        S.oacc[i] = 0ull;
        if (k >= nvalid) continue;
        const uint64_t col = col0 + uint64_t(k);
        if (col == A.n_cols - 1) v &= A.last_mask;
        A.obs[uint64_t(o) * A.n_cols + col] = v;
    }
    __syncthreads();
}

// One circuit: persistent CTAs take tiles blockIdx.x, blockIdx.x + gridDim.x, ...
template <int K>
__global__ void __launch_bounds__(1024) sig_kernel(const SigArgs A) {
    extern __shared__ __align__(128) uint64_t smem[];
    __shared__ uint32_t s_next;
    const SigSmem S = sig_layout(smem, A, K);
    if (threadIdx.x == 0) s_next = 0;
    sig_setup<K>(A, S);
    for (uint64_t tile = blockIdx.x; tile < A.n_tiles; tile += gridDim.x) sig_tile<K>(A, S, tile, &s_next);
}

// ---------------------------------------------------------------------------
// Pipelined event-signature kernel: the walk and the event application of
// sig_kernel without CTA barriers. The last warp of the CTA flushes; the
// others walk. Walkers take (tile, step, item, chunk) streams in CTA order
// from one shared counter, across step and tile boundaries; a stream of
// step q (counted over the CTA's tiles) starts once steps < q + 1 - lag are
// flushed, so at most `lag` steps are in flight and the ring (sized for any
// lag consecutive steps by the schedule builder) never holds two live
// detectors in one slot. A walker counts its finished streams per step and
// publishes the counts after applying its queued events; the flusher waits
// for step q's count to reach its stream total, writes and clears the
// detectors step q finalised (and the tile's observables after its last
// step), stages the item records of step q + lag, then advances `flushed`.
// Tile T's detector d lives in ring slot (T * n_det + d) mod ring, its
// observables in buffer T mod 2. Every wait is bounded (kWaitNs); on expiry
// the kernel sets the status bit and every warp leaves.

// events a walker lane applies per pass (build-time tuning value): the
// walk's state stays live across the apply, and batches of 2 or 4 measured
// slower than 1 on every workload
#ifndef TMCS_PIPE_APPLY
#define TMCS_PIPE_APPLY 1
#endif
constexpr int kPipeApply = TMCS_PIPE_APPLY;

struct PipeCtl {
    unsigned long long next;          // streams handed out
    uint32_t flushed;                 // steps flushed
    uint32_t abort;                   // a bounded wait expired
    uint32_t done[kSigMaxLag];        // published finished streams of step q (slot q mod lag)
    uint32_t wdone[32 * kSigMaxLag];  // per warp: finished streams not yet published
};

struct PipeSmem {
    uint64_t *ring, *oacc;
    uint32_t *stab;
    uint4 *sitems;
    uint64_t *queue;
};

// Same order and sizes as sig_smem_bytes for a pipelined schedule: ring,
// two observable buffers (padded to 16 bytes), gap tables, lag staging
// buffers of item records, event queue.
__device__ __forceinline__ PipeSmem pipe_layout(uint64_t *smem, const SigArgs &A, int K) {
    PipeSmem S;
    const size_t W = size_t(A.window_mask) + 1;
    S.ring = smem;
    S.oacc = smem + W * K;
    S.stab = reinterpret_cast<uint32_t *>(smem + (((W + 2 * size_t(A.n_obs)) * K + 1) & ~size_t(1)));
    S.sitems = reinterpret_cast<uint4 *>(S.stab + size_t(A.smem_tables) * kTableWords);
    S.queue = reinterpret_cast<uint64_t *>(S.sitems + size_t(A.stage_items) * A.lag);
    return S;
}

// Adds this warp's finished-stream counts to the step totals. All 32 lanes;
// every event of those streams has been applied by this warp before. The
// queue slice of a walker warp holds at least 64 events (two ballots).
__device__ __forceinline__ void pipe_publish(PipeCtl &C, uint32_t warp, uint32_t lag) {
    __syncwarp();
    const uint32_t lane = threadIdx.x & 31u;
    if (lane < lag) {
        const uint32_t v = C.wdone[warp * kSigMaxLag + lane];
        if (v) {
            C.wdone[warp * kSigMaxLag + lane] = 0;
            __threadfence_block();
            atomicAdd(&C.done[lane], v);
        }
    }
    __syncwarp();
}

template <bool SMT, int K>
__device__ __forceinline__ void pipe_walk(const SigArgs &A, const PipeSmem &S, PipeCtl &C, uint32_t nt,
                                          uint32_t nv_last, const uint32_t *tabs) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t lag = A.lag, n_steps = A.n_steps;
    const uint32_t wcap = A.queue_cap / ((blockDim.x >> 5) - 1u);
    uint64_t *wq = S.queue + size_t(warp) * wcap;
    const uint64_t per_tile = uint64_t(A.n_items) * K;
    const uint64_t total = uint64_t(nt - 1) * per_tile + uint64_t(A.n_items) * nv_last;
    uint32_t qn = 0, unpub = 0;  // warp-uniform
    bool have = false, pend = false, exhausted = false, waiting = false;
    // the lane's stream: Philox counter words (call, chunk, op, seg), first
    // event slot of the segment, event tag (chunk k, kind, ring offset,
    // observable buffer), gap table (word offset), position and length in
    // trials
    uint32_t call = 0, seg = 0, op = 0, chunk = 0, ubase = 0, tag = 0, toff = 0, t1 = 0, t2 = 0;
    int pos = -1, n_trials = 0;
    float inv = 0.f;
    // cursor over the CTA's tiles and steps; pq = the grabbed stream's index
    // within tile curT (valid while pend, and its step is curS)
    uint32_t curT = 0xFFFFFFFFu, curS = 0, ring_off = 0, pq = 0, t_wait = 0;
    uint64_t tbase = 0;
    for (;;) {
        if (!have && !pend && !exhausted) {
            const uint64_t p = grab_index64(&C.next);
            if (p >= total || ld_shared_volatile(&C.abort)) {
                exhausted = true;
            } else {
                if (curT == 0xFFFFFFFFu || p - tbase >= per_tile) {
                    curT = uint32_t(p / per_tile);
                    tbase = uint64_t(curT) * per_tile;
                    curS = 0;
                    ring_off = uint32_t((uint64_t(curT) * A.n_det) & A.window_mask);
                }
                pq = uint32_t(p - tbase);
                const uint32_t nv = curT == nt - 1 ? nv_last : uint32_t(K);
                const uint32_t il = nv == uint32_t(K) ? pq / uint32_t(K) : pq / nv;
                while (il >= __ldg(&A.steps[curS].y)) curS++;
                pend = true;
            }
        }
        if (pend && curT * n_steps + curS < ld_shared_volatile(&C.flushed) + lag) {
            __threadfence_block();  // the flusher's clears of the ring precede this stream's events
            const uint32_t nv = curT == nt - 1 ? nv_last : uint32_t(K);
            uint32_t il, k;
            if (nv == uint32_t(K)) {
                il = pq / uint32_t(K);
                k = pq % uint32_t(K);
            } else {
                il = pq / nv;
                k = pq - il * nv;
            }
            const uint32_t seq = curT * n_steps + curS;
            const uint4 rec = A.stage_items
                                  ? S.sitems[size_t(seq % lag) * A.stage_items + (il - __ldg(&A.steps[curS].x))]
                                  : __ldg(A.item_rec + il);
            const uint32_t kind = rec.w & 7u;
            toff = ((rec.w >> 3) & 0x1FFFu) * kTableWords;
            inv = __uint_as_float(tabs[toff + kGapLen]);
            seg = rec.y;
            op = rec.x;
            if (kind == N_PC1) {
                t1 = A.noise[rec.w >> 22].t1;
                t2 = A.noise[rec.w >> 22].t2;
            }
            const uint64_t col = (uint64_t(blockIdx.x) + uint64_t(curT) * gridDim.x) * K + k;
            chunk = A.first_chunk + uint32_t(col);
            ubase = rec.z;
            tag = (k << 6) | (kind << 13) | (ring_off << 16) | ((curT & 1u) << 30);
            n_trials = 64 * int(((rec.w >> 16) & 63u) + 1u);
            call = 0;
            pos = -1;
            have = true;
            pend = false;
        }
        const uint32_t act = __ballot_sync(0xFFFFFFFFu, have);
        const uint32_t gated = __ballot_sync(0xFFFFFFFFu, pend);
        // apply the queue and publish the finished streams (one place, so the
        // apply code is inlined once): when this iteration's events (at most
        // 64) might not fit, when lanes wait for a flush that may need this
        // warp's counts, and before leaving
        if (qn + 64u > wcap || (gated && unpub) || (!act && (qn || unpub))) {
            if (qn) sig_warp_apply<kPipeApply>(A, wq, qn, S.ring, S.oacc, K);
            qn = 0;
            if (unpub) pipe_publish(C, warp, lag);
            unpub = 0;
        }
        if (!act) {
            if (!gated) break;
            // every live lane waits for a flush: back off (bounded)
            if (!waiting) {
                t_wait = uint32_t(globaltimer_ns());
                waiting = true;
            } else if (__any_sync(0xFFFFFFFFu, uint32_t(globaltimer_ns()) - t_wait > uint32_t(kWaitNs) ||
                                                   ld_shared_volatile(&C.abort))) {
                // the whole warp leaves together
                if (lane == 0 && !ld_shared_volatile(&C.abort)) {
                    C.abort = 1u;
                    atomicOr(A.status, 1u);
                }
                return;
            }
            __nanosleep(128);
            continue;
        }
        waiting = false;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (have) w = philox4x32_10(call, chunk, op, seg, A.key0, A.key1);
        call++;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            bool ev = false, fin = false;
            uint64_t q = 0;
            if (have) {
                const uint32_t wg = h ? w.z : w.x, wp = h ? w.w : w.y;
                pos += 1 + gap_count_fast<SMT>(tabs + toff, inv, wg);
                if (pos >= n_trials) {
                    have = false;
                    fin = true;
                } else {
                    const uint32_t kind = (tag >> 13) & 7u;
                    const uint32_t pauli = kind == N_PC1 ? (wp < t1 ? 1u : wp < t2 ? 3u : 2u)
                                                         : 1u + __umulhi(wp, npauli_of(kind));
                    q = uint64_t(ubase + uint32_t(pos >> 6) * sig_paulis(kind) + (pauli - 1u)) |
                        (uint64_t(tag | uint32_t(pos & 63)) << 32);
                    ev = true;
                }
            }
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, ev);
            if (ev) wq[qn + uint32_t(__popc(m & lt))] = q;
            qn += uint32_t(__popc(m));
            const uint32_t f = __ballot_sync(0xFFFFFFFFu, fin);
            if (fin) atomicAdd(&C.wdone[warp * kSigMaxLag + (curT * n_steps + curS) % lag], 1u);
            unpub += uint32_t(__popc(f));
        }
    }
}

template <int K>
__device__ __forceinline__ void pipe_flush(const SigArgs &A, const PipeSmem &S, PipeCtl &C, uint32_t nt,
                                           uint32_t nv_last) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lag = A.lag, n_steps = A.n_steps, nseq = nt * n_steps;
    const uint32_t mask = A.window_mask;
    for (uint32_t seq = 0; seq < nseq; seq++) {
        const uint32_t T = seq / n_steps, s = seq - T * n_steps;
        const uint64_t tile = uint64_t(blockIdx.x) + uint64_t(T) * gridDim.x;
        const uint32_t nv = T == nt - 1 ? nv_last : uint32_t(K);
        const uint4 st = __ldg(A.steps + s);
        const uint32_t need = (st.y - st.x) * nv + ((seq == 0 && A.stall_flush) ? 1u : 0u);
        const uint32_t slot = seq % lag;
        uint32_t ok = 1;
        if (lane == 0 && ld_shared_volatile(&C.done[slot]) != need) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_shared_volatile(&C.done[slot]) != need) {
                if (ld_shared_volatile(&C.abort) || globaltimer_ns() - t0 > kWaitNs) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) {
            if (lane == 0) {
                C.abort = 1u;
                atomicOr(A.status, 1u);
            }
            return;
        }
        __threadfence_block();  // the walkers' events precede the reads below
        const uint32_t roff = uint32_t((uint64_t(T) * A.n_det) & mask);
        const uint64_t col0 = tile * K;
        const uint32_t nd = st.w - st.z;
        // 16-byte ring reads and output stores (two chunk words) when the
        // output rows allow them
        bool vec_done = false;
        if constexpr (K % 2 == 0) {
            if (A.vec_out) {
                vec_done = true;
                constexpr uint32_t H = uint32_t(K) / 2u;
                for (uint32_t i = lane; i < nd * H; i += 32u) {
                    const uint32_t d = st.z + i / H, k = 2u * (i % H);
                    ulonglong2 *r = reinterpret_cast<ulonglong2 *>(S.ring + size_t((d + roff) & mask) * K + k);
                    ulonglong2 v = *r;
                    *r = make_ulonglong2(0ull, 0ull);
                    if (k >= nv) continue;
                    const uint64_t col = col0 + k;
                    if (col == A.n_cols - 1) v.x &= A.last_mask;
                    if (col + 1 == A.n_cols - 1) v.y &= A.last_mask;
                    unsigned long long *out =
                        reinterpret_cast<unsigned long long *>(A.det + uint64_t(d) * A.n_cols + col);
                    if (k + 1 < nv) __stcs(reinterpret_cast<ulonglong2 *>(out), v);
                    else __stcs(out, v.x);
                }
            }
        }
        if (!vec_done) {
            for (uint32_t i = lane; i < nd * uint32_t(K); i += 32u) {
                const uint32_t d = st.z + i / uint32_t(K), k = i % uint32_t(K);
                uint64_t *r = S.ring + size_t((d + roff) & mask) * K + k;
                uint64_t v = *r;
                *r = 0ull;
                if (k >= nv) continue;
                const uint64_t col = col0 + k;
                if (col == A.n_cols - 1) v &= A.last_mask;
                __stcs(reinterpret_cast<unsigned long long *>(A.det + uint64_t(d) * A.n_cols + col), v);
            }
        }
        if (s == n_steps - 1) {
            uint64_t *ob = S.oacc + size_t(T & 1u) * A.n_obs * K;
            for (uint32_t i = lane; i < A.n_obs * uint32_t(K); i += 32u) {
                const uint32_t o = i / uint32_t(K), k = i % uint32_t(K);
                uint64_t v = ob[i];
                ob[i] = 0ull;
                if (k >= nv) continue;
                const uint64_t col = col0 + k;
                if (col == A.n_cols - 1) v &= A.last_mask;
                A.obs[uint64_t(o) * A.n_cols + col] = v;
            }
        }
        if (lane == 0) C.done[slot] = 0u;
        if (A.stage_items && seq + lag < nseq) {
            const uint4 s2 = __ldg(A.steps + (seq + lag) % n_steps);
            uint4 *dst = S.sitems + size_t(slot) * A.stage_items;
            for (uint32_t i = lane; i < s2.y - s2.x; i += 32u) dst[i] = __ldg(A.item_rec + s2.x + i);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            *reinterpret_cast<volatile uint32_t *>(&C.flushed) = seq + 1u;
        }
        __syncwarp();
    }
}

template <int K>
__global__ void __launch_bounds__(1024) sig_pipe_kernel(const SigArgs A) {
    extern __shared__ __align__(128) uint64_t smem[];
    __shared__ PipeCtl C;
    if (uint64_t(blockIdx.x) >= A.n_tiles) return;
    const PipeSmem S = pipe_layout(smem, A, K);
    const uint32_t tid = threadIdx.x, T_ = blockDim.x;
    const uint32_t W = A.window_mask + 1u;
    for (uint32_t i = tid; i < (W + 2u * A.n_obs) * uint32_t(K); i += T_) S.ring[i] = 0ull;
    for (uint32_t i = tid; i < A.smem_tables * kTableWords; i += T_) S.stab[i] = __ldg(A.tables + i);
    if (tid == 0) {
        C.next = 0ull;
        C.flushed = 0u;
        C.abort = 0u;
    }
    for (uint32_t i = tid; i < uint32_t(kSigMaxLag); i += T_) C.done[i] = 0u;
    for (uint32_t i = tid; i < 32u * kSigMaxLag; i += T_) C.wdone[i] = 0u;
    const uint64_t G = gridDim.x;
    const uint32_t nt = uint32_t((A.n_tiles - blockIdx.x + G - 1) / G);
    const uint64_t last = uint64_t(blockIdx.x) + uint64_t(nt - 1) * G;
    const uint64_t rem = A.n_cols - last * K;
    const uint32_t nv_last = rem < uint64_t(K) ? uint32_t(rem) : uint32_t(K);
    if (A.stage_items) {
        const uint32_t nseq = nt * A.n_steps;
        for (uint32_t j = 0; j < A.lag && j < nseq; j++) {
            const uint4 st = __ldg(A.steps + j % A.n_steps);
            for (uint32_t i = tid; i < st.y - st.x; i += T_)
                S.sitems[size_t(j) * A.stage_items + i] = __ldg(A.item_rec + st.x + i);
        }
    }
    __syncthreads();
    if ((tid >> 5) == (T_ >> 5) - 1u) pipe_flush<K>(A, S, C, nt, nv_last);
    else if (A.smem_tables) pipe_walk<true, K>(A, S, C, nt, nv_last, S.stab);
    else pipe_walk<false, K>(A, S, C, nt, nv_last, A.tables);
}

// Many circuits in one persistent launch: work items (job, tile) in job
// order, taken from a device counter; a CTA re-lays its shared memory out
// (and reloads gap tables) only when it moves to another job. The job table
// is a kernel parameter, so a launch is a memset and a kernel node under
// graph capture.
constexpr int kMaxSigBatch = 96;

struct SigBatchArgs {
    SigArgs jobs[kMaxSigBatch];
    uint64_t item_begin[kMaxSigBatch + 1];  // first work item of each job; [n_jobs] = total
    uint32_t n_jobs;
    unsigned long long *counter;
};

template <int K>
__global__ void __launch_bounds__(1024) sig_batch_kernel(const __grid_constant__ SigBatchArgs B) {
    extern __shared__ __align__(128) uint64_t smem[];
    __shared__ uint32_t s_next;
    __shared__ unsigned long long s_item;
    if (threadIdx.x == 0) s_next = 0;
    int cur = -1;
    SigSmem S{};
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(B.counter, 1ull);
        __syncthreads();
        const unsigned long long item = s_item;
        __syncthreads();
        if (item >= B.item_begin[B.n_jobs]) break;
        int lo = 0, hi = int(B.n_jobs) - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (B.item_begin[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const SigArgs &A = B.jobs[lo];
        if (lo != cur) {
            S = sig_layout(smem, A, K);
            sig_setup<K>(A, S);
            cur = lo;
        }
        sig_tile<K>(A, S, item - B.item_begin[lo], &s_next);
    }
}

constexpr uint32_t kSigQueueMax = 16384;  // events per shared queue (128 KB)
constexpr uint32_t kSigQueueMin = 256;

static size_t sig_table_bytes(const SigProgram &G) { return G.tables.size() * 4; }

// Step item records staged in shared memory per staging buffer (one for a
// barrier schedule, lag for a pipelined one): the largest step's, if all
// buffers together hold at most 1024 records.
static uint32_t sig_stage_items(const SigProgram &G, int sched) {
    const SigSchedule &S = G.sched[sched];
    uint32_t m = 0;
    for (const SigStep &st : S.steps) m = std::max(m, st.item_end - st.item_begin);
    return m * std::max<uint32_t>(S.lag, 1u) <= 1024 ? m : 0u;
}

static size_t sig_stage_bytes(const SigProgram &G, int sched) {
    return size_t(sig_stage_items(G, sched)) * std::max<uint32_t>(G.sched[sched].lag, 1u) * 16;
}

// ring and observables (two buffers when pipelined), padded to 16 bytes
static size_t sig_ring_bytes(const SigProgram &G, int sched, uint64_t n_obs, int K) {
    const size_t nob = G.sched[sched].lag ? 2 : 1;
    return ((size_t(G.sched[sched].window) + nob * size_t(n_obs)) * size_t(K) * 8 + 15) & ~size_t(15);
}

// Ring + observables + event queue: the queue takes what is left of `budget`
// (at least kSigQueueMin events, at most kSigQueueMax).
static uint32_t sig_queue_cap(const SigProgram &G, int sched, uint64_t n_obs, int K, size_t budget,
                              bool smem_tables) {
    const size_t ring = sig_ring_bytes(G, sched, n_obs, K) + (smem_tables ? sig_table_bytes(G) : 0) +
                        sig_stage_bytes(G, sched);
    const size_t left = budget > ring ? (budget - ring) / 8 : 0;
    return uint32_t(std::min<size_t>(kSigQueueMax, std::max<size_t>(kSigQueueMin, left & ~size_t(255))));
}

static size_t sig_smem_bytes(const SigProgram &G, int sched, uint64_t n_obs, int K, uint32_t qcap,
                             bool smem_tables) {
    return sig_ring_bytes(G, sched, n_obs, K) + (smem_tables ? sig_table_bytes(G) : 0) + sig_stage_bytes(G, sched) +
           size_t(qcap) * 8;
}

// ---------------------------------------------------------------------------
// Batched persistent launch: resident CTAs pull work items (job, tile) from a
// device counter until none are left; each item runs its job's program on
// one tile with the CTA-wide layer loop above. Jobs may have different
// circuits, tile sizes (K), seeds and outputs; the job table is a kernel
// parameter, so a launch needs no host-to-device copy.

constexpr int kMaxBatch = 96;

struct BatchJob {
    const Layer *layers;
    const uint32_t *args;
    const NoiseDesc *noise;
    const uint32_t *tables;
    uint64_t *det;
    uint64_t *obs;
    uint64_t n_cols;
    uint64_t last_mask;
    uint64_t item_begin;  // first work item of this job (items of a job are consecutive)
    uint32_t n_layers, n_slots, max_window_segs, key0, key1, K;
};

struct BatchArgs {
    uint32_t n_jobs;
    uint32_t pad;
    uint64_t total_items;
    unsigned long long *counter;  // work-queue head, zeroed before the launch
    uint32_t *status;
    BatchJob jobs[kMaxBatch];
};

template <int KMAX>
__global__ void __launch_bounds__(256, KMAX == 1 ? 4 : 3) batch_kernel(const __grid_constant__ BatchArgs B) {
    extern __shared__ __align__(128) uint64_t smem[];
    uint64_t *bars = smem;                                           // 2 mbarriers
    int *abort_flag = reinterpret_cast<int *>(smem + 2);
    unsigned long long *item_slot = reinterpret_cast<unsigned long long *>(smem + 3);
    uint32_t *stage0 = reinterpret_cast<uint32_t *>(smem + 16);      // 128-byte offset
    uint32_t *stage1 = stage0 + kStageWords;
    uint64_t *F = reinterpret_cast<uint64_t *>(stage1 + kStageWords);
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    for (;;) {
        if (threadIdx.x == 0) *item_slot = atomicAdd(B.counter, 1ull);
        __syncthreads();
        const unsigned long long item = *item_slot;
        __syncthreads();
        if (item >= B.total_items) break;
        uint32_t lo = 0, hi = B.n_jobs;  // last job with item_begin <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) / 2;
            if (B.jobs[mid].item_begin <= item) lo = mid; else hi = mid;
        }
        const BatchJob &J = B.jobs[lo];
        KernelArgs a{};
        a.layers = J.layers;
        a.args = J.args;
        a.noise = J.noise;
        a.tables = J.tables;
        a.status = B.status;
        a.n_layers = J.n_layers;
        a.n_slots = J.n_slots;
        a.max_window_segs = J.max_window_segs;
        a.key0 = J.key0;
        a.key1 = J.key1;
        a.first_chunk = 0;
        a.n_cols = J.n_cols;
        a.last_mask = J.last_mask;
        a.det = J.det;
        a.obs = J.obs;
        const uint64_t col0 = (item - J.item_begin) * J.K;
        EvUnit *ev = reinterpret_cast<EvUnit *>(F + size_t(J.n_slots) * J.K);
        if (KMAX >= 4 && J.K == 4)
            run_tile<KMAX >= 4 ? 4 : 1>(a, F, stage0, stage1, ev, bars, abort_flag, col0, parity);
        else if (KMAX >= 2 && J.K == 2)
            run_tile<KMAX >= 2 ? 2 : 1>(a, F, stage0, stage1, ev, bars, abort_flag, col0, parity);
        else
            run_tile<1>(a, F, stage0, stage1, ev, bars, abort_flag, col0, parity);
        if (*abort_flag) break;
    }
}

// Shared memory of batch_kernel for one job with tile size K.
static size_t batch_smem_bytes(uint32_t n_slots, uint32_t max_window_segs, int K) {
    return 128 + 2 * size_t(kStageWords) * 4 + size_t(n_slots) * K * 8 + size_t(max_window_segs) * K * sizeof(EvUnit);
}

// ---------------------------------------------------------------------------
// Warp-owned chunks (frame_kernel_w). Frame updates of different 64-shot
// chunks never interact, so each consumer warp owns KW chunks outright and
// runs the whole program on them, synchronising only within the warp. Warp 0
// is a producer: one lane streams every staged layer's argument block into a
// ring of kRing shared-memory stages with bulk asynchronous copies; a "full"
// mbarrier per stage completes when the bytes land, an "empty" mbarrier when
// every active consumer warp has finished with it. Consumers therefore drift
// apart by up to kRing staged layers instead of meeting at a CTA barrier after
// every layer, and a warp busy in a long noise walk does not stall the others.

constexpr uint32_t kRing = 4;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__host__ __device__ constexpr size_t ring_region_bytes() {
    return (size_t(kRing) * kStageWords * 4 + 2 * kRing * 8 + 16 + 127) & ~size_t(127);
}

__device__ __forceinline__ void group_sync(uint32_t bar_id, uint32_t nthreads) {
    if (nthreads == 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
}

// One chunk group: GT threads (GT/32 warps) run the program on the group's
// KW chunks; gtid is the thread's index in the group, bar_id its named
// barrier (1..15; a single-warp group uses __syncwarp).
template <int KW>
__device__ __forceinline__ void consumer_group(const KernelArgs &P, uint64_t *Fw, EvUnit *evbuf, const uint32_t *ring,
                                               uint64_t *full, uint64_t *empty, int *abort_flag, uint64_t col0,
                                               int nvalid, uint32_t gtid, uint32_t GT, uint32_t bar_id) {
    const uint32_t chunk0 = P.first_chunk + uint32_t(col0);
    Layer cur = P.layers[0];
    for (uint32_t L = 0; L < P.n_layers; L++) {
        const Layer nxt = (L + 1 < P.n_layers) ? P.layers[L + 1] : cur;
        const uint32_t *st = nullptr;
        uint32_t b = 0;
        if (cur.nwords) {
            b = cur.seq % kRing;
            if (!mbar_wait_bounded(&full[b], (cur.seq / kRing) & 1u)) {
                *reinterpret_cast<volatile int *>(abort_flag) = 1;
                if (gtid == 0) atomicOr(P.status, 1u);
                return;
            }
            st = ring + size_t(b) * kStageWords;
        }
        switch (cur.kind) {
        case L_ZERO:
            for (uint32_t i = gtid; i < cur.count; i += GT) {
                uint64_t *d = Fw + st[i] * KW;
#pragma unroll
                for (int k = 0; k < KW; k++) d[k] = 0ull;
            }
            break;
        case L_XOR:
        case L_COPY: {
            constexpr int U = 8;
            const bool is_xor = cur.kind == L_XOR;
            for (uint32_t i0 = gtid; i0 < cur.count; i0 += GT * U) {
                uint32_t w[U];
#pragma unroll
                for (int r = 0; r < U; r++) {
                    const uint32_t i = i0 + GT * r;
                    w[r] = i < cur.count ? st[i] : 0xFFFFFFFFu;
                }
                uint64_t a[U][KW], bb[U][KW];
#pragma unroll
                for (int r = 0; r < U; r++)
                    if (w[r] != 0xFFFFFFFFu) {
#pragma unroll
                        for (int k = 0; k < KW; k++) {
                            bb[r][k] = Fw[(w[r] >> 16) * KW + k];
                            if (is_xor) a[r][k] = Fw[(w[r] & 0xFFFFu) * KW + k];
                        }
                    }
#pragma unroll
                for (int r = 0; r < U; r++)
                    if (w[r] != 0xFFFFFFFFu) {
#pragma unroll
                        for (int k = 0; k < KW; k++)
                            Fw[(w[r] & 0xFFFFu) * KW + k] = is_xor ? (a[r][k] ^ bb[r][k]) : bb[r][k];
                    }
            }
            break;
        }
        case L_NGEN: {
            // walk the event streams of a window of upcoming noise ops into
            // the group's event buffer (one thread per (segment, chunk))
            const uint32_t units = P.fault_mode ? 0u : cur.aux2 * KW;
            for (uint32_t u = gtid; u < units; u += GT) {
                const uint32_t ws = u / KW;
                const int k = int(u % KW);
                uint32_t di = cur.aux, base = 0;
                uint32_t nseg = P.noise[di].n_seg;
                while (ws >= base + nseg) {
                    base += nseg;
                    nseg = P.noise[++di].n_seg;
                }
                EvUnit *E = evbuf + u;
                if (k >= nvalid) {
                    E->n = 0;
                    E->cont_d = 0xFFFFu;
                    continue;
                }
                const NoiseDesc nd = P.noise[di];
                const uint32_t *Tt = P.tables + size_t(nd.table) * kTableWords;
                const float inv = __uint_as_float(__ldg(Tt + kGapLen));
                walk_segment<KW>(nd, Tt, inv, ws - base, chunk0 + uint32_t(k), P.key0, P.key1, 0u, -1, E,
                                 nullptr, P.args + nd.tgt_off, k);
            }
            break;
        }
        case L_NAPPLY: {
            // apply the buffered events of one op (one thread per event slot);
            // a walk that overflowed its buffer resumes here
            if (P.fault_mode) {
                inject_faults<KW>(Fw, P, cur.aux, col0, nvalid, gtid, GT);
                break;
            }
            const NoiseDesc nd = P.noise[cur.aux];
            const uint32_t *tg = P.args + nd.tgt_off;
            const uint32_t items = nd.n_seg * KW * kEvCap;
            for (uint32_t i = gtid; i < items; i += GT) {
                const uint32_t uu = i / kEvCap, e = i % kEvCap;
                const uint32_t sg = uu / KW;
                const int k = int(uu % KW);
                if (k >= nvalid) continue;
                const EvUnit *E = evbuf + (cur.aux2 + sg) * KW + uint32_t(k);
                if (e < E->n) {
                    const uint32_t v = E->ev[e];
                    apply_event<KW>(Fw, tg, nd.kind, sg, int(v & 0xFFFu), v >> 12, k);
                }
                if (e == 0 && E->cont_d != 0xFFFFu) {
                    const uint32_t *Tt = P.tables + size_t(nd.table) * kTableWords;
                    const float inv = __uint_as_float(__ldg(Tt + kGapLen));
                    walk_segment<KW>(nd, Tt, inv, sg, chunk0 + uint32_t(k), P.key0, P.key1, E->cont_d,
                                     E->cont_pos, nullptr, Fw, tg, k);
                }
            }
            break;
        }
        case L_DET:
            for (uint32_t d = gtid; d < cur.count; d += GT) {
                const uint32_t lo = st[d], hi = st[d + 1];
                uint64_t v[KW];
#pragma unroll
                for (int k = 0; k < KW; k++) v[k] = 0ull;
                for (uint32_t t = lo; t < hi; t++) {
                    const uint64_t *x = Fw + st[t] * KW;
#pragma unroll
                    for (int k = 0; k < KW; k++) v[k] ^= x[k];
                }
                uint64_t *out = P.det + uint64_t(cur.aux + d) * P.n_cols + col0;
#pragma unroll
                for (int k = 0; k < KW; k++)
                    if (k < nvalid) out[k] = (col0 + uint64_t(k) == P.n_cols - 1) ? (v[k] & P.last_mask) : v[k];
            }
            break;
        case L_OBS:
            for (uint32_t d = gtid; d < cur.count; d += GT) {
                const uint32_t lo = st[d], hi = st[d + 1];
                uint64_t v[KW];
#pragma unroll
                for (int k = 0; k < KW; k++) v[k] = 0ull;
                for (uint32_t t = lo + 1; t < hi; t++) {
                    const uint64_t *x = Fw + st[t] * KW;
#pragma unroll
                    for (int k = 0; k < KW; k++) v[k] ^= x[k];
                }
                uint64_t *acc = Fw + st[lo] * KW;
#pragma unroll
                for (int k = 0; k < KW; k++) acc[k] ^= v[k];
            }
            break;
        case L_OBSOUT:
            for (uint32_t o = gtid; o < cur.count; o += GT) {
                const uint64_t *acc = Fw + st[o] * KW;
                uint64_t *out = P.obs + uint64_t(o) * P.n_cols + col0;
#pragma unroll
                for (int k = 0; k < KW; k++)
                    if (k < nvalid) out[k] = (col0 + uint64_t(k) == P.n_cols - 1) ? (acc[k] & P.last_mask) : acc[k];
            }
            break;
        default:
            break;
        }
        group_sync(bar_id, GT);
        if (cur.nwords && gtid == 0) mbar_arrive(&empty[b]);
        if (*reinterpret_cast<volatile int *>(abort_flag)) return;
        cur = nxt;
    }
}

__device__ __forceinline__ void producer_lane(const KernelArgs &P, uint32_t *ring, uint64_t *full, uint64_t *empty,
                                              int *abort_flag) {
    uint32_t q = 0;
    bool aborted = false;
    for (uint32_t L = 0; L < P.n_layers; L++) {
        const Layer ly = P.layers[L];
        if (!ly.nwords) continue;
        const uint32_t b = q % kRing, r = q / kRing;
        if (r >= 1 && !mbar_wait_bounded(&empty[b], (r - 1) & 1u)) {
            aborted = true;
            break;
        }
        if (*reinterpret_cast<volatile int *>(abort_flag)) {
            aborted = true;
            break;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[b], ly.nwords * 4u);
        bulk_copy_g2s(ring + size_t(b) * kStageWords, P.args + ly.off, ly.nwords * 4u, &full[b]);
        q++;
    }
    if (aborted) {
        *reinterpret_cast<volatile int *>(abort_flag) = 1;
        // wait (bounded) for the copies still in flight before leaving
        for (uint32_t j = q > kRing ? q - kRing : 0; j < q; j++) mbar_wait_bounded(&full[j % kRing], (j / kRing) & 1u);
        atomicOr(P.status, 1u);
    }
}

template <int KW>
__global__ void __launch_bounds__(544) frame_kernel_w(const KernelArgs P) {
    extern __shared__ __align__(128) uint64_t smem[];
    uint32_t *ring = reinterpret_cast<uint32_t *>(smem);
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + size_t(kRing) * kStageWords);
    uint64_t *empty = full + kRing;
    int *abort_flag = reinterpret_cast<int *>(empty + kRing);
    uint64_t *F = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(smem) + ring_region_bytes());
    const uint32_t warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t G = P.group_warps;                // warps per chunk group
    const uint32_t W = (blockDim.x / 32 - 1) / G;    // chunk groups
    const uint64_t tile0 = uint64_t(blockIdx.x) * W * KW;
    const uint64_t left = P.n_cols - tile0;
    const uint64_t need = (left + KW - 1) / KW;
    const uint32_t active = need < uint64_t(W) ? uint32_t(need) : W;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < kRing; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], active);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) producer_lane(P, ring, full, empty, abort_flag);
        return;
    }
    const uint32_t g = (warp - 1) / G;
    if (g >= active) return;
    const uint64_t col0 = tile0 + uint64_t(g) * KW;
    const uint64_t rem = P.n_cols - col0;
    const int nvalid = rem < uint64_t(KW) ? int(rem) : KW;
    // event buffers follow the frames of all W groups
    EvUnit *ev = reinterpret_cast<EvUnit *>(F + size_t(W) * P.n_slots * KW) + size_t(g) * P.max_window_segs * KW;
    consumer_group<KW>(P, F + size_t(g) * P.n_slots * KW, ev, ring, full, empty, abort_flag, col0, nvalid,
                       ((warp - 1) % G) * 32 + lane, 32 * G, 1 + g);
}

// Dynamic shared memory of frame_kernel_w<KW> with W chunk groups: ring,
// then every group's frames, then every group's event buffer.
static size_t kernel_w_smem_bytes(uint32_t n_slots, uint32_t max_window_segs, int KW, int W) {
    return ring_region_bytes() + size_t(W) * n_slots * KW * 8 + size_t(W) * max_window_segs * KW * sizeof(EvUnit);
}

// Dynamic shared memory of frame_kernel<K>.
static size_t kernel_smem_bytes(uint32_t n_slots, uint32_t max_window_segs, int K) {
    size_t b = (size_t(n_slots) * K * 8 + 127) & ~size_t(127);
    b += 2 * size_t(kStageWords) * 4;
    b += size_t(max_window_segs) * K * sizeof(EvUnit);
    b += 2 * 8 + 16;
    return b;
}

// Gap counts of words w by the device routines the kernels use (method 0:
// the decoupled kernel's walkers, one table read when |inv_log2| <
// kNearInv, else the two-read count; 1: the two-read count; 2: the log
// estimate with neighbour loops, which kernels 3 to 6 use where the one
// read is not allowed); table in global memory.
__global__ void gap_counts_kernel(const uint32_t *__restrict__ T, float inv, float c32, const uint32_t *__restrict__ w,
                                  uint64_t n, int method, int32_t *__restrict__ out) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint32_t x = w[i];
        int g;
        if (method == 0 && fabsf(inv) < kNearInv) g = gap_count_near<false>(T, inv, c32, x);
        else if (method <= 1) g = gap_count_est<false>(T, inv, c32, x);
        else g = gap_count(T, inv, x);
        out[i] = g;
    }
}

// ------------------------------------------------------------- host code

static int cuda_fail(cudaError_t e, const char *what) {
    return fail(TMCS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Upload (once per device) and return the device copy of a program; map is
// the circuit's per-device copies of that program.
static int upload_program(const tmcs_circuit *c, const Program &P, std::map<int, DeviceProgram> &map,
                          const DeviceProgram **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(c->mu);
    auto it = map.find(dev);
    if (it != map.end()) {
        *out = &it->second;
        return TMCS_OK;
    }
    const size_t b_layers = align256(P.layers.size() * sizeof(Layer));
    const size_t b_args = align256(P.args.size() * 4);
    const size_t b_noise = align256(P.noise.size() * sizeof(NoiseDesc));
    const size_t b_tables = align256(P.tables.size() * 4);
    const size_t b_fault = align256(P.fault_base.size() * 8);
    const size_t total = std::max<size_t>(b_layers + b_args + b_noise + b_tables + b_fault, 256);
    std::vector<uint8_t> host(total, 0);
    std::memcpy(host.data(), P.layers.data(), P.layers.size() * sizeof(Layer));
    std::memcpy(host.data() + b_layers, P.args.data(), P.args.size() * 4);
    std::memcpy(host.data() + b_layers + b_args, P.noise.data(), P.noise.size() * sizeof(NoiseDesc));
    std::memcpy(host.data() + b_layers + b_args + b_noise, P.tables.data(), P.tables.size() * 4);
    std::memcpy(host.data() + b_layers + b_args + b_noise + b_tables, P.fault_base.data(), P.fault_base.size() * 8);
    void *base = nullptr;
    e = cudaMalloc(&base, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TMCS_E_OOM, std::string("cudaMalloc of the device program: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(base, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(base);
        return cuda_fail(e, "cudaMemcpy of the device program");
    }
    DeviceProgram dp;
    dp.device = dev;
    dp.base = base;
    dp.bytes = total;
    uint8_t *b = static_cast<uint8_t *>(base);
    dp.layers = reinterpret_cast<const Layer *>(b);
    dp.args = reinterpret_cast<const uint32_t *>(b + b_layers);
    dp.noise = reinterpret_cast<const NoiseDesc *>(b + b_layers + b_args);
    dp.tables = reinterpret_cast<const uint32_t *>(b + b_layers + b_args + b_noise);
    dp.fault_base = reinterpret_cast<const uint64_t *>(b + b_layers + b_args + b_noise + b_tables);
    auto ins = map.emplace(dev, dp);
    *out = &ins.first->second;
    return TMCS_OK;
}

static int device_program(const tmcs_circuit *c, const DeviceProgram **out) {
    return upload_program(c, c->prog, c->dev, out);
}

// Upload (once per device) the event-signature program.
static int device_sig(const tmcs_circuit *c, const DeviceSig **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(c->mu);
    auto it = c->dev_sig.find(dev);
    if (it != c->dev_sig.end()) {
        *out = &it->second;
        return TMCS_OK;
    }
    const SigProgram &G = c->sig;
    const size_t b_noise = align256(G.noise.size() * sizeof(NoiseDesc));
    const size_t b_tables = align256(G.tables.size() * 4);
    const size_t n_sched = G.sched.size();
    size_t b_items[kSigMaxSchedules] = {}, b_steps[kSigMaxSchedules] = {}, b_sev[kSigMaxSchedules] = {},
           b_desc[kSigMaxSchedules] = {}, b_sched = 0;
    for (size_t k = 0; k < n_sched; k++) {
        b_items[k] = align256(G.sched[k].item_rec.size() * 4);
        b_steps[k] = align256(G.sched[k].steps.size() * sizeof(SigStep));
        b_sev[k] = align256(G.sched[k].step_events.size() * sizeof(float));
        b_desc[k] = align256(G.sched[k].item_desc.size() * 4);
        b_sched += b_items[k] + b_steps[k] + b_sev[k] + b_desc[k];
    }
    const size_t b_ent = align256(G.ev_ent.size() * 4);
    const size_t total = std::max<size_t>(b_noise + b_tables + b_sched + b_ent, 256);
    std::vector<uint8_t> host(total, 0);
    size_t o = 0;
    auto put = [&](const void *src, size_t n, size_t span) {
        if (n) std::memcpy(host.data() + o, src, n);
        const size_t at = o;
        o += span;
        return at;
    };
    std::vector<NoiseDesc> dn = G.noise;
    for (size_t i = 0; i < dn.size(); i++) dn[i].tgt_off = G.ev_base[i];
    const size_t o_noise = put(dn.data(), dn.size() * sizeof(NoiseDesc), b_noise);
    const size_t o_tables = put(G.tables.data(), G.tables.size() * 4, b_tables);
    size_t o_items[kSigMaxSchedules] = {}, o_steps[kSigMaxSchedules] = {}, o_sev[kSigMaxSchedules] = {},
           o_desc[kSigMaxSchedules] = {};
    for (size_t k = 0; k < n_sched; k++) {
        const SigSchedule &S = G.sched[k];
        o_items[k] = put(S.item_rec.data(), S.item_rec.size() * 4, b_items[k]);
        o_steps[k] = put(S.steps.data(), S.steps.size() * sizeof(SigStep), b_steps[k]);
        o_sev[k] = put(S.step_events.data(), S.step_events.size() * sizeof(float), b_sev[k]);
        o_desc[k] = put(S.item_desc.data(), S.item_desc.size() * 4, b_desc[k]);
    }
    const size_t o_ent = put(G.ev_ent.data(), G.ev_ent.size() * 4, b_ent);
    void *base = nullptr;
    e = cudaMalloc(&base, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TMCS_E_OOM, std::string("cudaMalloc of the signature program: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpy(base, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(base);
        return cuda_fail(e, "cudaMemcpy of the signature program");
    }
    DeviceSig ds;
    ds.device = dev;
    ds.base = base;
    ds.bytes = total;
    uint8_t *b = static_cast<uint8_t *>(base);
    ds.noise = reinterpret_cast<const NoiseDesc *>(b + o_noise);
    ds.tables = reinterpret_cast<const uint32_t *>(b + o_tables);
    for (size_t k = 0; k < n_sched; k++) {
        ds.items[k] = reinterpret_cast<const uint32_t *>(b + o_items[k]);
        ds.steps[k] = reinterpret_cast<const SigStep *>(b + o_steps[k]);
        ds.step_events[k] = reinterpret_cast<const float *>(b + o_sev[k]);
        ds.item_desc[k] = reinterpret_cast<const uint32_t *>(b + o_desc[k]);
    }
    ds.ev_ent = reinterpret_cast<const uint32_t *>(b + o_ent);
    auto ins = c->dev_sig.emplace(dev, ds);
    *out = &ins.first->second;
    return TMCS_OK;
}

void free_device_programs(tmcs_circuit *c) {
    std::lock_guard<std::mutex> lock(c->mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto *m : {&c->dev, &c->dev_meas}) {
        for (auto &kv : *m) {
            cudaSetDevice(kv.first);
            cudaFree(kv.second.base);
        }
        m->clear();
    }
    for (auto &kv : c->dev_sig) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second.base);
    }
    c->dev_sig.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

struct DeviceLimits {
    int sms = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;
};

static int device_limits(DeviceLimits *lim) {
    int dev = 0, v = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    lim->sms = v;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    lim->smem_optin = size_t(v);
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    lim->smem_per_sm = size_t(v);
    return TMCS_OK;
}

struct LaunchShape {
    int mode = 3;      // 3: CTA-wide layers (frame_kernel), 4: warp-owned chunks (frame_kernel_w),
                       // 5: event signatures (sig_kernel; tiles = resident CTAs),
                       // 6: pipelined event signatures (sig_pipe_kernel; tiles = resident CTAs)
    int K = 1;         // chunks per CTA (mode 3) or per consumer warp (mode 4)
    int warps = 0;     // chunk groups (mode 4)
    int group = 1;     // warps per chunk group (mode 4)
    int threads = 256;
    size_t smem = 0;
    uint64_t tiles = 0;
    int sms = 0;       // mode 5: SM count (grid = SMs x resident CTAs per SM)
    uint32_t qcap = 0; // mode 5: event-queue capacity
    bool smem_tables = false;  // mode 5: gap tables staged in shared memory
    int sched = 0;     // mode 5, 6, 7: schedule of the signature program (lag 0 for mode 5, 7; > 0 for 6)
    FlowShape flow;    // mode 7: decoupled event-signature kernel (flow_kernel)
};

static int env_int(const char *name, int dflt) {
    const char *v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

// Tile shape. Shared memory per 64-shot chunk is fixed by the circuit (its
// frame slots), so the choice is how many chunks one CTA owns (K) and how many
// threads run each layer: larger tiles amortise the per-layer cost (staging,
// dispatch, barrier) over more shots, smaller ones put more CTAs on an SM to
// overlap one CTA's barriers and noise walks with another's updates. The
// autotuner below times the feasible shapes; this heuristic is its fallback.
// Tuning knobs (they change only the launch shape, never the output bits):
// TMCS_TILE_K caps the chunks per CTA, TMCS_THREADS fixes the CTA size,
// TMCS_AUTOTUNE=0 disables timing.
static bool shape_fits(const Program &P, const DeviceLimits &lim, int K) {
    return kernel_smem_bytes(P.n_slots, P.max_window_segs, K) <= lim.smem_optin;
}

static LaunchShape make_shape(const Program &P, uint64_t n_cols, int K, int threads) {
    LaunchShape s;
    s.mode = 3;
    s.K = K;
    s.threads = threads;
    s.smem = kernel_smem_bytes(P.n_slots, P.max_window_segs, K);
    s.tiles = (n_cols + K - 1) / K;
    return s;
}

// Largest chunk-group count (<= 15: one named barrier each) whose frames
// fit next to the ring, with at most 16 consumer warps.
static int max_groups_w(const Program &P, const DeviceLimits &lim, int KW, int G) {
    int W = std::min(15, 16 / G);
    while (W > 0 && kernel_w_smem_bytes(P.n_slots, P.max_window_segs, KW, W) > lim.smem_optin) W--;
    return W;
}

static LaunchShape make_shape_w(const Program &P, uint64_t n_cols, int KW, int W, int G) {
    LaunchShape s;
    s.mode = 4;
    s.K = KW;
    s.warps = W;
    s.group = G;
    s.threads = 32 * (W * G + 1);
    s.smem = kernel_w_smem_bytes(P.n_slots, P.max_window_segs, KW, W);
    s.tiles = (n_cols + uint64_t(W) * KW - 1) / (uint64_t(W) * KW);
    return s;
}

// Event-signature kernel: K chunks per CTA, persistent grid of the CTAs that
// fit on the device at once (shared memory and thread limits).
static bool sig_fits(const tmcs_circuit *c, const DeviceLimits &lim, int K, int sched = 0) {
    return c->sig.ok && sig_smem_bytes(c->sig, sched, c->n_obs, K, kSigQueueMin, false) + 1024 <= lim.smem_optin;
}

// The queue gets the shared memory left once the CTAs that the register file
// allows at this CTA size (64 registers per thread) each hold their ring.
static LaunchShape make_shape_sig(const tmcs_circuit *c, uint64_t n_cols, const DeviceLimits &lim, int K,
                                  int threads, int sched = 0) {
    LaunchShape s;
    s.mode = c->sig.sched[sched].lag ? 6 : 5;
    s.sched = sched;
    s.K = K;
    s.threads = threads;
    s.sms = lim.sms;
    const size_t ctas = size_t(std::max(1, 1024 / threads));
    // leave 1 KB for the kernel's static shared variables (dynamic + static
    // must fit the per-block limit)
    const size_t budget = std::min(lim.smem_optin - 1024, lim.smem_per_sm / ctas - 1024);
    // gap tables go to shared memory if they fit next to the ring and a
    // queue of 2048 events
    s.smem_tables = sig_smem_bytes(c->sig, sched, c->n_obs, K, 2048, true) <= budget;
    s.qcap = sig_queue_cap(c->sig, sched, c->n_obs, K, budget, s.smem_tables);
    const int qforce = env_int("TMCS_SIG_QUEUE", 0);  // tuning/testing knob: queue capacity
    if (qforce > 0) s.qcap = uint32_t(std::min<int>(qforce, int(kSigQueueMax)));
    // every warp's slice holds at least one ballot's worth (32 events); a
    // pipelined walker's slice at least one iteration's worth (64)
    s.qcap = std::max<uint32_t>(s.qcap, uint32_t(s.mode == 6 ? 2 * threads : threads));
    s.smem = sig_smem_bytes(c->sig, sched, c->n_obs, K, s.qcap, s.smem_tables);
    const uint64_t n_tiles = (n_cols + K - 1) / K;
    s.tiles = std::min<uint64_t>(n_tiles, uint64_t(lim.sms) * ctas);
    return s;
}

// Decoupled event-signature kernel (mode 7): one CTA per SM, K chunks per
// tile, `appliers` of its warps apply steps, the others walk. mode = 0 when
// the shape does not fit.
static LaunchShape make_shape_flow(const tmcs_circuit *c, uint64_t n_cols, const DeviceLimits &lim, int sched, int K,
                                   int threads, int appliers, bool global_arena = false, int window = 0) {
    LaunchShape s;
    s.mode = 0;
    if (!flow_shape(c, sched, K, threads, appliers, lim.smem_optin - 1024, &s.flow, global_arena, window)) return s;
    // a global arena has one slice per resident CTA (at most two per SM)
    if (global_arena) s.flow.garena_ctas = uint32_t(2 * lim.sms);
    s.mode = 7;
    s.sched = sched;
    s.K = K;
    s.threads = threads;
    s.warps = appliers;
    s.group = global_arena ? 1 : 0;
    s.sms = lim.sms;
    s.smem = s.flow.smem;
    s.smem_tables = s.flow.smem_tables;
    s.qcap = s.flow.arena;
    s.tiles = std::min<uint64_t>((n_cols + K - 1) / K, uint64_t(lim.sms));
    return s;
}

// Dynamic shared memory of a signature shape plus 1 KB of static shared
// variables within the per-block limit.
static bool sig_shape_fits(const LaunchShape &s, const DeviceLimits &lim) { return s.smem + 1024 <= lim.smem_optin; }

static LaunchShape choose_shape_cta(const Program &P, uint64_t n_cols, const DeviceLimits &lim);

static LaunchShape choose_shape(const Program &P, uint64_t n_cols, const DeviceLimits &lim) {
    const int mode = env_int("TMCS_KERNEL", 0);
    const int kcap = env_int("TMCS_TILE_K", 0);
    if (mode == 4) {
        const int KW = kcap >= 2 ? 2 : 1;
        int G = env_int("TMCS_GROUP", 1);
        G = (G == 2 || G == 4 || G == 8) ? G : 1;
        int W = max_groups_w(P, lim, KW, G);
        const int wforce = env_int("TMCS_WARPS", 0);
        if (wforce > 0 && wforce < W) W = wforce;
        if (W >= 1) return make_shape_w(P, n_cols, KW, W, G);
        // frames of even one group do not fit next to the ring: use mode 3
    }
    return choose_shape_cta(P, n_cols, lim);
}

// CTA-wide kernel shape (mode 3) from the shared-memory and grid heuristics.
static LaunchShape choose_shape_cta(const Program &P, uint64_t n_cols, const DeviceLimits &lim) {
    const int kcap = env_int("TMCS_TILE_K", 0);
    int K = 16;
    if (kcap > 0)
        while (K > 1 && K > kcap) K >>= 1;
    while (K > 1 && !shape_fits(P, lim, K)) K >>= 1;
    if (kcap <= 0)
        while (K > 1 && 2 * (kernel_smem_bytes(P.n_slots, P.max_window_segs, K) + 1024) > lim.smem_per_sm) K >>= 1;
    while (K > 1 && (n_cols + K - 1) / K < uint64_t(2 * lim.sms)) K >>= 1;
    int threads = 256;
    const int tforce = env_int("TMCS_THREADS", 0);
    if (tforce >= 32 && tforce <= 512 && tforce % 32 == 0) threads = tforce;
    return make_shape(P, n_cols, K, threads);
}

template <int K>
static cudaError_t launch_k(const KernelArgs &a, const LaunchShape &s, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(frame_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem));
    if (e != cudaSuccess) return e;
    frame_kernel<K><<<unsigned(s.tiles), s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

template <int KW>
static cudaError_t launch_w(const KernelArgs &a, const LaunchShape &s, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(frame_kernel_w<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem));
    if (e != cudaSuccess) return e;
    frame_kernel_w<KW><<<unsigned(s.tiles), s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

// Persistent grid: as many CTAs as are resident at once (occupancy query),
// never more than there are tiles.
template <int K>
static cudaError_t launch_sig(const SigArgs &a, const LaunchShape &s, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sig_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sig_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sig_kernel<K>, s.threads, s.smem);
    if (e != cudaSuccess) return e;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(a.n_tiles, uint64_t(s.sms) * uint64_t(std::max(per_sm, 1))));
    sig_kernel<K><<<unsigned(grid), s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

// Mode 5 takes the event-signature program (device copy ds, host G); its
// output, seed and chunk range come from a0 like the frame kernels'.
template <int K>
static cudaError_t launch_pipe(const SigArgs &a, const LaunchShape &s, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sig_pipe_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sig_pipe_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sig_pipe_kernel<K>, s.threads, s.smem);
    if (e != cudaSuccess) return e;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(a.n_tiles, uint64_t(s.sms) * uint64_t(std::max(per_sm, 1))));
    // steps are counted per CTA in 32 bits
    if ((a.n_tiles / grid + 1) * uint64_t(a.n_steps) >= (uint64_t(1) << 31)) return cudaErrorInvalidValue;
    sig_pipe_kernel<K><<<unsigned(grid), s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

// ---- scratch of the decoupled kernel's global arena: one grow-only buffer
// per (device, stream), so launches on different streams never share arena
// slices (library-owned; allocated by the first call on that stream that
// needs it, which must not be under stream capture)
static std::mutex g_flow_scratch_mu;
static std::map<std::pair<int, cudaStream_t>, std::pair<uint32_t *, size_t>> g_flow_scratch;

static cudaError_t flow_scratch(cudaStream_t st, size_t bytes, uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_flow_scratch_mu);
    auto &slot = g_flow_scratch[{dev, st}];
    if (slot.second < bytes) {
        if (slot.first) {
            // in-flight kernels may still use the old buffer
            if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
            cudaFree(slot.first);
            slot = {nullptr, 0};
        }
        void *p = nullptr;
        if ((e = cudaMalloc(&p, bytes)) != cudaSuccess) return e;
        slot = {static_cast<uint32_t *>(p), bytes};
    }
    *out = slot.first;
    return cudaSuccess;
}

static cudaError_t launch(const KernelArgs &a0, const LaunchShape &s, cudaStream_t st,
                          const DeviceSig *ds = nullptr, const SigProgram *G = nullptr, uint32_t n_obs = 0) {
    if (s.mode == 7) {
        if (!ds || !G) return cudaErrorInvalidValue;
        FlowCall call;
        call.key0 = a0.key0;
        call.key1 = a0.key1;
        call.first_chunk = a0.first_chunk;
        call.n_cols = a0.n_cols;
        call.last_mask = a0.last_mask;
        call.det = a0.det;
        call.obs = a0.obs;
        call.status = a0.status;
        if (s.flow.global_arena) {
            call.scratch_bytes = size_t(s.flow.garena_ctas) * s.flow.arena * 4;
            const cudaError_t e = flow_scratch(st, call.scratch_bytes, &call.scratch);
            if (e != cudaSuccess) return e;
        }
        return flow_launch(*G, n_obs, ds, s.flow, call, s.sms, st);
    }
    if (s.mode == 5 || s.mode == 6) {
        if (!ds || !G || s.sched < 0 || size_t(s.sched) >= G->sched.size()) return cudaErrorInvalidValue;
        const SigSchedule &S = G->sched[s.sched];
        SigArgs a{};
        a.noise = ds->noise;
        a.tables = ds->tables;
        a.item_rec = reinterpret_cast<const uint4 *>(ds->items[s.sched]);
        a.steps = reinterpret_cast<const uint4 *>(ds->steps[s.sched]);
        a.ev_ent = ds->ev_ent;
        a.n_steps = uint32_t(S.steps.size());
        a.window_mask = S.window - 1u;
        a.n_obs = n_obs;
        a.queue_cap = s.qcap;
        a.smem_tables = s.smem_tables ? uint32_t(G->tables.size() / kTableWords) : 0u;
        a.stage_items = sig_stage_items(*G, s.sched);
        a.key0 = a0.key0;
        a.key1 = a0.key1;
        a.first_chunk = a0.first_chunk;
        a.n_cols = a0.n_cols;
        a.last_mask = a0.last_mask;
        a.n_tiles = (a0.n_cols + uint64_t(s.K) - 1) / uint64_t(s.K);
        a.det = a0.det;
        a.obs = a0.obs;
        LaunchShape t = s;
        t.tiles = std::min<uint64_t>(s.tiles, a.n_tiles);
        if (s.mode == 6) {
            if (!S.lag || s.threads < 64) return cudaErrorInvalidValue;
            a.lag = S.lag;
            a.n_items = uint32_t(S.items.size() / 2);
            a.n_det = G->n_det;
            a.vec_out = (reinterpret_cast<uintptr_t>(a0.det) % 16 == 0 && a0.n_cols % 2 == 0) ? 1u : 0u;
            a.status = a0.status;
            // testing knob: make the flusher's bounded wait run out (the
            // kernel then reports TMCS_E_TIMEOUT through the status word)
            a.stall_flush = env_int("TMCS_TEST_STALL_FLUSH", 0) > 0 ? 1u : 0u;
            switch (s.K) {
            case 16: return launch_pipe<16>(a, t, st);
            case 8: return launch_pipe<8>(a, t, st);
            case 4: return launch_pipe<4>(a, t, st);
            case 2: return launch_pipe<2>(a, t, st);
            default: return launch_pipe<1>(a, t, st);
            }
        }
        switch (s.K) {
        case 16: return launch_sig<16>(a, t, st);
        case 8: return launch_sig<8>(a, t, st);
        case 4: return launch_sig<4>(a, t, st);
        case 2: return launch_sig<2>(a, t, st);
        default: return launch_sig<1>(a, t, st);
        }
    }
    KernelArgs a = a0;
    a.group_warps = uint32_t(s.group);
    if (s.mode == 4) return s.K == 2 ? launch_w<2>(a, s, st) : launch_w<1>(a, s, st);
    switch (s.K) {
    case 16: return launch_k<16>(a, s, st);
    case 8: return launch_k<8>(a, s, st);
    case 4: return launch_k<4>(a, s, st);
    case 2: return launch_k<2>(a, s, st);
    default: return launch_k<1>(a, s, st);
    }
}

// ---- per-device status word (library scratch, allocated on first use)

static std::mutex g_status_mu;
static std::map<int, uint32_t *> g_status;

uint32_t *device_status_word(int device) {
    std::lock_guard<std::mutex> lock(g_status_mu);
    auto it = g_status.find(device);
    if (it != g_status.end()) return it->second;
    void *p = nullptr;
    if (cudaMalloc(&p, 256) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemset(p, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return nullptr;
    }
    g_status[device] = static_cast<uint32_t *>(p);
    return static_cast<uint32_t *>(p);
}

// Times every feasible launch shape of both kernels on the first columns of
// this call (the real launch overwrites them) and records the fastest per
// chunk for the circuit on this device. Synchronous; runs once per circuit
// and device.
static int autotune(const tmcs_circuit *c, int device, KernelArgs a, const DeviceLimits &lim, uint64_t n_cols,
                    cudaStream_t st, LaunchShape *best, const DeviceSig *ds) {
    const Program &P = c->prog;
    std::vector<LaunchShape> cands;
    // every schedule of the signature program (barrier kernel for lag 0,
    // pipelined kernel otherwise) x chunks per CTA x CTA size
    if (ds)
        for (int sched = 0; sched < int(c->sig.sched.size()); sched++)
            for (int K = 1; K <= 16; K *= 2) {
                if (!sig_fits(c, lim, K, sched)) break;
                for (int threads : {256, 512, 1024}) {
                    const LaunchShape cs = make_shape_sig(c, n_cols, lim, K, threads, sched);
                    if (sig_shape_fits(cs, lim)) cands.push_back(cs);
                }
            }
    // decoupled kernel: every barrier schedule x chunks per tile x applier
    // warps x walker window (3 or 4 Philox calls), 1024 threads. Circuits
    // whose events flip many outputs (BB codes: weight-6 checks, several
    // observables) want more applier warps than the surface-code ones.
    if (ds)
        for (int sched = 0; sched < int(c->sig.sched.size()); sched++) {
            if (c->sig.sched[sched].lag) continue;
            for (int K = 1; K <= 16; K *= 2)
                for (int app : {8, 12, 16, 20, 24})
                    for (int win : {3, 4}) {
                        // shared-memory arena (the global-memory arena, a
                        // tuning knob, measured no faster: its reads cost an
                        // L2 trip)
                        const LaunchShape cs = make_shape_flow(c, n_cols, lim, sched, K, 1024, app, false, win);
                        if (cs.mode == 7 && (win == 3 || cs.flow.window == 4)) cands.push_back(cs);
                    }
        }
    // With a signature program the frame kernels are compared through their
    // heuristic shape only (they lost to kernel 4 on every measured
    // workload); without one, every feasible frame shape is timed.
    if (ds) {
        cands.push_back(choose_shape_cta(P, n_cols, lim));
    } else {
        for (int K = 1; K <= 16; K *= 2) {
            if (!shape_fits(P, lim, K)) break;
            for (int threads : {128, 256, 512}) cands.push_back(make_shape(P, n_cols, K, threads));
        }
        for (int KW = 1; KW <= 2; KW++)
            for (int G : {1, 2, 4}) {
                const int Wmax = max_groups_w(P, lim, KW, G);
                if (Wmax >= 1) cands.push_back(make_shape_w(P, n_cols, KW, Wmax, G));
                if ((Wmax + 1) / 2 >= 1 && (Wmax + 1) / 2 < Wmax)
                    cands.push_back(make_shape_w(P, n_cols, KW, (Wmax + 1) / 2, G));
            }
    }
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    double best_per_chunk = 1e30;
    LaunchShape chosen = *best;
    for (const LaunchShape &full : cands) {
        const uint64_t per_tile = full.mode == 4 ? uint64_t(full.warps) * full.K : uint64_t(full.K);
        const uint64_t cols = std::min<uint64_t>(n_cols, uint64_t(4) * lim.sms * per_tile);
        if (cols / per_tile < uint64_t(lim.sms)) continue;
        LaunchShape s = full;
        if (s.mode != 5 && s.mode != 7) s.tiles = (cols + per_tile - 1) / per_tile;
        KernelArgs t = a;
        t.n_cols = cols;
        t.last_mask = ~uint64_t(0);
        float ms = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
            if ((e = launch(t, s, st, ds, &c->sig, uint32_t(c->n_obs))) != cudaSuccess) break;
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "autotune launch");
        }
        const double per_chunk = double(ms) / double(cols);
        if (per_chunk < best_per_chunk) {
            best_per_chunk = per_chunk;
            chosen = full;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best = chosen;
    std::lock_guard<std::mutex> lock(c->mu);
    DeviceProgram &mdp = c->dev[device];
    mdp.tuned_mode = chosen.mode;
    mdp.tuned_K = chosen.K;
    mdp.tuned_warps = chosen.warps;  // mode 7: applier warps
    mdp.tuned_group = chosen.group;
    mdp.tuned_threads = chosen.threads;
    mdp.tuned_sched = chosen.sched;
    mdp.tuned_flow = chosen.mode == 7 ? chosen.flow : FlowShape();
    return TMCS_OK;
}

// Default shape of the event-signature kernel: the largest K (<= 4) that
// leaves room for two CTAs per SM and still gives every SM two tiles.
static LaunchShape choose_shape_sig(const tmcs_circuit *c, uint64_t n_cols, const DeviceLimits &lim) {
    const int kcap = env_int("TMCS_TILE_K", 0);
    if (env_int("TMCS_KERNEL", 0) == 7) {
        // forced decoupled kernel: TMCS_SIG_SCHED picks among the barrier
        // schedules, TMCS_TILE_K the chunks per tile (default 4),
        // TMCS_FLOW_APPLIERS the applier warps (default 8), TMCS_THREADS the
        // CTA size (default 1024); mode 0 if that shape does not fit
        int n_barrier = 0;
        while (n_barrier < int(c->sig.sched.size()) && !c->sig.sched[n_barrier].lag) n_barrier++;
        const int sched = std::min(std::max(env_int("TMCS_SIG_SCHED", 0), 0), std::max(n_barrier - 1, 0));
        int K = kcap > 0 ? std::min(kcap, 16) : 4;
        while (K > 1 && (K & (K - 1))) K--;
        const int tforce = env_int("TMCS_THREADS", 0);
        const int threads = (tforce >= 64 && tforce <= 1024 && tforce % 32 == 0) ? tforce : 1024;
        return make_shape_flow(c, n_cols, lim, sched, K, threads, env_int("TMCS_FLOW_APPLIERS", 8),
                               env_int("TMCS_FLOW_GLOBAL_ARENA", 0) > 0);
    }
    // tuning/testing knobs: TMCS_SIG_SCHED = schedule index among the barrier
    // schedules (0 = largest ring window), or among the pipelined ones with
    // TMCS_KERNEL=6
    int n_barrier = 0;
    while (n_barrier < int(c->sig.sched.size()) && !c->sig.sched[n_barrier].lag) n_barrier++;
    const bool pipe = env_int("TMCS_KERNEL", 0) == 6 && n_barrier < int(c->sig.sched.size());
    const int lo = pipe ? n_barrier : 0, hi = pipe ? int(c->sig.sched.size()) - 1 : n_barrier - 1;
    const int sched = std::min(std::max(lo + env_int("TMCS_SIG_SCHED", 0), lo), hi);
    int K = kcap > 0 ? std::min(kcap, 16) : 4;
    while (K > 1 && (K & (K - 1))) K--;
    while (K > 1 && !sig_fits(c, lim, K, sched)) K >>= 1;
    if (kcap <= 0) {
        while (K > 1 && 2 * (sig_smem_bytes(c->sig, sched, c->n_obs, K, kSigQueueMin, false) + 1024) > lim.smem_per_sm)
            K >>= 1;
        while (K > 1 && (n_cols + K - 1) / K < uint64_t(2 * lim.sms)) K >>= 1;
    }
    int threads = K >= 4 ? 1024 : 512;
    const int tforce = env_int("TMCS_THREADS", 0);
    if (tforce >= 32 && tforce <= 1024 && tforce % 32 == 0) threads = tforce;
    LaunchShape s = make_shape_sig(c, n_cols, lim, K, threads, sched);
    // the queue floor (one ballot per warp) may not fit next to a large ring
    while (!sig_shape_fits(s, lim) && (s.K > 1 || s.threads > 128)) {
        if (s.threads > 128) s = make_shape_sig(c, n_cols, lim, s.K, s.threads / 2, sched);
        else s = make_shape_sig(c, n_cols, lim, s.K / 2, threads, sched);
    }
    return s;
}

static int sample_range(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                        uint64_t *det, uint64_t *obs, void *stream, bool fault_mode = false,
                        uint64_t fault_first = 0) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    if (shots == 0) return fail(TMCS_E_INVALID, "shots must be positive");
    if ((c->n_det && !det) || (c->n_obs && !obs)) return fail(TMCS_E_INVALID, "output buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(det) & 7) || (reinterpret_cast<uintptr_t>(obs) & 7))
        return fail(TMCS_E_BUFFER, "output buffers must be 8-byte aligned");
    const uint64_t n_cols = (shots + 63) / 64;
    if (first_chunk >= (uint64_t(1) << 32) || n_cols > (uint64_t(1) << 32) - first_chunk)
        return fail(TMCS_E_INVALID, "chunk range beyond 2^32");
    const DeviceProgram *dp = nullptr;
    int rc = device_program(c, &dp);
    if (rc) return rc;
    DeviceLimits lim;
    if ((rc = device_limits(&lim))) return rc;
    const Program &P = c->prog;
    if (kernel_smem_bytes(P.n_slots, P.max_window_segs, 1) > lim.smem_optin)
        return fail(TMCS_E_INVALID, "circuit needs " + std::to_string(P.n_slots) +
                                        " frame slots; one 64-shot chunk does not fit in shared memory");
    if (P.layers.empty()) return TMCS_OK;
    uint32_t *status = device_status_word(dp->device);
    if (!status) return fail(TMCS_E_OOM, "cannot allocate the device status word");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int kmode = env_int("TMCS_KERNEL", 0);
    const DeviceSig *ds = nullptr;
    if (!fault_mode && c->sig.ok && sig_fits(c, lim, 1) && kmode != 3 && kmode != 4) {
        if ((rc = device_sig(c, &ds))) return rc;
    }
    if ((kmode == 5 || kmode == 6 || kmode == 7) && !ds && !fault_mode)
        return fail(TMCS_E_INVALID, "TMCS_KERNEL=5/6/7: no event-signature program for this circuit (" +
                                        (c->sig.ok ? std::string("ring does not fit") : c->sig.why) + ")");
    if (kmode == 6 && ds && !c->sig.sched.back().lag)
        return fail(TMCS_E_INVALID, "TMCS_KERNEL=6: the event-signature program has no pipelined schedule");
    LaunchShape s = ds ? choose_shape_sig(c, n_cols, lim) : choose_shape(P, n_cols, lim);
    if (ds && kmode == 7 && s.mode != 7 && !fault_mode)
        return fail(TMCS_E_INVALID, "TMCS_KERNEL=7: the decoupled kernel's shape does not fit this circuit");
    if (ds && !sig_shape_fits(s, lim)) {  // no signature shape fits: frame kernels
        if ((kmode == 5 || kmode == 6) && !fault_mode)
            return fail(TMCS_E_INVALID, "TMCS_KERNEL=5/6: the signature kernel's shared memory does not fit");
        ds = nullptr;
        s = choose_shape(P, n_cols, lim);
    }
    const bool forced = env_int("TMCS_TILE_K", 0) > 0 || env_int("TMCS_THREADS", 0) > 0 ||
                        kmode > 0 || env_int("TMCS_WARPS", 0) > 0 || env_int("TMCS_GROUP", 0) > 0 ||
                        env_int("TMCS_SIG_SCHED", 0) > 0;
    if (!forced && !fault_mode) {
        std::lock_guard<std::mutex> lock(c->mu);
        DeviceProgram &mdp = c->dev[dp->device];
        if (mdp.tuned_mode == 3) s = make_shape(P, n_cols, mdp.tuned_K, mdp.tuned_threads);
        if (mdp.tuned_mode == 4) s = make_shape_w(P, n_cols, mdp.tuned_K, mdp.tuned_warps, mdp.tuned_group);
        if ((mdp.tuned_mode == 5 || mdp.tuned_mode == 6) && ds)
            s = make_shape_sig(c, n_cols, lim, mdp.tuned_K, mdp.tuned_threads, mdp.tuned_sched);
        if (mdp.tuned_mode == 7 && ds) {
            const LaunchShape f = make_shape_flow(c, n_cols, lim, mdp.tuned_sched, mdp.tuned_K, mdp.tuned_threads,
                                                  mdp.tuned_warps, mdp.tuned_group == 1, mdp.tuned_flow.window);
            if (f.mode == 7) s = f;
        }
    }
    if (fault_mode) s = choose_shape(P, n_cols, lim);
    KernelArgs a{};
    a.layers = dp->layers;
    a.args = dp->args;
    a.noise = dp->noise;
    a.tables = dp->tables;
    a.status = status;
    a.n_layers = uint32_t(P.layers.size());
    a.n_slots = P.n_slots;
    a.max_window_segs = P.max_window_segs;
    a.key0 = uint32_t(seed);
    a.key1 = uint32_t(seed >> 32);
    a.first_chunk = uint32_t(first_chunk);
    a.n_cols = n_cols;
    a.last_mask = (shots % 64) ? ((uint64_t(1) << (shots % 64)) - 1) : ~uint64_t(0);
    a.det = det;
    a.obs = obs;
    a.fault_base = dp->fault_base;
    a.fault_first = fault_first;
    a.fault_mode = fault_mode ? 1u : 0u;
    if (!fault_mode && !forced && env_int("TMCS_AUTOTUNE", 1) != 0) {
        bool tuned;
        {
            std::lock_guard<std::mutex> lock(c->mu);
            tuned = c->dev[dp->device].tuned_mode != 0;
        }
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        if (!tuned && cap == cudaStreamCaptureStatusNone && n_cols >= uint64_t(16 * lim.sms)) {
            int rc2 = autotune(c, dp->device, a, lim, n_cols, st, &s, ds);
            if (rc2) return rc2;
        }
    }
    cudaError_t e = launch(a, s, st, ds, &c->sig, uint32_t(c->n_obs));
    if (e != cudaSuccess) return cuda_fail(e, "frame kernel launch");
    return TMCS_OK;
}

// ---- raw measurement records

// Same noise draws as sample_range (noise ops keep their op indices), plus the
// gauge words; records land in meas (n_meas rows of n_cols words). Always the
// CTA-wide kernel: the warp-owned kernel does not run gauge/record layers.
static int sample_measurements(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                               uint64_t *meas, void *stream) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    if (shots == 0) return fail(TMCS_E_INVALID, "shots must be positive");
    if (c->n_meas && !meas) return fail(TMCS_E_INVALID, "output buffer is NULL");
    if (reinterpret_cast<uintptr_t>(meas) & 7) return fail(TMCS_E_BUFFER, "output buffer must be 8-byte aligned");
    const uint64_t n_cols = (shots + 63) / 64;
    if (first_chunk >= (uint64_t(1) << 32) || n_cols > (uint64_t(1) << 32) - first_chunk)
        return fail(TMCS_E_INVALID, "chunk range beyond 2^32");
    {
        std::lock_guard<std::mutex> lock(c->mu);
        int rc = build_measurement_program(const_cast<tmcs_circuit *>(c));
        if (rc) return rc;
    }
    const Program &P = c->prog_meas;
    const DeviceProgram *dp = nullptr;
    int rc = upload_program(c, P, c->dev_meas, &dp);
    if (rc) return rc;
    DeviceLimits lim;
    if ((rc = device_limits(&lim))) return rc;
    if (kernel_smem_bytes(P.n_slots, P.max_window_segs, 1) > lim.smem_optin)
        return fail(TMCS_E_INVALID, "circuit needs " + std::to_string(P.n_slots) +
                                        " frame slots; one 64-shot chunk does not fit in shared memory");
    if (P.layers.empty()) return TMCS_OK;
    uint32_t *status = device_status_word(dp->device);
    if (!status) return fail(TMCS_E_OOM, "cannot allocate the device status word");
    KernelArgs a{};
    a.layers = dp->layers;
    a.args = dp->args;
    a.noise = dp->noise;
    a.tables = dp->tables;
    a.status = status;
    a.n_layers = uint32_t(P.layers.size());
    a.n_slots = P.n_slots;
    a.max_window_segs = P.max_window_segs;
    a.key0 = uint32_t(seed);
    a.key1 = uint32_t(seed >> 32);
    a.first_chunk = uint32_t(first_chunk);
    a.n_cols = n_cols;
    a.last_mask = (shots % 64) ? ((uint64_t(1) << (shots % 64)) - 1) : ~uint64_t(0);
    a.det = meas;
    a.obs = nullptr;
    a.fault_base = dp->fault_base;
    cudaError_t e = launch(a, choose_shape_cta(P, n_cols, lim), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "frame kernel launch");
    return TMCS_OK;
}

// ---- batched launch

static std::mutex g_batch_mu;
static std::map<int, unsigned long long *> g_batch_counter;

// Per-device work-queue counter of batch_kernel (library scratch, allocated
// on the first batched call on a device; make that call before any capture).
static int batch_counter(int dev, unsigned long long **out) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batch_counter.find(dev);
    if (it != g_batch_counter.end()) {
        *out = it->second;
        return TMCS_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TMCS_E_OOM, std::string("cudaMalloc of the batch work queue: ") + cudaGetErrorString(e));
    }
    g_batch_counter[dev] = static_cast<unsigned long long *>(p);
    *out = static_cast<unsigned long long *>(p);
    return TMCS_OK;
}

// Per-device side stream and fork/join events of batched launches (created
// on the first batched call that needs them; make that call before capture).
struct BatchSide {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
static std::map<int, BatchSide> g_batch_side;

static cudaError_t batch_side_stream(int dev, cudaStream_t *s, cudaEvent_t *f, cudaEvent_t *j) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchSide &b = g_batch_side[dev];
    cudaError_t e = cudaSuccess;
    if (!b.s && (e = cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if (!b.fork && (e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if (!b.join && (e = cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming)) != cudaSuccess) return e;
    *s = b.s;
    *f = b.fork;
    *j = b.join;
    return cudaSuccess;
}

static_assert(sizeof(SigBatchArgs) <= 32000, "batch job table exceeds the kernel parameter limit");

// Batched launch through the event-signature kernel. Two size classes run
// concurrently (forked stream): circuits whose 8-chunk tile fits in half of an
// SM's shared memory (512 threads, two CTAs per SM), and the rest (4-chunk
// tiles, 1024 threads, one CTA per SM). *used = false (nothing launched) if
// some job cannot take this path; the caller then uses the frame kernels.
template <int K>
static cudaError_t launch_sig_batch(const SigBatchArgs &B, int threads, size_t smem, int sms, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(sig_batch_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sig_batch_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             int(cudaSharedmemCarveoutMaxShared));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sig_batch_kernel<K>, threads, smem);
    if (e != cudaSuccess) return e;
    const uint64_t items = B.item_begin[B.n_jobs];
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(items, uint64_t(sms) * uint64_t(std::max(per_sm, 1))));
    sig_batch_kernel<K><<<unsigned(grid), threads, smem, st>>>(B);
    return cudaGetLastError();
}

static int sig_batch_sample(const tmcs_job *jobs, size_t n_jobs, cudaStream_t st, const DeviceLimits &lim, int dev,
                            unsigned long long *counter, bool *used) {
    *used = false;
    if (env_int("TMCS_KERNEL", 0) == 3 || env_int("TMCS_KERNEL", 0) == 4) return TMCS_OK;
    struct Cls {
        int K, threads;
        size_t budget;
    };
    // dynamic shared memory budgets leave 1 KB for the kernel's static shared
    // variables (dynamic + static must fit the per-block limit)
    const Cls cls_def[2] = {{4, 1024, lim.smem_optin - 1024},
                            {8, 512, std::min(lim.smem_optin - 1024, lim.smem_per_sm / 2 - 2048)}};
    struct Item {
        size_t j;
        const DeviceSig *ds;
        double cost;
    };
    std::vector<Item> cls[2];
    for (size_t j = 0; j < n_jobs; j++) {
        const tmcs_job &J = jobs[j];
        const SigProgram &G = J.c->sig;
        if (!G.ok) return TMCS_OK;
        int ci = -1;
        for (int c = 1; c >= 0 && ci < 0; c--) {
            const int warps = cls_def[c].threads / 32;
            if (sig_smem_bytes(G, 0, J.c->n_obs, cls_def[c].K, uint32_t(32 * warps), false) <= cls_def[c].budget) ci = c;
        }
        if (ci < 0) return TMCS_OK;
        cls[ci].push_back({j, nullptr, double(G.sched[0].items.size() / 2 + 1) * double((J.shots + 63) / 64)});
    }
    for (auto &v : cls)
        for (Item &it : v) {
            int rc = device_sig(jobs[it.j].c, &it.ds);
            if (rc) return rc;
        }
    *used = true;
    for (auto &v : cls)
        std::stable_sort(v.begin(), v.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
    const bool fork = !cls[0].empty() && !cls[1].empty();
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaError_t e;
    if (fork) {
        if ((e = batch_side_stream(dev, &side, &ev_fork, &ev_join)) != cudaSuccess) return cuda_fail(e, "batch stream");
        if ((e = cudaEventRecord(ev_fork, st)) != cudaSuccess) return cuda_fail(e, "batch fork");
        if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return cuda_fail(e, "batch fork");
    }
    for (int ci = 0; ci < 2; ci++) {
        const Cls &C = cls_def[ci];
        cudaStream_t cs = (fork && ci == 1) ? side : st;
        unsigned long long *ctr = counter + (ci == 1 ? 16 : 0);
        const std::vector<Item> &ord = cls[ci];
        for (size_t base = 0; base < ord.size(); base += kMaxSigBatch) {
            const size_t nb = std::min<size_t>(kMaxSigBatch, ord.size() - base);
            SigBatchArgs B;
            std::memset(&B, 0, sizeof(B));
            uint64_t items = 0;
            for (size_t i = 0; i < nb; i++) {
                const tmcs_job &J = jobs[ord[base + i].j];
                const SigProgram &G = J.c->sig;
                const DeviceSig *ds = ord[base + i].ds;
                const uint64_t n_cols = (J.shots + 63) / 64;
                const uint32_t qmin = uint32_t(C.threads);
                // the batch runs every job on its main (largest-window) schedule
                const bool tabs = sig_smem_bytes(G, 0, J.c->n_obs, C.K, 2048, true) <= C.budget;
                SigArgs &a = B.jobs[i];
                a.noise = ds->noise;
                a.tables = ds->tables;
                a.item_rec = reinterpret_cast<const uint4 *>(ds->items[0]);
                a.steps = reinterpret_cast<const uint4 *>(ds->steps[0]);
                a.ev_ent = ds->ev_ent;
                a.n_steps = uint32_t(G.sched[0].steps.size());
                a.window_mask = G.sched[0].window - 1u;
                a.n_obs = uint32_t(J.c->n_obs);
                a.smem_tables = tabs ? uint32_t(G.tables.size() / kTableWords) : 0u;
                a.queue_cap = std::max(qmin, sig_queue_cap(G, 0, J.c->n_obs, C.K, C.budget, tabs));
                a.stage_items = sig_stage_items(G, 0);
                a.key0 = uint32_t(J.seed);
                a.key1 = uint32_t(J.seed >> 32);
                a.first_chunk = 0;
                a.n_cols = n_cols;
                a.last_mask = (J.shots % 64) ? ((uint64_t(1) << (J.shots % 64)) - 1) : ~uint64_t(0);
                a.n_tiles = (n_cols + uint64_t(C.K) - 1) / uint64_t(C.K);
                a.det = J.det;
                a.obs = J.obs;
                B.item_begin[i] = items;
                items += a.n_tiles;
            }
            B.item_begin[nb] = items;
            B.n_jobs = uint32_t(nb);
            B.counter = ctr;
            if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), cs)) != cudaSuccess)
                return cuda_fail(e, "batch queue reset");
            e = ci == 0 ? launch_sig_batch<4>(B, C.threads, C.budget, lim.sms, cs)
                        : launch_sig_batch<8>(B, C.threads, C.budget, lim.sms, cs);
            if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
        }
    }
    if (fork) {
        if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) return cuda_fail(e, "batch join");
        if ((e = cudaStreamWaitEvent(st, ev_join, 0)) != cudaSuccess) return cuda_fail(e, "batch join");
    }
    return TMCS_OK;
}

static int batch_sample_shared(const tmcs_job *jobs, size_t n_jobs, void *stream);

// Jobs that fill the GPU on their own (at least 16 chunks per SM) and have
// an event-signature program run as single calls, with the launch shape
// tuned for their circuit (tuned on their first call, outside graph
// capture); the others share the persistent batch launches. Same bits
// either way.
static int batch_sample(const tmcs_job *jobs, size_t n_jobs, void *stream) {
    if (n_jobs && !jobs) return fail(TMCS_E_INVALID, "jobs is NULL");
    if (n_jobs == 0) return TMCS_OK;
    DeviceLimits lim;
    int rc = device_limits(&lim);
    if (rc) return rc;
    std::vector<tmcs_job> rest;
    rest.reserve(n_jobs);
    for (size_t j = 0; j < n_jobs; j++) {
        const tmcs_job &J = jobs[j];
        const bool large = J.c && J.c->sig.ok && J.shots > 0 && (J.shots + 63) / 64 >= uint64_t(16) * lim.sms &&
                           env_int("TMCS_KERNEL", 0) != 3 && env_int("TMCS_KERNEL", 0) != 4;
        if (!large) {
            rest.push_back(J);
            continue;
        }
        if ((rc = sample_range(J.c, 0, J.shots, J.seed, J.det, J.obs, stream)))
            return fail(rc, "job " + std::to_string(j) + ": " + tmcs_last_error());
    }
    return batch_sample_shared(rest.data(), rest.size(), stream);
}

static int batch_sample_shared(const tmcs_job *jobs, size_t n_jobs, void *stream) {
    if (n_jobs == 0) return TMCS_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    DeviceLimits lim;
    int rc = device_limits(&lim);
    if (rc) return rc;
    uint32_t *status = device_status_word(dev);
    if (!status) return fail(TMCS_E_OOM, "cannot allocate the device status word");
    unsigned long long *counter = nullptr;
    if ((rc = batch_counter(dev, &counter))) return rc;
    // validate and upload every job's program; order by decreasing work
    struct Item {
        size_t j;
        const DeviceProgram *dp;
        double cost;
    };
    std::vector<Item> order;
    order.reserve(n_jobs);
    for (size_t j = 0; j < n_jobs; j++) {
        const tmcs_job &J = jobs[j];
        const std::string at = "job " + std::to_string(j) + ": ";
        if (!J.c) return fail(TMCS_E_INVALID, at + "circuit is NULL");
        if (J.shots == 0) return fail(TMCS_E_INVALID, at + "shots must be positive");
        if ((J.c->n_det && !J.det) || (J.c->n_obs && !J.obs)) return fail(TMCS_E_INVALID, at + "output buffer is NULL");
        if ((reinterpret_cast<uintptr_t>(J.det) & 7) || (reinterpret_cast<uintptr_t>(J.obs) & 7))
            return fail(TMCS_E_BUFFER, at + "output buffers must be 8-byte aligned");
        if ((J.shots + 63) / 64 > (uint64_t(1) << 32)) return fail(TMCS_E_INVALID, at + "too many shots");
        const Program &P = J.c->prog;
        if (batch_smem_bytes(P.n_slots, P.max_window_segs, 1) > lim.smem_optin)
            return fail(TMCS_E_INVALID, at + "one 64-shot chunk of this circuit does not fit in shared memory");
        const DeviceProgram *dp = nullptr;
        if ((rc = device_program(J.c, &dp))) return rc;
        if (P.layers.empty()) continue;
        order.push_back({j, dp, double(P.args.size() + 64 * P.layers.size()) * double((J.shots + 63) / 64)});
    }
    std::stable_sort(order.begin(), order.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        bool used = false;
        if ((rc = sig_batch_sample(jobs, n_jobs, st, lim, dev, counter, &used))) return rc;
        if (used) return TMCS_OK;
    }
    // Size classes: jobs whose single 64-shot chunk needs more than 24 KB of
    // shared memory share one launch; smaller circuits get their own launch
    // with a smaller budget (more CTAs per SM, larger tiles). The classes run
    // concurrently on streams forked from `stream` and joined back to it.
    std::vector<Item> cls[2];
    for (const Item &it : order) {
        const Program &P = jobs[it.j].c->prog;
        cls[batch_smem_bytes(P.n_slots, P.max_window_segs, 1) > (size_t(24) << 10) + 16384 + 128 ? 0 : 1].push_back(it);
    }
    const bool fork = !cls[0].empty() && !cls[1].empty();
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    if (fork) {
        if ((e = batch_side_stream(dev, &side, &ev_fork, &ev_join)) != cudaSuccess) return cuda_fail(e, "batch stream");
        if ((e = cudaEventRecord(ev_fork, st)) != cudaSuccess) return cuda_fail(e, "batch fork");
        if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return cuda_fail(e, "batch fork");
    }
    for (int ci = 0; ci < 2; ci++) {
        const std::vector<Item> &ord = cls[ci];
        cudaStream_t cs = (fork && ci == 1) ? side : st;
        unsigned long long *ctr = counter + (ci == 1 ? 16 : 0);
        for (size_t base = 0; base < ord.size(); base += kMaxBatch) {
            const size_t nb = std::min<size_t>(kMaxBatch, ord.size() - base);
            // one shared-memory budget per launch: its largest job at K = 1;
            // each job then takes the largest tile (K <= 4) that fits it
            size_t budget = 0;
            for (size_t i = 0; i < nb; i++) {
                const Program &P = jobs[ord[base + i].j].c->prog;
                budget = std::max(budget, batch_smem_bytes(P.n_slots, P.max_window_segs, 1));
            }
            budget = std::max(budget, size_t(40) << 10);
            budget = std::min(budget, lim.smem_optin);
            BatchArgs B;
            std::memset(&B, 0, sizeof(B));
            uint64_t items = 0;
            for (size_t i = 0; i < nb; i++) {
                const tmcs_job &J = jobs[ord[base + i].j];
                const Program &P = J.c->prog;
                const DeviceProgram *dp = ord[base + i].dp;
                const uint64_t n_cols = (J.shots + 63) / 64;
                int K = ci == 0 ? 1 : 4;  // batch tiles: K = 1 for large circuits, up to 4 for small ones
                while (K > 1 && batch_smem_bytes(P.n_slots, P.max_window_segs, K) > budget) K >>= 1;
                while (K > 1 && (n_cols + K - 1) / K < 8) K >>= 1;
                BatchJob &bj = B.jobs[i];
                bj.layers = dp->layers;
                bj.args = dp->args;
                bj.noise = dp->noise;
                bj.tables = dp->tables;
                bj.det = J.det;
                bj.obs = J.obs;
                bj.n_cols = n_cols;
                bj.last_mask = (J.shots % 64) ? ((uint64_t(1) << (J.shots % 64)) - 1) : ~uint64_t(0);
                bj.item_begin = items;
                bj.n_layers = uint32_t(P.layers.size());
                bj.n_slots = P.n_slots;
                bj.max_window_segs = P.max_window_segs;
                bj.key0 = uint32_t(J.seed);
                bj.key1 = uint32_t(J.seed >> 32);
                bj.K = uint32_t(K);
                items += (n_cols + K - 1) / K;
            }
            B.n_jobs = uint32_t(nb);
            B.total_items = items;
            B.counter = ctr;
            B.status = status;
            const int per_sm = std::max(1, std::min(ci == 0 ? 4 : 3, int(lim.smem_per_sm / (budget + 1024))));
            const uint64_t grid = std::min<uint64_t>(items, uint64_t(lim.sms) * per_sm);
            if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), cs)) != cudaSuccess)
                return cuda_fail(e, "batch queue reset");
            auto kern = ci == 0 ? batch_kernel<1> : batch_kernel<4>;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(budget))) != cudaSuccess)
                return cuda_fail(e, "batch kernel attribute");
            kern<<<unsigned(grid), 256, budget, cs>>>(B);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch kernel launch");
        }
    }
    if (fork) {
        if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) return cuda_fail(e, "batch join");
        if ((e = cudaStreamWaitEvent(st, ev_join, 0)) != cudaSuccess) return cuda_fail(e, "batch join");
    }
    return TMCS_OK;
}

// ---- allocation-free sampling
//
// Some callers cannot allocate device memory once they are running: a
// service whose device memory is owned by another allocator's pool (a direct
// cudaMalloc can fail there or fragment the pool), a real-time host that
// forbids allocation on its request path, or code between stream-ordered
// operations that must not be forced to synchronise the device (cudaMalloc and
// cudaFree can). tmcs_sample_noalloc serves them: instead of the per-circuit
// device program and status word that tmcs_sample allocates on first use, it
// copies the compiled program into this file-scope array (held by every GPU
// that loads the library until the process exits) and runs the same kernel on
// it. Every call shares the array and leaves its own program in it, so calls
// that overlap on the GPU (different streams, or different host threads) race
// and must be serialised by the caller.

constexpr size_t kNoAllocBytes = size_t(8) << 20;  // 8 MiB: status word + one compiled program
constexpr size_t kNoAllocStatusBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device

// Device address of the array on the current device: looked up once per
// device, with that device current, when its status word (the first 256
// bytes) is also cleared. Kernels only ever set bits of that word; it is
// read and cleared by tmcs_check_device, so an expired wait of any call is
// reported until then.
static int noalloc_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(TMCS_E_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
        if ((e = cudaMemset(p, 0, kNoAllocStatusBytes)) != cudaSuccess) return cuda_fail(e, "status clear");
        g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_addr[dev];
    return TMCS_OK;
}

// Status word in the array on device dev (nullptr before its first call).
static uint32_t *noalloc_status(int dev) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    return reinterpret_cast<uint32_t *>(g_noalloc_addr[dev]);
}

static int sample_noalloc(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                          uint64_t *det, uint64_t *obs, void *stream) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    const Program &P = c->prog;
    const size_t b_layers = align256(P.layers.size() * sizeof(Layer));
    const size_t b_args = align256(P.args.size() * 4);
    const size_t b_noise = align256(P.noise.size() * sizeof(NoiseDesc));
    const size_t b_tables = align256(P.tables.size() * 4);
    const size_t need = kNoAllocStatusBytes + b_layers + b_args + b_noise + b_tables;
    if (need > kNoAllocBytes)
        return fail(TMCS_E_INVALID, "compiled program needs " + std::to_string(need) +
                                        " bytes; the allocation-free entry point holds at most " +
                                        std::to_string(kNoAllocBytes) + " (use tmcs_sample_range)");
    if (shots == 0) return fail(TMCS_E_INVALID, "shots must be positive");
    if ((c->n_det && !det) || (c->n_obs && !obs)) return fail(TMCS_E_INVALID, "output buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(det) & 7) || (reinterpret_cast<uintptr_t>(obs) & 7))
        return fail(TMCS_E_BUFFER, "output buffers must be 8-byte aligned");
    const uint64_t n_cols = (shots + 63) / 64;
    if (first_chunk >= (uint64_t(1) << 32) || n_cols > (uint64_t(1) << 32) - first_chunk)
        return fail(TMCS_E_INVALID, "chunk range beyond 2^32");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char *base = nullptr;
    int rc = noalloc_scratch(dev, &base);
    if (rc) return rc;
    DeviceLimits lim;
    if ((rc = device_limits(&lim))) return rc;
    if (kernel_smem_bytes(P.n_slots, P.max_window_segs, 1) > lim.smem_optin)
        return fail(TMCS_E_INVALID, "circuit needs " + std::to_string(P.n_slots) +
                                        " frame slots; one 64-shot chunk does not fit in shared memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // program sections go after the status word (cleared at set-up)
    unsigned char *b = base + kNoAllocStatusBytes;
    // testing knob: record an expired wait in the status word, as a kernel
    // that gave up would, so the tests can check tmcs_check_device reports it
    if (env_int("TMCS_TEST_NOALLOC_EXPIRED", 0) > 0 &&
        (e = cudaMemsetAsync(base, 0x01, 1, st)) != cudaSuccess)
        return cuda_fail(e, "status mark");
    const struct {
        const void *src;
        size_t bytes;
        size_t off;
    } parts[4] = {{P.layers.data(), P.layers.size() * sizeof(Layer), 0},
                  {P.args.data(), P.args.size() * 4, b_layers},
                  {P.noise.data(), P.noise.size() * sizeof(NoiseDesc), b_layers + b_args},
                  {P.tables.data(), P.tables.size() * 4, b_layers + b_args + b_noise}};
    for (const auto &pt : parts)
        if (pt.bytes && (e = cudaMemcpyAsync(b + pt.off, pt.src, pt.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "program copy into the scratch array");
    if (P.layers.empty()) return TMCS_OK;
    LaunchShape s = choose_shape(P, n_cols, lim);
    KernelArgs a{};
    a.layers = reinterpret_cast<const Layer *>(b);
    a.args = reinterpret_cast<const uint32_t *>(b + b_layers);
    a.noise = reinterpret_cast<const NoiseDesc *>(b + b_layers + b_args);
    a.tables = reinterpret_cast<const uint32_t *>(b + b_layers + b_args + b_noise);
    a.status = reinterpret_cast<uint32_t *>(base);
    a.n_layers = uint32_t(P.layers.size());
    a.n_slots = P.n_slots;
    a.max_window_segs = P.max_window_segs;
    a.key0 = uint32_t(seed);
    a.key1 = uint32_t(seed >> 32);
    a.first_chunk = uint32_t(first_chunk);
    a.n_cols = n_cols;
    a.last_mask = (shots % 64) ? ((uint64_t(1) << (shots % 64)) - 1) : ~uint64_t(0);
    a.det = det;
    a.obs = obs;
    if ((e = launch(a, s, st)) != cudaSuccess) return cuda_fail(e, "frame kernel launch");
    return TMCS_OK;
}

}  // namespace tmcs

using namespace tmcs;

extern "C" {

int tmcs_sample(const tmcs_circuit *c, uint64_t shots, uint64_t seed, uint64_t *detector_bits,
                uint64_t *observable_bits, void *stream) {
    return sample_range(c, 0, shots, seed, detector_bits, observable_bits, stream);
}

int tmcs_sample_range(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                      uint64_t *detector_bits, uint64_t *observable_bits, void *stream) {
    return sample_range(c, first_chunk, shots, seed, detector_bits, observable_bits, stream);
}

int tmcs_sample_noalloc(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                        uint64_t *detector_bits, uint64_t *observable_bits, void *stream) {
    return sample_noalloc(c, first_chunk, shots, seed, detector_bits, observable_bits, stream);
}

int tmcs_sample_measurements(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                             uint64_t *meas_bits, void *stream) {
    return sample_measurements(c, first_chunk, shots, seed, meas_bits, stream);
}

int tmcs_fault_signatures(const tmcs_circuit *c, uint64_t first_fault, uint64_t n_faults, uint64_t *detector_bits,
                          uint64_t *observable_bits, void *stream) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    if (first_fault % 64) return fail(TMCS_E_INVALID, "first_fault must be a multiple of 64");
    if (n_faults == 0 || first_fault + n_faults > c->prog.n_faults)
        return fail(TMCS_E_INVALID, "fault range outside [0, tmcs_fault_count)");
    return sample_range(c, 0, n_faults, 0, detector_bits, observable_bits, stream, true, first_fault);
}

int tmcs_debug_gap_counts(double p, const uint32_t *words, uint64_t n, int32_t *counts, int method, void *stream) {
    if (!words || !counts) return fail(TMCS_E_INVALID, "null words or counts");
    if (method < 0 || method > 2) return fail(TMCS_E_INVALID, "method must be 0, 1 or 2");
    std::vector<uint32_t> tables;
    std::vector<double> table_p;
    uint32_t id = 0;
    if (int rc = table_for_p(tables, table_p, p, &id)) return rc;
    float inv = 0.f;
    std::memcpy(&inv, &tables[kGapLen], 4);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *T = nullptr;
    cudaError_t e = cudaMalloc(&T, tables.size() * 4);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (gap table)");
    e = cudaMemcpyAsync(T, tables.data(), tables.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n) {
        const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 4096);
        gap_counts_kernel<<<unsigned(blocks), 256, 0, st>>>(T, inv, -32.0f * inv, words, n, method, counts);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(T);
    return e == cudaSuccess ? TMCS_OK : cuda_fail(e, "gap counts");
}

int tmcs_check_device(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    uint32_t *w = device_status_word(dev);
    if (!w) return fail(TMCS_E_OOM, "cannot allocate the device status word");
    uint32_t v = 0;
    if ((e = cudaMemcpy(&v, w, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "status read");
    if (v && (e = cudaMemset(w, 0, 4)) != cudaSuccess) return cuda_fail(e, "status clear");
    // the allocation-free entry point's own status word (in its array)
    uint32_t v2 = 0;
    if (uint32_t *w2 = noalloc_status(dev)) {
        if ((e = cudaMemcpy(&v2, w2, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "status read");
        if (v2 && (e = cudaMemset(w2, 0, 4)) != cudaSuccess) return cuda_fail(e, "status clear");
    }
    if (v || v2) return fail(TMCS_E_TIMEOUT, "a kernel gave up on a bounded device-side wait");
    return TMCS_OK;
}

int tmcs_launch_shape(const tmcs_circuit *c, int *mode, int *chunks, int *threads, int *ring_window) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(c->mu);
    auto it = c->dev.find(dev);
    const DeviceProgram *dp = it == c->dev.end() ? nullptr : &it->second;
    if (mode) *mode = dp ? dp->tuned_mode : 0;
    if (chunks) *chunks = dp ? dp->tuned_K : 0;
    if (threads) *threads = dp ? dp->tuned_threads : 0;
    if (ring_window) {
        const int k = dp ? dp->tuned_sched : 0;
        *ring_window = (dp && (dp->tuned_mode == 5 || dp->tuned_mode == 6 || dp->tuned_mode == 7) &&
                        size_t(k) < c->sig.sched.size())
                           ? int(c->sig.sched[k].window)
                           : 0;
    }
    return TMCS_OK;
}

int tmcs_launch_flow_shape(const tmcs_circuit *c, int *appliers, int *window, int *global_arena, int *arena_entries) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(c->mu);
    auto it = c->dev.find(dev);
    const bool flow = it != c->dev.end() && it->second.tuned_mode == 7;
    const FlowShape f = flow ? it->second.tuned_flow : FlowShape();
    if (appliers) *appliers = flow ? f.appliers : 0;
    if (window) *window = flow ? f.window : 0;
    if (global_arena) *global_arena = flow && f.global_arena ? 1 : 0;
    if (arena_entries) *arena_entries = flow ? int(f.arena) : 0;
    return TMCS_OK;
}

int tmcs_batch_sample(const tmcs_job *jobs, size_t n_jobs, void *stream) {
    return batch_sample(jobs, n_jobs, stream);
}

}  // extern "C"
