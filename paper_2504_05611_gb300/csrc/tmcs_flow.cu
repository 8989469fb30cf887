// Decoupled event-signature sampler (sm_103a): the walk of the noise streams
// and the application of their events to the detector words run in
// different warps, joined by a shared-memory event arena instead of CTA
// barriers.
//
// What it computes is what sig_kernel computes (Methods "Simulation":
// detector and observable flips as XORs of the output lists of the sampled
// noise events, each event drawn from the Philox4x32-10 streams of the
// sampling specification), with the same schedule: items (64-unit noise
// segments) in steps whose detectors lie in a ring window above the step's
// flush point. The difference is the execution:
//
//  * Walker warps take (tile, step, item, chunk) streams in CTA order from
//    one shared counter, across step and tile boundaries, and append every
//    event as one 32-bit word (event slot, chunk, lane) to their step's
//    region of a circular arena. No lane waits for the end of a step.
//  * Applier warps take steps in order: once every stream of step Q has
//    finished, they apply its events to the ring (shared-memory atomic XORs
//    of the event's output list), write the detectors the step finalises to
//    HBM, clear them, and free the step's arena region.
//
// A step's region has a capacity fixed at launch from the expected number
// of its events (mean + 6 sigma + 64, at most the arena). A walker may start
// a stream of step Q only when Q's region no longer overlaps an unapplied
// step's; an event beyond its region's capacity is held by its lane, which
// stops walking until Q is the step being applied and then XORs the event
// into the ring itself before reporting its stream finished. The ring is
// therefore only ever touched for the step being applied, so it needs one
// window of detectors, while the arena keeps several steps of walking in
// flight. All waits are bounded (kWaitNs); on expiry the kernel sets bit 0
// of the status word and every warp leaves.
#include <cuda.h>  // CUtensorMap (encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "tmcs_device.cuh"
#include "tmcs_internal.h"

namespace tmcs {

constexpr uint32_t kFlowSlots = 64;       // steps in flight (done / count slots)
// events an applier lane loads at once (build-time tuning value)
#ifndef TMCS_FLOW_APPLY_BATCH
#define TMCS_FLOW_APPLY_BATCH 4
#endif
constexpr uint32_t kFlowApplyBatch = TMCS_FLOW_APPLY_BATCH;
constexpr uint32_t kFlowMinArena = 1024;  // smallest useful arena (entries)
// arena entry of an event that flips nothing (no event word takes this value:
// flow_shape keeps event slots x 64 x K below 2^32)
constexpr uint32_t kFlowDead = 0xFFFFFFFFu;
constexpr uint32_t kFlowMaxArena = 65536;

struct FlowArgs {
    CUtensorMap tmap;           // det as a [n_det][ld] uint64 tensor (tensor-store flush), when tma_rows > 0
    const NoiseDesc *noise;
    const uint32_t *tables;
    const uint4 *item_desc;     // walker descriptors, two uint4 per item (see SigSchedule::item_desc)
    const uint4 *steps;         // item_begin, item_end, flush_lo, flush_hi
    const float *step_events;   // expected events per chunk of each step
    const uint32_t *ev_ent;     // two words per event slot, then the overflow lists
    uint32_t n_steps, n_items, window_mask, n_obs;
    uint32_t arena;             // arena entries (power of two)
    uint32_t test_cap;          // testing: capacity of every step's region (0: from step_events)
    uint32_t smem_tables;       // gap tables staged in shared memory (count), 0: read from global
    uint32_t walkers;           // walker warps; the CTA's other warps apply
    uint32_t key0, key1, first_chunk;
    uint32_t vec_out;           // det 16-byte aligned and n_cols even: 16-byte output stores
    uint64_t n_cols, last_mask, n_tiles;
    uint64_t ld;                // words between output rows (the call's column count; a launch may cover a slice)
    uint32_t *garena;           // arena in global memory (a slice of `arena` entries per CTA), or null
    uint32_t tma_rows;          // detector rows per tensor-store box of the flush (0: plain stores)
    uint64_t col_base;          // column of this launch's column 0 in the tensor map (sliced launches)
    uint64_t *det;
    uint64_t *obs;
    uint32_t *status;
};

// Arena positions are kept modulo 2^32: only differences (less than the
// arena size plus one step's region) and positions modulo the arena size
// (a power of two) are used.
struct FlowCtl {
    uint32_t next;                 // streams handed out (CTA sequence; a launch keeps it below 2^31)
    uint32_t u_applied;            // arena position of the first unapplied step
    uint32_t applied;              // steps applied (CTA sequence)
    uint32_t abort;                // a bounded wait expired
    uint32_t app_stop;             // appliers leave (written by applier thread 0 before a barrier)
    uint32_t done[kFlowSlots];     // finished streams of step Q (slot Q mod kFlowSlots)
    uint32_t cnt[kFlowSlots];      // arena entries reserved by step Q's events
};

// Shared-memory regions (same order and sizes as flow_smem_bytes): ring and
// observable rows, step table (item end, region capacity, region offset per
// step, then the tile's total), gap tables, arena.
struct FlowSmem {
    uint64_t *ring;
    uint32_t *send, *scap, *soff;
    uint32_t *stab;
    uint32_t *arena;
};

__host__ __device__ inline size_t flow_ring_bytes(uint32_t W, uint32_t n_obs, int K) {
    return ((size_t(W) + n_obs) * size_t(K) * 8 + 15) & ~size_t(15);
}
__host__ __device__ inline size_t flow_step_bytes(uint32_t n_steps) {
    return ((3 * size_t(n_steps) + 1) * 4 + 15) & ~size_t(15);
}

__device__ __forceinline__ FlowSmem flow_layout(uint64_t *smem, const FlowArgs &A, int K) {
    FlowSmem S;
    unsigned char *b = reinterpret_cast<unsigned char *>(smem);
    S.ring = smem;
    b += flow_ring_bytes(A.window_mask + 1u, A.n_obs, K);
    S.send = reinterpret_cast<uint32_t *>(b);
    S.scap = S.send + A.n_steps;
    S.soff = S.scap + A.n_steps;
    b += flow_step_bytes(A.n_steps);
    S.stab = reinterpret_cast<uint32_t *>(b);
    b += size_t(A.smem_tables) * kTableWords * 4;
    S.arena = reinterpret_cast<uint32_t *>(b);
    return S;
}

template <int K>
struct FlowLog {
    static constexpr uint32_t v = K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : K == 8 ? 3 : 4;
};

__device__ __forceinline__ unsigned long long ld_shared_volatile64(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// XORs one event into the ring: word wv = event slot << (6 + log2 K) |
// chunk << 6 | lane, v = the slot's two words (an entry is observable flag
// << 29 | output index; observables are the rows after the ring).
template <int K>
__device__ __forceinline__ void flow_put(const FlowArgs &A, uint64_t *ring, uint32_t wv, uint2 v) {
    if (v.x == kEvNone) return;
    const uint32_t lane = wv & 63u, k = (wv >> 6) & uint32_t(K - 1);
    uint32_t *base = reinterpret_cast<uint32_t *>(ring) + 2u * k + (lane >> 5);
    const uint32_t bit = 1u << (lane & 31u);
    const uint32_t obs_row = A.window_mask + 1u;
    auto put = [&](uint32_t e) {
        const uint32_t idx = e & 0x1FFFFFFFu;
        const uint32_t row = (e & (1u << 29)) ? obs_row + idx : (idx & A.window_mask);
        atomicXor(base + size_t(row) * (2u * uint32_t(K)), bit);
    };
    if (v.x & kEvOverflow) {
        const uint32_t *ov = A.ev_ent + (v.x & ~kEvOverflow);
        for (uint32_t x = 0; x < v.y; x++) put(__ldg(ov + x));
    } else {
        put(v.x);
        if (v.y != kEvNone) put(v.y);
    }
}

template <int K>
__device__ __forceinline__ void flow_put_word(const FlowArgs &A, uint64_t *ring, uint32_t wv) {
    if (wv == kFlowDead) return;
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(A.ev_ent) + (wv >> (6u + FlowLog<K>::v)));
    flow_put<K>(A, ring, wv, v);
}

// Walker warps. Every lane holds at most one stream; streams are handed out
// in CTA order (tile, step, item, chunk). An iteration is a window of
// W Philox calls (two draws each) of every walking lane's stream,
// with the window's events kept in registers; then the warp reserves arena
// entries for all of them at once, together with the lanes whose streams
// belong to the same step (one shared atomic per step and warp), reports the
// streams that ended and refills those lanes. Streams longer than a window
// continue in the next one. The per-iteration work of the warp (refill,
// reservation, completion) is thus shared by up to 2 W draws per lane.
template <int K, int W, bool SMT, bool GA>
__device__ __forceinline__ void flow_walk(const FlowArgs &A, const FlowSmem &S, FlowCtl &C, uint32_t nt,
                                          uint32_t nv_last, const uint32_t *tabs) {
    constexpr uint32_t LK = FlowLog<K>::v;
    constexpr int NE = 2 * W;  // events a lane can draw per window
    static_assert(NE < 16, "event counts per window are reserved with four count-bit ballots at most");
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t n_steps = A.n_steps, amask = A.arena - 1u;
    // the arena: shared memory, or this CTA's slice of a global buffer
    // (L2-resident; entries written and read past L1)
    uint32_t *const arena = GA ? A.garena + size_t(blockIdx.x) * A.arena : S.arena;
    const uint32_t per_tile = A.n_items << LK;
    const uint32_t total = nt * per_tile;
    const uint32_t c_tile = S.soff[n_steps];
    bool have = false, live = false, ended = false, exhausted = false;
    uint32_t tcur = 0xFFFFFFFFu, tbase = 0;
    // the lane's stream: step Q, its region (capacity, low word of its
    // unwrapped arena position, gate), Philox stream words, call counter,
    // first event slot, kind, Pauli counts, gap table offset, chunk tag,
    // position and length in trials
    uint32_t Q = 0, cap = 0, uq = 0, gate = 0;
    PhiloxStream ps{0u, 0u, 0u};
    // event words: slot << S | chunk << 6 | lane (S = 6 + log2 K) with slot =
    // ubase + (pos >> 6) kp + (Pauli index - 1), formed as
    // evb + (pos >> 6) kpm + pos + (Pauli index - 1) 2^S, where evb = ubase 2^S
    // + chunk 2^6 and kpm = kp 2^S - 64 (all modulo 2^32)
    constexpr uint32_t S_EV = 6u + LK;
    uint32_t call = 0, evb = 0, kind = 0, npauli = 1, kpm = 0, toff = 0, t1 = 0, t2 = 0, live_k = 0;
    int pos = -1, n_trials = 0;
    float inv = 0.f, c32 = 0.f;
    // the window's events; ev[held .. ne) are events that did not fit their
    // step's region and wait for it to be the step being applied
    uint32_t ev[NE];
    uint32_t ne = 0, held = 0;
    uint32_t t_wait = 0, iter = 0;
    bool waiting = false;
    for (;;) {
        if ((iter++ & 7u) == 0u && __any_sync(0xFFFFFFFFu, ld_shared_volatile(&C.abort) != 0u)) return;
        if (!have && !exhausted) {
            const uint32_t g = grab_index(&C.next);
            if (g >= total) {
                exhausted = true;
            } else {
                if (tcur == 0xFFFFFFFFu || g - tbase >= per_tile) {
                    tcur = g / per_tile;
                    tbase = tcur * per_tile;
                }
                const uint32_t sl = g - tbase;
                const uint32_t it = sl >> LK, k = sl & uint32_t(K - 1);
                const uint4 d0 = __ldg(A.item_desc + 2 * it), d1 = __ldg(A.item_desc + 2 * it + 1);
                const uint32_t q = d1.x >> 17;
                Q = tcur * n_steps + q;
                const uint32_t U = tcur * c_tile + S.soff[q];  // modulo 2^32
                cap = S.scap[q];
                gate = U + cap - A.arena;
                uq = U;
                kind = d1.x & 7u;
                npauli = (d1.x >> 3) & 15u;
                kpm = (((d1.x >> 7) & 15u) << S_EV) - 64u;
                toff = (d1.y & 0x1FFFu) * kTableWords;
                inv = __uint_as_float(d1.z);
                c32 = -32.0f * inv;  // exact (a power-of-two scaling)
                live_k = d1.w;
                if (kind == N_PC1) {
                    t1 = __ldg(&A.noise[d1.y >> 13].t1);
                    t2 = __ldg(&A.noise[d1.y >> 13].t2);
                }
                const uint32_t nv = tcur == nt - 1u ? nv_last : uint32_t(K);
                const uint32_t chunk = A.first_chunk + (blockIdx.x + tcur * gridDim.x) * uint32_t(K) + k;
                // Philox round 1 of this stream from the descriptor's product
                // of the op index (counter words: call, chunk, op, segment)
                ps.a0 = d0.x ^ chunk ^ A.key0;
                ps.a1 = d0.y;
                ps.a3 = d0.z ^ A.key1;
                evb = (d0.w << S_EV) | (k << 6);
                // chunks past the end of the call (ragged last tile): no trials
                n_trials = k < nv ? 64 * int(((d1.x >> 11) & 63u) + 1u) : 0;
                call = 0;
                pos = -1;
                have = true;
                live = false;
                ended = false;
            }
        }
        // the stream may start once its step's arena region is free and the
        // step is within the slots in flight
        if (have && !live) {
            // acquire: the appliers' last reads of the region and their
            // reset of the step's counters precede our writes. The region
            // is free once u_applied has reached the gate (signed
            // difference: positions are modulo 2^32).
            const uint32_t ua = ld_acquire_shared(&C.u_applied);
            if (int32_t(ua - gate) >= 0 && Q - ld_acquire_shared(&C.applied) < kFlowSlots) live = true;
        }
        // events held back by a full region: once step Q is the one being
        // applied, XOR them into the ring directly
        if (held < ne && ld_acquire_shared(&C.applied) == Q) {
#pragma unroll
            for (int j = 0; j < NE; j++)
                if (uint32_t(j) >= held && uint32_t(j) < ne) flow_put_word<K>(A, S.ring, ev[j]);
            held = ne;
        }
        const bool walk = live && !ended && held == ne;
        const uint32_t wm = __ballot_sync(0xFFFFFFFFu, walk);
        if (wm) {
            if (walk) {
                ne = 0;
                held = 0;
                // the window's W Philox calls and 2W gap counts do not depend
                // on one another: straight-line code, so their latencies
                // overlap; draws after the stream's last one are computed
                // and discarded (the warp runs them for its other lanes)
                uint32_t wp[NE];
                int gp[NE];
                // one table read per gap when every walking lane's p allows
                // it (warp-uniform choice), else the two-read count
                if (__all_sync(wm, fabsf(inv) < kNearInv)) {
#pragma unroll
                    for (int c = 0; c < W; c++) {
                        const uint4 w = philox_call(ps, call + uint32_t(c), A.key0, A.key1);
                        gp[2 * c] = gap_count_near_at<SMT>(tabs, toff - 1u, inv, c32, w.x);
                        gp[2 * c + 1] = gap_count_near_at<SMT>(tabs, toff - 1u, inv, c32, w.z);
                        wp[2 * c] = w.y;
                        wp[2 * c + 1] = w.w;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < W; c++) {
                        const uint4 w = philox_call(ps, call + uint32_t(c), A.key0, A.key1);
                        gp[2 * c] = gap_count_est<SMT>(tabs + toff, inv, c32, w.x);
                        gp[2 * c + 1] = gap_count_est<SMT>(tabs + toff, inv, c32, w.z);
                        wp[2 * c] = w.y;
                        wp[2 * c + 1] = w.w;
                    }
                }
                call += uint32_t(W);
                // positions in draw order (increasing): every draw before the
                // one that passes the end of the segment is an event
                int pd[NE];
#pragma unroll
                for (int d = 0; d < NE; d++) {
                    pos += 1 + gp[d];
                    pd[d] = pos;
                }
                ne = 0;
#pragma unroll
                for (int d = 0; d < NE; d++) ne = pd[d] < n_trials ? uint32_t(d + 1) : ne;
                ended = pos >= n_trials;
                // Pauli index - 1: PAULI_CHANNEL_1 thresholds, else uniform
                // (the thresholds are only looked at in warps that have a
                // PAULI_CHANNEL_1 lane). An event whose Pauli index flips
                // nothing in any unit of the segment becomes kFlowDead: it
                // keeps its arena entry but costs the appliers no table read.
                auto words = [&](auto pc1) {
#pragma unroll
                    for (int d = 0; d < NE; d++) {
                        uint32_t k1 = __umulhi(wp[d], npauli);
                        if constexpr (decltype(pc1)::value)
                            if (kind == N_PC1) k1 = wp[d] < t1 ? 0u : wp[d] < t2 ? 2u : 1u;
                        const uint32_t pu = uint32_t(pd[d]);
                        const uint32_t wd = (pu >> 6) * kpm + (evb + pu) + (k1 << S_EV);
                        ev[d] = wd | (((live_k >> k1) & 1u) - 1u);  // kFlowDead when not live
                    }
                };
                if (__any_sync(wm, kind == N_PC1)) words(std::true_type{});
                else words(std::false_type{});
            }
            // reserve the window's events: lanes of the same step share one
            // atomic; a lane's offset among them from bit ballots of its count
            const bool res = walk && ne != 0;
            const uint32_t em = __ballot_sync(0xFFFFFFFFu, res);
            if (res) {
                const uint32_t peers = __match_any_sync(em, Q);
                // counts reach NE (6 or 8 for windows of 3 or 4 calls): one
                // ballot per bit of the count
                constexpr int NB = NE >= 8 ? 4 : 3;
                uint32_t n = 0, off = 0;
#pragma unroll
                for (int bit = 0; bit < NB; bit++) {
                    const uint32_t bm = __ballot_sync(em, (ne >> bit) & 1u) & peers;
                    n += uint32_t(__popc(bm)) << bit;
                    off += uint32_t(__popc(bm & lt)) << bit;
                }
                const uint32_t leader = uint32_t(__ffs(peers)) - 1u;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(&C.cnt[Q & (kFlowSlots - 1u)], n);
                const uint32_t idx = __shfl_sync(peers, base, int(leader)) + off;
                // entries past the region's capacity stay in ev[] (held)
                held = idx >= cap ? 0u : min(ne, cap - idx);
                // the entries are contiguous unless they wrap past the
                // arena's end
                const uint32_t a0 = (uq + idx) & amask;
                if (a0 + uint32_t(NE) <= A.arena) {
                    uint32_t *const at = arena + a0;
#pragma unroll
                    for (int j = 0; j < NE; j++)
                        if (uint32_t(j) < held) {
                            if constexpr (GA) __stcg(at + j, ev[j]);
                            else at[j] = ev[j];
                        }
                } else {
#pragma unroll
                    for (int j = 0; j < NE; j++)
                        if (uint32_t(j) < held) {
                            if constexpr (GA) __stcg(arena + ((a0 + uint32_t(j)) & amask), ev[j]);
                            else arena[(a0 + uint32_t(j)) & amask] = ev[j];
                        }
                }
            }
        }
        // a stream whose walk ended and whose events are all stored or
        // applied is reported to its step
        const bool complete = have && ended && held == ne;
        const uint32_t cm = __ballot_sync(0xFFFFFFFFu, complete);
        if (complete) {
            // the stream's events (stored or applied by this lane) precede
            // the count: a release add per lane (cheaper than grouping the
            // lanes of a step behind one add)
            red_release_add_shared(&C.done[Q & (kFlowSlots - 1u)], 1u);
            have = false;
            live = false;
            ended = false;
            ne = 0;
            held = 0;
        }
        if (wm | cm) {
            waiting = false;
            continue;
        }
        // nothing to walk: every lane is done, gated or holding events
        if (!__any_sync(0xFFFFFFFFu, have)) return;
        if (__any_sync(0xFFFFFFFFu, ld_shared_volatile(&C.abort) != 0u)) return;
        if (!waiting) {
            t_wait = uint32_t(globaltimer_ns());
            waiting = true;
        } else if (uint32_t(globaltimer_ns()) - t_wait > uint32_t(kWaitNs)) {
            if (lane == 0) {
                C.abort = 1u;
                atomicOr(A.status, 1u);
            }
            return;
        }
        __nanosleep(64);
    }
}

__device__ __forceinline__ void flow_bar(uint32_t nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(shared_addr(src))
                 : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Flush of detectors [z, w) with tensor stores: the rows of each ring
// segment (at most two: the ring wraps) go out as boxes of tma_rows rows x K
// chunk words issued by the first applier warp, starting at a ring row whose
// address is 128-byte aligned; the few rows before that point and after the
// last whole box are written with plain stores. Every row is cleared: the
// boxes' rows once the tensor stores have read them. The last column of the
// call (in the call's last tile) gets its pad bits masked in the ring first.
// Every applier has fenced its ring writes for the async proxy before the
// barrier that precedes this call. Ends with the boxes' rows cleared; the
// caller's barrier follows.
// Rows [d0, d1) of one contiguous stretch of the ring: plain head rows
// [d0, dh) up to the first 128-byte aligned ring row, whole boxes [dh, db),
// plain tail rows [db, d1).
struct FlushSeg {
    uint32_t d0, dh, db, d1;
};

template <int K>
__device__ __forceinline__ FlushSeg flush_seg(uint32_t d, uint32_t e, uint32_t mask, uint32_t R) {
    constexpr uint32_t AL = K >= 16 ? 1u : 16u / uint32_t(K);  // ring rows per 128 bytes
    FlushSeg g;
    g.d0 = d;
    g.d1 = e;
    g.dh = min(e, d + (AL - (d & mask) % AL) % AL);
    g.db = g.dh + (e - g.dh) / R * R;
    return g;
}

template <int K>
__device__ __forceinline__ void flush_plain_rows(const FlowArgs &A, const FlowSmem &S, const FlushSeg &g,
                                                 uint64_t col0, uint32_t nv, uint32_t at, uint32_t nthr) {
    const uint32_t nh = g.dh - g.d0, nt = g.d1 - g.db;
    for (uint32_t i = at; i < (nh + nt) * uint32_t(K); i += nthr) {
        const uint32_t row = i / uint32_t(K), k = i % uint32_t(K);
        const uint32_t d = row < nh ? g.d0 + row : g.db + (row - nh);
        uint64_t *r = S.ring + size_t(d & A.window_mask) * K + k;
        const uint64_t v = *r;
        *r = 0ull;
        if (k < nv) __stcs(reinterpret_cast<unsigned long long *>(A.det + uint64_t(d) * A.ld + col0 + k), v);
    }
}

template <int K>
__device__ __forceinline__ void flush_clear_boxes(const FlowArgs &A, const FlowSmem &S, const FlushSeg &g,
                                                  uint32_t at, uint32_t nthr) {
    ulonglong2 *base = reinterpret_cast<ulonglong2 *>(S.ring + size_t(g.dh & A.window_mask) * K);
    const uint32_t nw = (g.db - g.dh) * uint32_t(K) / 2u;
    for (uint32_t i = at; i < nw; i += nthr) base[i] = make_ulonglong2(0ull, 0ull);
}

// Flush of detectors [z, w) (w - z at most the ring's rows) with tensor
// stores: the rows of each stretch of the ring (at most two: the ring wraps)
// go out as boxes of tma_rows rows x K chunk words issued by the first
// applier warp, each starting at a 128-byte aligned ring row; the few rows
// before the first aligned row and after the last whole box are written with
// plain stores. Every row is cleared: the boxes' rows once the tensor stores
// have read them. The call's last column (in the call's last tile) gets its
// pad bits masked in the ring first. Every applier has fenced its ring
// writes for the async proxy before the barrier that precedes this call.
// Ends with the boxes' rows cleared; the caller's barrier follows.
template <int K>
__device__ __forceinline__ void flow_flush_tma(const FlowArgs &A, const FlowSmem &S, uint32_t z, uint32_t w,
                                               uint64_t col0, uint32_t nv, uint32_t at, uint32_t nthr) {
    const uint32_t mask = A.window_mask, R = A.tma_rows;
    if (col0 + uint64_t(K) > A.n_cols - 1) {  // this tile holds the call's last column
        const uint32_t kl = uint32_t(A.n_cols - 1 - col0);
        for (uint32_t i = at; i < w - z; i += nthr) S.ring[size_t((z + i) & mask) * K + kl] &= A.last_mask;
        fence_proxy_async_shared();
        flow_bar(nthr);
    }
    const uint32_t split = min(w, z + (mask + 1u - (z & mask)));  // first row past the ring's end
    const FlushSeg g0 = flush_seg<K>(z, split, mask, R), g1 = flush_seg<K>(split, w, mask, R);
    const uint32_t n0 = (g0.db - g0.dh) / R, nbox = n0 + (g1.db - g1.dh) / R;
    const bool issuer = at < 32u;
    if (issuer) {
        const int x = int(A.col_base + col0);
        for (uint32_t b = at; b < nbox; b += 32u) {
            const uint32_t d = b < n0 ? g0.dh + b * R : g1.dh + (b - n0) * R;
            tma_store_2d(&A.tmap, x, int(d), S.ring + size_t(d & mask) * K);
        }
        tma_commit();
    }
    flush_plain_rows<K>(A, S, g0, col0, nv, at, nthr);
    flush_plain_rows<K>(A, S, g1, col0, nv, at, nthr);
    if (issuer) tma_wait_read();
    flow_bar(nthr);
    flush_clear_boxes<K>(A, S, g0, at, nthr);
    flush_clear_boxes<K>(A, S, g1, at, nthr);
}

// Applier warps: steps in CTA order.
template <int K, bool GA>
__device__ __forceinline__ void flow_apply(const FlowArgs &A, const FlowSmem &S, FlowCtl &C, uint32_t nt,
                                           uint32_t nv_last) {
    constexpr uint32_t LK = FlowLog<K>::v;
    const uint32_t nthr = blockDim.x - 32u * A.walkers;
    const uint32_t at = threadIdx.x - 32u * A.walkers;
    const uint32_t amask = A.arena - 1u, mask = A.window_mask;
    const uint32_t obs_row = A.window_mask + 1u;
    const uint2 *ev2 = reinterpret_cast<const uint2 *>(A.ev_ent);
    const uint32_t *const arena = GA ? A.garena + size_t(blockIdx.x) * A.arena : S.arena;
    // tensor-store flush: needs the ring 128-byte aligned in shared memory
    // and boxes of a whole number of 128-byte ring stretches (each box then
    // starts aligned)
    const bool tma = (K % 2 == 0) && A.tma_rows != 0 && (A.tma_rows * uint32_t(K)) % 16u == 0 &&
                     (shared_addr(S.ring) & 127u) == 0;
    uint32_t U = 0;  // arena position of step Q, modulo 2^32
    for (uint32_t T = 0; T < nt; T++) {
        const uint64_t tile = uint64_t(blockIdx.x) + uint64_t(T) * gridDim.x;
        const uint64_t col0 = tile * uint64_t(K);
        const uint32_t nv = T == nt - 1u ? nv_last : uint32_t(K);
        for (uint32_t q = 0; q < A.n_steps; q++) {
            const uint32_t Q = T * A.n_steps + q;
            const uint4 st = __ldg(A.steps + q);
            const uint32_t need = (st.y - st.x) << LK;
            const uint32_t slot = Q & (kFlowSlots - 1u);
            // thread 0 waits for the step's streams and decides for all
            // appliers whether they go on (one value read after the barrier,
            // so every applier thread leaves or none does)
            if (at == 0) {
                uint32_t stop = ld_shared_volatile(&C.abort);
                if (!stop && ld_shared_volatile(&C.done[slot]) != need) {
                    const uint64_t t0 = globaltimer_ns();
                    while (ld_shared_volatile(&C.done[slot]) != need) {
                        if (ld_shared_volatile(&C.abort)) {
                            stop = 1u;
                            break;
                        }
                        if (globaltimer_ns() - t0 > kWaitNs) {
                            C.abort = 1u;
                            atomicOr(A.status, 1u);
                            stop = 1u;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                C.app_stop = stop;
            }
            flow_bar(nthr);
            if (C.app_stop) {
                if (tma && at < 32u) tma_wait_all();
                return;
            }
            __threadfence_block();  // the walkers' events precede the reads below
            const uint32_t n = min(ld_shared_volatile(&C.cnt[slot]), S.scap[q]);
            const uint32_t u0 = U;
            for (uint32_t e = at; e < n; e += nthr * kFlowApplyBatch) {
                uint32_t wv[kFlowApplyBatch];
                uint2 v[kFlowApplyBatch];
#pragma unroll
                for (uint32_t j = 0; j < kFlowApplyBatch; j++) {
                    const uint32_t i = e + j * nthr;
                    if constexpr (GA) wv[j] = i < n ? __ldcg(arena + ((u0 + i) & amask)) : 0u;
                    else wv[j] = i < n ? arena[(u0 + i) & amask] : 0u;
                }
#pragma unroll
                for (uint32_t j = 0; j < kFlowApplyBatch; j++)
                    v[j] = e + j * nthr < n && wv[j] != kFlowDead ? __ldg(ev2 + (wv[j] >> (6u + LK)))
                                                                   : make_uint2(kEvNone, kEvNone);
#pragma unroll
                for (uint32_t j = 0; j < kFlowApplyBatch; j++) flow_put<K>(A, S.ring, wv[j], v[j]);
            }
            if (tma) fence_proxy_async_shared();  // ring writes before the tensor stores read them
            flow_bar(nthr);
            // every applier has read the step's arena entries (barrier): the
            // region is free for the walkers of later steps while the
            // appliers flush (release: those reads precede the hand-off)
            U += S.scap[q];
            if (at == 0) st_release_shared(&C.u_applied, U);
            // detectors [flush_lo, flush_hi) are final: write and clear them
            const uint32_t nd = st.w - st.z;
            bool vec_done = false;
            if constexpr (K % 2 == 0) {
                if (tma) {
                    vec_done = true;
                    flow_flush_tma<K>(A, S, st.z, st.w, col0, nv, at, nthr);
                } else if (A.vec_out) {
                    vec_done = true;
                    constexpr uint32_t H = uint32_t(K) / 2u;
                    for (uint32_t i = at; i < nd * H; i += nthr) {
                        const uint32_t d = st.z + i / H, k = 2u * (i % H);
                        ulonglong2 *r = reinterpret_cast<ulonglong2 *>(S.ring + size_t(d & mask) * K + k);
                        ulonglong2 v = *r;
                        *r = make_ulonglong2(0ull, 0ull);
                        if (k >= nv) continue;
                        const uint64_t col = col0 + k;
                        if (col == A.n_cols - 1) v.x &= A.last_mask;
                        if (col + 1 == A.n_cols - 1) v.y &= A.last_mask;
                        unsigned long long *out =
                            reinterpret_cast<unsigned long long *>(A.det + uint64_t(d) * A.ld + col);
                        if (k + 1 < nv) __stcs(reinterpret_cast<ulonglong2 *>(out), v);
                        else __stcs(out, v.x);
                    }
                }
            }
            if (!vec_done) {
                for (uint32_t i = at; i < nd * uint32_t(K); i += nthr) {
                    const uint32_t d = st.z + i / uint32_t(K), k = i % uint32_t(K);
                    uint64_t *r = S.ring + size_t(d & mask) * K + k;
                    uint64_t v = *r;
                    *r = 0ull;
                    if (k >= nv) continue;
                    const uint64_t col = col0 + k;
                    if (col == A.n_cols - 1) v &= A.last_mask;
                    __stcs(reinterpret_cast<unsigned long long *>(A.det + uint64_t(d) * A.ld + col), v);
                }
            }
            if (q == A.n_steps - 1u) {
                uint64_t *ob = S.ring + size_t(obs_row) * K;
                for (uint32_t i = at; i < A.n_obs * uint32_t(K); i += nthr) {
                    const uint32_t o = i / uint32_t(K), k = i % uint32_t(K);
                    uint64_t v = ob[i];
                    ob[i] = 0ull;
                    if (k >= nv) continue;
                    const uint64_t col = col0 + k;
                    if (col == A.n_cols - 1) v &= A.last_mask;
                    A.obs[uint64_t(o) * A.ld + col] = v;
                }
            }
            flow_bar(nthr);
            if (at == 0) {
                C.done[slot] = 0u;
                C.cnt[slot] = 0u;
                // release: every applier's ring writes of this step (ordered
                // before by the barrier) and the counter resets precede the
                // hand-off of the ring window and the step's slots
                st_release_shared(&C.applied, Q + 1u);
            }
        }
    }
    if (tma && at < 32u) tma_wait_all();  // the tensor stores have written the outputs
}

// CTA size the kernel is compiled for (its register budget follows from it)
#ifndef TMCS_FLOW_MAX_THREADS
#define TMCS_FLOW_MAX_THREADS 1024
#endif

template <int K, int W, bool GA>
__global__ void __launch_bounds__(TMCS_FLOW_MAX_THREADS, 1) flow_kernel(const __grid_constant__ FlowArgs A) {
    extern __shared__ __align__(128) uint64_t smem[];
    __shared__ FlowCtl C;
    if (uint64_t(blockIdx.x) >= A.n_tiles) return;
    const FlowSmem S = flow_layout(smem, A, K);
    const uint32_t tid = threadIdx.x, T_ = blockDim.x;
    const uint32_t rows = A.window_mask + 1u;
    for (uint32_t i = tid; i < (rows + A.n_obs) * uint32_t(K); i += T_) S.ring[i] = 0ull;
    for (uint32_t i = tid; i < A.smem_tables * kTableWords; i += T_) S.stab[i] = __ldg(A.tables + i);
    // region capacities: mean + 6 sigma + 64 of the step's events over K
    // chunks (Poisson-like counts), at most the arena; steps without items
    // hold none
    for (uint32_t i = tid; i < A.n_steps; i += T_) {
        const uint4 st = __ldg(A.steps + i);
        const float mu = __ldg(A.step_events + i) * float(K);
        uint32_t cap = A.test_cap ? A.test_cap : uint32_t(ceilf(mu + 6.0f * sqrtf(mu) + 64.0f));
        cap = st.y > st.x ? min(cap, A.arena) : 0u;
        S.send[i] = st.y;
        S.scap[i] = cap;
    }
    if (tid < kFlowSlots) {
        C.done[tid] = 0u;
        C.cnt[tid] = 0u;
    }
    if (tid == 0) {
        C.next = 0u;
        C.u_applied = 0u;
        C.applied = 0u;
        C.abort = 0u;
        C.app_stop = 0u;
    }
    __syncthreads();
    // region offsets: exclusive prefix sum of the capacities (warp 0)
    if (tid < 32) {
        const uint32_t per = (A.n_steps + 31u) / 32u, lo = tid * per, hi = min(A.n_steps, lo + per);
        uint32_t sum = 0;
        for (uint32_t i = lo; i < hi; i++) sum += S.scap[i];
        uint32_t incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (int(tid) >= o) incl += v;
        }
        uint32_t run = incl - sum;
        for (uint32_t i = lo; i < hi; i++) {
            S.soff[i] = run;
            run += S.scap[i];
        }
        if (tid == 31) S.soff[A.n_steps] = incl;
    }
    const uint64_t G = gridDim.x;
    const uint32_t nt = uint32_t((A.n_tiles - blockIdx.x + G - 1) / G);
    const uint64_t last = uint64_t(blockIdx.x) + uint64_t(nt - 1) * G;
    const uint64_t rem = A.n_cols - last * K;
    const uint32_t nv_last = rem < uint64_t(K) ? uint32_t(rem) : uint32_t(K);
    __syncthreads();
    if ((tid >> 5) >= A.walkers) flow_apply<K, GA>(A, S, C, nt, nv_last);
    else if (A.smem_tables) flow_walk<K, W, true, GA>(A, S, C, nt, nv_last, S.stab);
    else flow_walk<K, W, false, GA>(A, S, C, nt, nv_last, A.tables);
}

// ------------------------------------------------------------------- host

static int env_int_flow(const char *name, int dflt) {
    const char *v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

// Philox calls per walker window: TMCS_FLOW_WINDOW (2 to 4) when set, else
// the requested one (2 to 4), else 3
static int flow_window(int window) {
    const int wforce = env_int_flow("TMCS_FLOW_WINDOW", 0);
    if (wforce >= 2 && wforce <= 4) return wforce;
    return (window >= 2 && window <= 4) ? window : 3;
}

static size_t flow_fixed_bytes(const SigProgram &G, int sched, uint32_t n_obs, int K) {
    const SigSchedule &S = G.sched[sched];
    return flow_ring_bytes(S.window, n_obs, K) + flow_step_bytes(uint32_t(S.steps.size()));
}

bool flow_shape(const tmcs_circuit *c, int sched, int K, int threads, int appliers, size_t budget, FlowShape *out,
                bool global_arena, int window) {
    const SigProgram &G = c->sig;
    if (!G.ok || sched < 0 || size_t(sched) >= G.sched.size()) return false;
    const SigSchedule &S = G.sched[sched];
    if (S.lag || S.steps.empty() || S.steps.size() > kFlowMaxSteps || S.step_events.size() != S.steps.size())
        return false;
    if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16) return false;
    if (threads < 64 || threads > TMCS_FLOW_MAX_THREADS || threads % 32 || appliers < 1 || appliers >= threads / 32)
        return false;
    // event words: slot << (6 + log2 K) | chunk << 6 | lane must fit 32 bits
    // and never equal kFlowDead
    if (uint64_t(G.n_event_slots) * 64u * uint64_t(K) >= (uint64_t(1) << 32)) return false;
    const size_t fixed = flow_fixed_bytes(G, sched, uint32_t(c->n_obs), K);
    const size_t tabs = G.tables.size() * 4;
    auto arena_for = [&](size_t used) {
        uint32_t a = kFlowMaxArena;
        while (a >= kFlowMinArena && used + size_t(a) * 4 > budget) a >>= 1;
        return a;
    };
    FlowShape s;
    s.sched = sched;
    s.K = K;
    s.threads = threads;
    s.appliers = appliers;
    // global arena: tables stay in shared memory, the arena is an L2-resident
    // slice per CTA of the library's scratch buffer
    if (global_arena) {
        if (fixed + tabs > budget) return false;
        const int gforce = env_int_flow("TMCS_FLOW_GARENA", 0);  // tuning knob: global arena entries per CTA
        s.arena = (gforce >= int(kFlowMinArena) && !(gforce & (gforce - 1))) ? uint32_t(gforce) : 65536u;
        s.smem_tables = true;
        s.smem = fixed + tabs;
        s.garena_ctas = 0;  // set by the caller (resident CTAs)
        s.window = flow_window(window);
        s.global_arena = true;
        *out = s;
        return true;
    }
    s.window = flow_window(window);
    // gap tables in shared memory when that still leaves an arena of 8192
    // entries, else read through L1
    s.smem_tables = arena_for(fixed + tabs) >= 8192u;
    s.arena = arena_for(fixed + (s.smem_tables ? tabs : 0));
    const int aforce = env_int_flow("TMCS_FLOW_ARENA", 0);  // tuning/testing knob: arena entries
    if (aforce >= int(kFlowMinArena) && !(aforce & (aforce - 1)) && uint32_t(aforce) < s.arena)
        s.arena = uint32_t(aforce);
    if (s.arena < kFlowMinArena) return false;
    s.smem = fixed + (s.smem_tables ? tabs : 0) + size_t(s.arena) * 4;
    if (s.smem > budget) return false;
    *out = s;
    return true;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if unavailable
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor map of the call's detector words for the tensor-store flush: a
// [n_det][ld] uint64 tensor, boxes of K chunk words x rows detectors. Needs
// K >= 2 (16-byte box rows), a 16-byte aligned buffer, an even row stride
// and coordinates below 2^31; returns false otherwise.
static bool encode_det_map(CUtensorMap *map, uint64_t *det, uint64_t n_det, uint64_t ld, int K, uint32_t rows) {
    if (K < 2 || !det || reinterpret_cast<uintptr_t>(det) % 16 || ld % 2 || ld >= (uint64_t(1) << 31) ||
        n_det == 0 || n_det >= (uint64_t(1) << 31) || rows == 0 || rows > 256)
        return false;
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dim[2] = {ld, n_det};
    const cuuint64_t stride[1] = {ld * 8};
    const cuuint32_t box[2] = {cuuint32_t(K), rows};
    const cuuint32_t estride[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, det, dim, stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int K, int W, bool GA>
static cudaError_t flow_go(const FlowArgs &a, const FlowShape &s, int sms, cudaStream_t st) {
    auto kern = flow_kernel<K, W, GA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.threads, s.smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(a.n_tiles, uint64_t(sms) * uint64_t(per_sm)));
    // a global arena holds one slice per CTA
    if (GA) grid = std::min<uint64_t>(grid, s.garena_ctas);
    // streams and steps are counted per CTA in 32 bits (flow_launch slices
    // calls so that this holds)
    const uint64_t tiles_per_cta = (a.n_tiles + grid - 1) / grid;
    if (tiles_per_cta * uint64_t(a.n_steps) >= (uint64_t(1) << 31) ||
        tiles_per_cta * (uint64_t(a.n_items) * uint64_t(K)) >= (uint64_t(1) << 31))
        return cudaErrorInvalidValue;
    kern<<<unsigned(grid), s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

template <int W, bool GA>
static cudaError_t flow_go_kg(const FlowArgs &a, const FlowShape &s, int sms, cudaStream_t st) {
    switch (s.K) {
    case 16: return flow_go<16, W, GA>(a, s, sms, st);
    case 8: return flow_go<8, W, GA>(a, s, sms, st);
    case 4: return flow_go<4, W, GA>(a, s, sms, st);
    case 2: return flow_go<2, W, GA>(a, s, sms, st);
    default: return flow_go<1, W, GA>(a, s, sms, st);
    }
}

template <int W>
static cudaError_t flow_go_k(const FlowArgs &a, const FlowShape &s, int sms, cudaStream_t st) {
    return a.garena ? flow_go_kg<W, true>(a, s, sms, st) : flow_go_kg<W, false>(a, s, sms, st);
}

cudaError_t flow_launch(const SigProgram &G, uint32_t n_obs, const DeviceSig *ds, const FlowShape &s,
                        const FlowCall &call, int sms, cudaStream_t st) {
    if (!ds || s.sched < 0 || size_t(s.sched) >= G.sched.size() || !ds->step_events[s.sched])
        return cudaErrorInvalidValue;
    const SigSchedule &S = G.sched[s.sched];
    FlowArgs a{};
    a.noise = ds->noise;
    a.tables = ds->tables;
    a.item_desc = reinterpret_cast<const uint4 *>(ds->item_desc[s.sched]);
    a.steps = reinterpret_cast<const uint4 *>(ds->steps[s.sched]);
    a.step_events = ds->step_events[s.sched];
    a.ev_ent = ds->ev_ent;
    a.n_steps = uint32_t(S.steps.size());
    a.n_items = uint32_t(S.items.size() / 2);
    a.window_mask = S.window - 1u;
    a.n_obs = n_obs;
    a.arena = s.arena;
    a.test_cap = uint32_t(std::max(0, env_int_flow("TMCS_TEST_FLOW_CAP", 0)));
    a.smem_tables = s.smem_tables ? uint32_t(G.tables.size() / kTableWords) : 0u;
    a.walkers = uint32_t(s.threads / 32 - s.appliers);
    a.key0 = call.key0;
    a.key1 = call.key1;
    a.ld = call.n_cols;
    // tensor-store flush: by default for tiles of 8 or more chunks (rows of
    // 64 bytes or more; narrower boxes measured slower than plain stores);
    // TMCS_FLOW_TMA=1 for any even tile, 0 never; TMCS_FLOW_TMA_ROWS sets
    // the rows per box (default 64, rounded up to whole 128-byte stretches
    // of the ring)
    const uint32_t al = s.K >= 16 ? 1u : 16u / uint32_t(std::max(s.K, 1));
    const uint32_t trows = (uint32_t(std::max(env_int_flow("TMCS_FLOW_TMA_ROWS", 64), 1)) + al - 1) / al * al;
    const int tma = env_int_flow("TMCS_FLOW_TMA", -1);
    if ((tma > 0 || (tma < 0 && s.K >= 8)) && encode_det_map(&a.tmap, call.det, G.n_det, call.n_cols, s.K, trows))
        a.tma_rows = trows;
    if (s.garena_ctas) {
        if (!call.scratch || call.scratch_bytes < size_t(s.garena_ctas) * s.arena * 4) return cudaErrorInvalidValue;
        a.garena = call.scratch;
    }
    // A CTA counts its streams and its steps in 32 bits: a call with more
    // tiles per CTA than that allows runs as several launches over column
    // slices (each a multiple of the tile size, in column order).
    const uint64_t per_tile_streams = uint64_t(a.n_items) * uint64_t(s.K);
    const uint64_t per_tile_steps = a.n_steps;
    const uint64_t lim = (uint64_t(1) << 31) - 1;
    const uint64_t max_tiles_per_cta =
        std::max<uint64_t>(1, std::min(lim / std::max<uint64_t>(per_tile_streams, 1), lim / per_tile_steps) - 1);
    uint64_t slice_cols = max_tiles_per_cta * uint64_t(sms) * uint64_t(s.K);
    // testing knob: slices of this many tiles (so the sliced path runs at
    // sizes the tests can check)
    const int tslice = env_int_flow("TMCS_TEST_FLOW_SLICE_TILES", 0);
    if (tslice > 0) slice_cols = std::min<uint64_t>(slice_cols, uint64_t(tslice) * uint64_t(s.K));
    for (uint64_t c0 = 0; c0 < call.n_cols; c0 += slice_cols) {
        const uint64_t n = std::min(slice_cols, call.n_cols - c0);
        a.first_chunk = call.first_chunk + uint32_t(c0);
        a.n_cols = n;
        a.last_mask = c0 + n == call.n_cols ? call.last_mask : ~uint64_t(0);
        a.n_tiles = (n + uint64_t(s.K) - 1) / uint64_t(s.K);
        a.det = call.det + c0;
        a.col_base = c0;
        a.obs = call.obs ? call.obs + c0 : nullptr;
        a.vec_out = (reinterpret_cast<uintptr_t>(a.det) % 16 == 0 && a.ld % 2 == 0) ? 1u : 0u;
        a.status = call.status;
        cudaError_t e;
        switch (s.window) {
        case 2: e = flow_go_k<2>(a, s, sms, st); break;
        case 4: e = flow_go_k<4>(a, s, sms, st); break;
        default: e = flow_go_k<3>(a, s, sms, st); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tmcs
