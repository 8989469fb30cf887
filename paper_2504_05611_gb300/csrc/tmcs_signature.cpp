// Event-signature program: per-generator output lists by a transposed frame
// pass, and the step schedule of the signature sampler.
//
// Why it is exact: with the noiseless reference fixed, each detector and
// observable flip is a parity of record flips, and every record flip is a
// GF(2)-linear function of the Pauli events of the shot (frames only ever
// XOR; Methods "Simulation" noise channels are Pauli). So the flips of a shot
// are the XOR over its events of each event's signature, the output of the
// frame program with that one event injected -- the DEM columns of Methods
// "Decoding". A Pauli event is the product of its X/Z generators, so its
// signature is the XOR of theirs.
//
// Transposed pass: the frame maps (CX c->t: x_t ^= x_c, z_c ^= z_t; H swaps
// x and z; S: z ^= x; R/RX clear both; M/MX record x/z; XFEED/ZFEED XOR a
// record into x/z) are linear; running their transposes over the op list
// from the end, on bit masks of a group of 64 outputs, gives at each point
// the set of outputs an X (mask sx) or Z (mask sz) flip there would flip.
// The pass for a group starts at the last op holding one of its records and
// stops as soon as no mask and no pending record sensitivity is left.
#include <algorithm>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <system_error>
#include <thread>

#include "tmcs_internal.h"

namespace tmcs {

int table_for_p(std::vector<uint32_t> &tables, std::vector<double> &table_p, double p, uint32_t *out) {
    for (size_t i = 0; i < table_p.size(); i++)
        if (table_p[i] == p) {
            *out = uint32_t(i);
            return TMCS_OK;
        }
    const uint32_t id = uint32_t(table_p.size());
    table_p.push_back(p);
    tables.resize(tables.size() + kTableWords, 0u);
    uint32_t *tab = &tables[size_t(id) * kTableWords];
    int rc = gap_table(p, tab);
    if (rc) return rc;
    const float inv = p >= 1.0 ? 0.0f : float(1.0 / std::log2(1.0 - p));
    std::memcpy(tab + kGapLen, &inv, 4);
    *out = id;
    return TMCS_OK;
}

namespace {

bool noise_code(uint32_t code) {
    return code == TMCS_X_ERROR || code == TMCS_Z_ERROR || code == TMCS_DEPOLARIZE1 ||
           code == TMCS_DEPOLARIZE2 || code == TMCS_PAULI_CHANNEL_1;
}

uint32_t kind_of(uint32_t code) {
    return code == TMCS_X_ERROR ? N_XERR : code == TMCS_Z_ERROR ? N_ZERR : code == TMCS_DEPOLARIZE1 ? N_DEP1
           : code == TMCS_DEPOLARIZE2 ? N_DEP2 : N_PC1;
}

struct Edge {
    uint32_t gen;
    uint32_t out;
};

// State of one transposed pass (reused across the passes of one thread).
struct Pass {
    std::vector<uint64_t> sx, sz, rs;  // per qubit / per record sensitivity masks
    std::vector<uint32_t> rs_touched;
    int64_t nz = 0;                    // nonzero entries among sx, sz, rs

    void set(uint64_t &v, uint64_t nv) {
        nz += int64_t(nv != 0) - int64_t(v != 0);
        v = nv;
    }
};

}  // namespace

// Pauli indices of a segment that can flip an output: bit k - 1 is set when
// event (unit, Pauli index k) has a non-empty output list for some unit of
// the segment (slots slot0 .. slot0 + units * paulis - 1, unit-major). The
// decoupled kernel drops the other events of the segment's streams before
// they reach its arena: they flip nothing, so the result is unchanged.
static uint32_t live_paulis(const SigProgram &G, uint32_t slot0, uint32_t units, uint32_t paulis) {
    uint32_t m = 0;
    for (uint32_t u = 0; u < units; u++)
        for (uint32_t k = 0; k < paulis; k++)
            if (G.ev_ent[2 * (size_t(slot0) + size_t(u) * paulis + k)] != kEvNone) m |= 1u << k;
    return m;
}

// Checks every invariant the signature kernels rely on, after each build:
// the memory safety of each index they form from the program (event slots
// and overflow lists, observable and detector ids, gap tables, item
// records) and the schedules' rules (steps partition the items and the
// detectors; in a barrier schedule every item's detectors lie in its step's
// window above the flush point; in a pipelined one every run of `lag`
// consecutive steps, of this tile and the next, fits the ring). Returns an
// empty string or the first violation.
static std::string validate_signature_program(const SigProgram &G, uint64_t D, uint64_t O) {
    const size_t n_tables = G.tables.size() / kTableWords;
    if (G.ev_base.size() != G.noise.size()) return "event bases";
    uint64_t slots = 0;
    for (size_t di = 0; di < G.noise.size(); di++) {
        const NoiseDesc &nd = G.noise[di];
        if (nd.kind > N_PC1 || nd.table >= n_tables) return "noise descriptor";
        if (nd.n_seg != (nd.n_units + kSegUnits - 1) / kSegUnits) return "segment count";
        if (G.ev_base[di] != slots) return "event slots out of order";
        slots += uint64_t(nd.n_units) * sig_paulis(nd.kind);
    }
    if (G.ev_ent.size() < 2 * slots) return "event table too short";
    auto entry_ok = [&](uint32_t e) {
        const uint32_t idx = e & 0x1FFFFFFFu;
        return (e >> 30) == 0u && ((e & (1u << 29)) ? idx < O : idx < D);
    };
    for (size_t k = 0; k < slots; k++) {
        const uint32_t w0 = G.ev_ent[2 * k], w1 = G.ev_ent[2 * k + 1];
        if (w0 == kEvNone) {
            if (w1 != kEvNone) return "event slot";
        } else if (w0 & kEvOverflow) {
            const uint64_t off = w0 & ~kEvOverflow;
            if (off < 2 * slots || w1 < 3 || off + w1 > G.ev_ent.size()) return "overflow list";
            for (uint32_t x = 0; x < w1; x++)
                if (!entry_ok(G.ev_ent[off + x])) return "overflow entry";
        } else if (!entry_ok(w0) || (w1 != kEvNone && !entry_ok(w1))) {
            return "event entry";
        }
    }
    // detector span [lo, hi) of every segment (first segment of descriptor
    // di at seg0[di]): the union of its single-generator events' lists, i.e.
    // of all its events' entries
    std::vector<uint64_t> seg0(G.noise.size() + 1, 0);
    for (size_t di = 0; di < G.noise.size(); di++) seg0[di + 1] = seg0[di] + G.noise[di].n_seg;
    std::vector<uint64_t> seg_lo(seg0.back(), UINT64_MAX), seg_hi(seg0.back(), 0);
    for (size_t di = 0; di < G.noise.size(); di++) {
        const NoiseDesc &nd = G.noise[di];
        const uint32_t KP = sig_paulis(nd.kind);
        for (uint64_t k = G.ev_base[di]; k < G.ev_base[di] + uint64_t(nd.n_units) * KP; k++) {
            const uint64_t sg = seg0[di] + (k - G.ev_base[di]) / KP / kSegUnits;
            auto see = [&](uint32_t e) {
                if (e & (1u << 29)) return;
                seg_lo[sg] = std::min<uint64_t>(seg_lo[sg], e & 0x1FFFFFFFu);
                seg_hi[sg] = std::max<uint64_t>(seg_hi[sg], uint64_t(e & 0x1FFFFFFFu) + 1);
            };
            const uint32_t w0 = G.ev_ent[2 * k], w1 = G.ev_ent[2 * k + 1];
            if (w0 == kEvNone) continue;
            if (w0 & kEvOverflow) {
                for (uint32_t x = 0; x < w1; x++) see(G.ev_ent[(w0 & ~kEvOverflow) + x]);
            } else {
                see(w0);
                if (w1 != kEvNone) see(w1);
            }
        }
    }
    for (const SigSchedule &S : G.sched) {
        const size_t n_items = S.items.size() / 2;
        const uint32_t W = S.window;
        if (W < 256 || (W & (W - 1)) || S.lag > uint32_t(kSigMaxLag) || (S.lag && W > 16384)) return "schedule shape";
        if (S.item_rec.size() != 4 * n_items || S.steps.empty()) return "schedule size";
        if (S.step_events.size() != S.steps.size()) return "step event counts";
        if (S.item_desc.size() != 8 * n_items || S.steps.size() > (1u << 15)) return "walker descriptors size";
        std::vector<uint64_t> lo(n_items), hi(n_items);
        for (size_t k = 0; k < n_items; k++) {
            const uint32_t di = S.items[2 * k], sg = S.items[2 * k + 1];
            if (di >= G.noise.size() || sg >= G.noise[di].n_seg) return "item";
            const NoiseDesc &nd = G.noise[di];
            const uint32_t units = std::min(kSegUnits, nd.n_units - sg * kSegUnits);
            const uint32_t *r = &S.item_rec[4 * k];
            if (r[0] != nd.op_index || r[1] != sg || r[2] != G.ev_base[di] + sg * kSegUnits * sig_paulis(nd.kind) ||
                r[3] != (nd.kind | (nd.table << 3) | ((units - 1) << 16) | (di << 22)))
                return "item record";
            // walker descriptor: the indices the decoupled kernel forms from it
            const uint32_t *wd = &S.item_desc[8 * k];
            const uint64_t m = uint64_t(0xCD9E8D57u) * nd.op_index;
            const uint32_t step = wd[4] >> 17;
            if (wd[0] != uint32_t(m >> 32) || wd[1] != uint32_t(m) || wd[2] != sg || wd[3] != r[2] ||
                (wd[4] & 7u) != nd.kind || ((wd[4] >> 3) & 15u) != (nd.kind == 3u ? 15u : nd.kind == 2u ? 3u : 1u) ||
                ((wd[4] >> 7) & 15u) != sig_paulis(nd.kind) || ((wd[4] >> 11) & 63u) != units - 1 ||
                step >= S.steps.size() || k < S.steps[step].item_begin || k >= S.steps[step].item_end ||
                (wd[5] & 0x1FFFu) != nd.table || (wd[5] >> 13) != di ||
                wd[6] != G.tables[size_t(nd.table) * kTableWords + kGapLen] ||
                wd[7] != live_paulis(G, r[2], units, sig_paulis(nd.kind)))
                return "walker descriptor";
            lo[k] = seg_lo[seg0[di] + sg];
            hi[k] = seg_hi[seg0[di] + sg];
        }
        const size_t ns = S.steps.size();
        std::vector<uint64_t> shi(ns);
        for (size_t t = 0; t < ns; t++) {
            const SigStep &st = S.steps[t];
            const uint32_t b0 = t ? S.steps[t - 1].item_end : 0u, f0 = t ? S.steps[t - 1].flush_hi : 0u;
            if (st.item_begin != b0 || st.item_end < st.item_begin || st.flush_lo != f0 || st.flush_hi < st.flush_lo)
                return "steps not contiguous";
            shi[t] = st.flush_hi;
            for (uint32_t k = st.item_begin; k < st.item_end; k++) {
                if (lo[k] == UINT64_MAX) continue;
                if (lo[k] < st.flush_lo) return "item below its step's flush point";
                if (!S.lag && hi[k] > uint64_t(st.flush_lo) + W) return "item beyond its step's window";
                shi[t] = std::max(shi[t], hi[k]);
            }
        }
        if (S.steps.back().item_end != n_items || S.steps.back().flush_hi != D) return "steps do not cover";
        if (S.lag)
            for (size_t v = 0; v < 2 * ns; v++) {
                const size_t v0 = v + 1 >= S.lag ? v + 1 - S.lag : 0;
                uint64_t h = 0;
                for (size_t u = v0; u <= v; u++) h = std::max<uint64_t>(h, shi[u % ns] + (u / ns) * D);
                if (h - (S.steps[v0 % ns].flush_lo + (v0 / ns) * D) > W) return "ring too small for its lag";
            }
    }
    return std::string();
}

int build_signature_program(tmcs_circuit *c, uint32_t max_window) {
    const auto t_start = std::chrono::steady_clock::now();
    SigProgram &G = c->sig;
    G = SigProgram();
    const size_t n_ops = c->ops.size();
    const uint64_t Q = c->n_qubits, M = c->n_meas, D = c->n_det, O = c->n_obs;
    if (D >= kSigObsFlag || O > 4096) {
        G.why = "too many outputs";
        return TMCS_OK;
    }
    G.n_det = uint32_t(D);

    // ---- noise descriptors and generator ids (every noise op with p > 0)
    std::vector<uint32_t> op_desc(n_ops, 0xFFFFFFFFu);
    std::vector<double> table_p;
    uint64_t n_gens = 0;
    for (size_t i = 0; i < n_ops; i++) {
        const HostOp &op = c->ops[i];
        if (!noise_code(op.code) || !(op.p > 0.0) || op.nt == 0) continue;
        NoiseDesc nd{};
        nd.op_index = uint32_t(i);
        nd.kind = kind_of(op.code);
        if (nd.kind == N_PC1) {
            nd.t1 = op.arg;
            nd.t2 = op.arg2;
        }
        int rc = table_for_p(G.tables, table_p, op.p, &nd.table);
        if (rc) return rc;
        nd.n_units = nd.kind == N_DEP2 ? op.nt / 2 : op.nt;
        nd.n_seg = (nd.n_units + kSegUnits - 1) / kSegUnits;
        if (n_gens + uint64_t(nd.n_units) * sig_gens(nd.kind) >= 0xFFFFFFFFull) {
            G.why = "too many noise generators";
            return TMCS_OK;
        }
        nd.tgt_off = uint32_t(n_gens);
        n_gens += uint64_t(nd.n_units) * sig_gens(nd.kind);
        op_desc[i] = uint32_t(G.noise.size());
        G.noise.push_back(nd);
    }

    // ---- records: producing op, first record of each measuring op
    std::vector<uint32_t> rec_op(M), rec_base(n_ops, 0);
    {
        uint64_t m = 0;
        for (size_t i = 0; i < n_ops; i++) {
            const HostOp &op = c->ops[i];
            rec_base[i] = uint32_t(m);
            if (op.code == TMCS_M || op.code == TMCS_MX)
                for (uint32_t a = 0; a < op.nt; a++) rec_op[m++] = uint32_t(i);
        }
    }
    // output record lists: detectors 0..D-1, then observables D..D+O-1
    std::vector<uint32_t> out_off(D + O + 1, 0), out_rec;
    {
        std::vector<std::vector<uint32_t>> obs_recs(O);
        uint64_t d = 0;
        for (size_t i = 0; i < n_ops; i++) {
            const HostOp &op = c->ops[i];
            const uint32_t *t = c->targets.data() + op.toff;
            if (op.code == TMCS_DETECTOR) {
                out_rec.insert(out_rec.end(), t, t + op.nt);
                out_off[++d] = uint32_t(out_rec.size());
            } else if (op.code == TMCS_OBSERVABLE) {
                obs_recs[op.arg].insert(obs_recs[op.arg].end(), t, t + op.nt);
            }
        }
        for (uint64_t o = 0; o < O; o++) {
            out_rec.insert(out_rec.end(), obs_recs[o].begin(), obs_recs[o].end());
            out_off[D + o + 1] = uint32_t(out_rec.size());
        }
    }

    // ---- transposed passes, one per group of 64 outputs (detector groups
    // never mix with observables)
    const uint64_t n_gd = (D + 63) / 64, n_go = (O + 63) / 64, n_groups = n_gd + n_go;
    std::vector<std::vector<Edge>> edges(n_groups);
    auto run_group = [&](uint64_t g, Pass &S) {
        const bool obs = g >= n_gd;
        const uint64_t b = obs ? D + 64 * (g - n_gd) : 64 * g;
        const uint64_t e = obs ? std::min<uint64_t>(D + O, b + 64) : std::min<uint64_t>(D, b + 64);
        const uint32_t tag = obs ? kSigObsFlag : 0u;
        const uint64_t base_out = obs ? b - D : b;
        int64_t start = -1;
        for (uint64_t j = b; j < e; j++)
            for (uint32_t k = out_off[j]; k < out_off[j + 1]; k++) {
                const uint32_t r = out_rec[k];
                S.set(S.rs[r], S.rs[r] ^ (1ull << (j - b)));
                S.rs_touched.push_back(r);
                start = std::max<int64_t>(start, rec_op[r]);
            }
        std::vector<Edge> &E = edges[g];
        for (int64_t i = start; i >= 0 && S.nz > 0; i--) {
            const HostOp &op = c->ops[size_t(i)];
            const uint32_t *t = c->targets.data() + op.toff;
            switch (op.code) {
            case TMCS_M:
            case TMCS_MX: {
                const bool zb = op.code == TMCS_MX;
                for (uint32_t a = op.nt; a-- > 0;) {
                    const uint32_t r = rec_base[size_t(i)] + a;
                    const uint64_t v = S.rs[r];
                    if (!v) continue;
                    uint64_t &f = zb ? S.sz[t[a]] : S.sx[t[a]];
                    S.set(f, f ^ v);
                    S.set(S.rs[r], 0);
                }
                break;
            }
            case TMCS_R:
            case TMCS_RX:
                for (uint32_t a = op.nt; a-- > 0;) {
                    S.set(S.sx[t[a]], 0);
                    S.set(S.sz[t[a]], 0);
                }
                break;
            case TMCS_H:
                for (uint32_t a = op.nt; a-- > 0;) std::swap(S.sx[t[a]], S.sz[t[a]]);
                break;
            case TMCS_S:
                for (uint32_t a = op.nt; a-- > 0;) S.set(S.sx[t[a]], S.sx[t[a]] ^ S.sz[t[a]]);
                break;
            case TMCS_CX:
                for (uint32_t a = op.nt; a >= 2; a -= 2) {
                    const uint32_t cq = t[a - 2], tq = t[a - 1];
                    S.set(S.sx[cq], S.sx[cq] ^ S.sx[tq]);
                    S.set(S.sz[tq], S.sz[tq] ^ S.sz[cq]);
                }
                break;
            case TMCS_XFEED:
            case TMCS_ZFEED: {
                const bool zb = op.code == TMCS_ZFEED;
                for (uint32_t a = op.nt; a >= 2; a -= 2) {
                    const uint32_t r = t[a - 2], q = t[a - 1];
                    const uint64_t v = zb ? S.sz[q] : S.sx[q];
                    if (!v) continue;
                    S.set(S.rs[r], S.rs[r] ^ v);
                    S.rs_touched.push_back(r);
                }
                break;
            }
            default:
                if (op_desc[size_t(i)] != 0xFFFFFFFFu) {
                    const NoiseDesc &nd = G.noise[op_desc[size_t(i)]];
                    const uint32_t ng = sig_gens(nd.kind);
                    for (uint32_t u = 0; u < nd.n_units; u++)
                        for (uint32_t gg = 0; gg < ng; gg++) {
                            const uint32_t q = nd.kind == N_DEP2 ? t[2 * u + gg / 2] : t[u];
                            uint64_t m = (gg & 1u) ? S.sz[q] : S.sx[q];
                            while (m) {
                                const int bit = __builtin_ctzll(m);
                                m &= m - 1;
                                E.push_back({nd.tgt_off + u * ng + gg, uint32_t(base_out + uint64_t(bit)) | tag});
                            }
                        }
                }
                break;
            }
        }
        if (S.nz != 0) {
            std::fill(S.sx.begin(), S.sx.end(), 0);
            std::fill(S.sz.begin(), S.sz.end(), 0);
        }
        for (uint32_t r : S.rs_touched) S.rs[r] = 0;
        S.rs_touched.clear();
        S.nz = 0;
    };
    unsigned n_thr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n_groups < 4 * n_thr) n_thr = 1;
    std::vector<std::thread> pool;
    auto worker = [&](unsigned w) {
        Pass S;
        S.sx.assign(Q, 0);
        S.sz.assign(Q, 0);
        S.rs.assign(M, 0);
        for (uint64_t g = w; g < n_groups; g += n_thr) run_group(g, S);
    };
    try {
        if (n_thr == 1) {
            worker(0);
        } else {
            for (unsigned w = 0; w < n_thr; w++) pool.emplace_back(worker, w);
            for (auto &th : pool) th.join();
        }
    } catch (const std::system_error &) {
        for (auto &th : pool)
            if (th.joinable()) th.join();
        pool.clear();
        worker(0);
    }

    // ---- CSR by generator (group order within a generator)
    G.gen_off.assign(n_gens + 1, 0);
    uint64_t n_ent = 0;
    for (const auto &E : edges)
        for (const Edge &x : E) G.gen_off[x.gen + 1]++;
    for (uint64_t g = 0; g < n_gens; g++) G.gen_off[g + 1] += G.gen_off[g];
    n_ent = G.gen_off[n_gens];
    if (n_ent >= 0xFFFFFFFFull) {
        G.why = "too many signature entries";
        return TMCS_OK;
    }
    G.gen_ent.assign(n_ent, 0);
    {
        std::vector<uint32_t> fill(G.gen_off.begin(), G.gen_off.end() - 1);
        for (const auto &E : edges)
            for (const Edge &x : E) G.gen_ent[fill[x.gen]++] = x.out;
    }
    edges.clear();

    // ---- device layout: one 8-byte slot per (unit, Pauli index) in fault
    // order (descriptor, unit, Pauli index - 1), holding the output list of
    // that event: the symmetric difference of its generators' lists. Word 0
    // = the first entry, kEvNone (no outputs) or kEvOverflow | offset (the
    // list lies in the overflow area after the slots and word 1 is its
    // length); word 1 = the second entry or kEvNone. An entry is observable
    // flag << 29 | output index. Most events flip at most two outputs, so an
    // event is one aligned 8-byte load.
    {
        if (D >= (1u << 29) || O >= (1u << 29)) {
            G.why = "too many outputs for the device layout";
            return TMCS_OK;
        }
        uint64_t slots = 0;
        for (const NoiseDesc &nd : G.noise) {
            G.ev_base.push_back(uint32_t(slots));
            slots += uint64_t(nd.n_units) * sig_paulis(nd.kind);
            if (slots >= (uint64_t(1) << 31)) {
                G.why = "too many noise events for the device layout";
                return TMCS_OK;
            }
        }
        G.n_event_slots = uint32_t(slots);
        G.ev_ent.assign(2 * slots, kEvNone);
        std::vector<uint32_t> v;
        for (uint32_t di = 0; di < G.noise.size(); di++) {
            const NoiseDesc &nd = G.noise[di];
            const uint32_t ng = sig_gens(nd.kind), KP = sig_paulis(nd.kind);
            for (uint32_t u = 0; u < nd.n_units; u++) {
                const uint32_t g0 = nd.tgt_off + u * ng;
                if (G.gen_off[g0] == G.gen_off[g0 + ng]) continue;  // every event of the unit flips nothing
                for (uint32_t pk = 1; pk <= KP; pk++) {
                    const uint32_t mask = sig_mask(nd.kind, pk);
                    v.clear();
                    for (uint32_t g = 0; g < ng; g++)
                        if (mask >> g & 1u)
                            for (uint32_t k = G.gen_off[g0 + g]; k < G.gen_off[g0 + g + 1]; k++) {
                                const uint32_t e = G.gen_ent[k];
                                v.push_back((e & kSigObsFlag) ? ((1u << 29) | (e & ~kSigObsFlag)) : e);
                            }
                    std::sort(v.begin(), v.end());
                    size_t n = 0;  // XOR: keep entries that occur an odd number of times
                    for (size_t i = 0; i < v.size();) {
                        size_t j = i;
                        while (j < v.size() && v[j] == v[i]) j++;
                        if ((j - i) & 1) v[n++] = v[i];
                        i = j;
                    }
                    const size_t slot = 2 * (size_t(G.ev_base[di]) + size_t(u) * KP + (pk - 1));
                    if (n <= 2) {
                        for (size_t i = 0; i < n; i++) G.ev_ent[slot + i] = v[i];
                    } else {
                        const size_t off = G.ev_ent.size();
                        if (off + n >= size_t(kEvNone & ~kEvOverflow)) {
                            G.why = "too many signature entries";
                            return TMCS_OK;
                        }
                        G.ev_ent[slot] = kEvOverflow | uint32_t(off);
                        G.ev_ent[slot + 1] = uint32_t(n);
                        G.ev_ent.insert(G.ev_ent.end(), v.begin(), v.begin() + n);
                    }
                }
            }
        }
        while (G.ev_ent.size() % 4) G.ev_ent.push_back(kEvNone);
    }

    // ---- items: segments whose events flip anything; detector span per item
    std::vector<uint32_t> items, dmin, dmax;
    for (uint32_t di = 0; di < G.noise.size(); di++) {
        const NoiseDesc &nd = G.noise[di];
        const uint32_t ng = sig_gens(nd.kind);
        for (uint32_t s = 0; s < nd.n_seg; s++) {
            const uint32_t u0 = s * kSegUnits, u1 = std::min(nd.n_units, u0 + kSegUnits);
            const uint32_t g0 = nd.tgt_off + u0 * ng, g1 = nd.tgt_off + u1 * ng;
            if (G.gen_off[g0] == G.gen_off[g1]) continue;
            uint32_t lo = 0xFFFFFFFFu, hi = 0;
            bool any_det = false;
            for (uint32_t k = G.gen_off[g0]; k < G.gen_off[g1]; k++) {
                const uint32_t v = G.gen_ent[k];
                if (v & kSigObsFlag) continue;
                lo = std::min(lo, v);
                hi = std::max(hi, v);
                any_det = true;
            }
            items.push_back(di);
            items.push_back(s);
            dmin.push_back(any_det ? lo : 0xFFFFFFFFu);
            dmax.push_back(any_det ? hi : 0u);
        }
    }
    const size_t n_items = dmin.size();
    // Items in order of their highest detector: the items that fit a step's
    // window above its flush point are then always a prefix of the items
    // left, so the greedy cut below takes every item that fits (events XOR
    // into the ring, so the order of items does not change the output).
    {
        std::vector<uint32_t> ord(n_items);
        for (size_t k = 0; k < n_items; k++) ord[k] = uint32_t(k);
        std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
            const uint64_t ax = dmin[x] == 0xFFFFFFFFu ? 0 : uint64_t(dmax[x]) + 1;
            const uint64_t ay = dmin[y] == 0xFFFFFFFFu ? 0 : uint64_t(dmax[y]) + 1;
            return ax < ay;
        });
        std::vector<uint32_t> it2(2 * n_items), dmin2(n_items), dmax2(n_items);
        for (size_t k = 0; k < n_items; k++) {
            it2[2 * k] = items[2 * ord[k]];
            it2[2 * k + 1] = items[2 * ord[k] + 1];
            dmin2[k] = dmin[ord[k]];
            dmax2[k] = dmax[ord[k]];
        }
        items.swap(it2);
        dmin.swap(dmin2);
        dmax.swap(dmax2);
    }
    std::vector<uint64_t> sufmin(n_items + 1, D);
    for (size_t i = n_items; i-- > 0;) sufmin[i] = std::min<uint64_t>(sufmin[i + 1], dmin[i]);
    if (G.noise.size() > 1024 || G.tables.size() / kTableWords > 8192) {
        G.why = "too many noise ops or distinct probabilities for the device item records";
        return TMCS_OK;
    }

    // ---- schedules. The smallest feasible window is the smallest power of
    // two >= 1024 that holds every item's detector span above its flush
    // point; the main schedule raises it to max_window (fewer, larger steps,
    // capped by D), and up to two more schedules halve it while feasible
    // (a smaller ring lets more chunks or CTAs share an SM; the autotuner
    // picks).
    uint64_t need = 0;
    for (size_t i = 0; i < n_items; i++)
        if (dmin[i] != 0xFFFFFFFFu) need = std::max<uint64_t>(need, uint64_t(dmax[i]) - sufmin[i] + 1);
    uint64_t Wmin = 1024;
    while (Wmin < need) Wmin <<= 1;
    uint64_t Dp = 1024;
    while (Dp < D) Dp <<= 1;
    const uint64_t W0 = std::max<uint64_t>(Wmin, std::min<uint64_t>(max_window, Dp));
    if (W0 > max_window) {
        G.why = "detector window " + std::to_string(need) + " exceeds " + std::to_string(max_window);
        return TMCS_OK;
    }
    auto build_schedule = [&](uint64_t W, SigSchedule &S) {
        S = SigSchedule();
        S.window = uint32_t(W);
        S.items = items;
        uint64_t F = 0;
        size_t i = 0;
        while (i < n_items) {
            size_t j = i;
            while (j < n_items && (dmin[j] == 0xFFFFFFFFu || dmax[j] < F + W)) j++;
            if (j == i) return false;  // cannot happen: W >= need and F <= sufmin[i]
            const uint64_t F2 = sufmin[j];
            S.steps.push_back({uint32_t(i), uint32_t(j), uint32_t(F), uint32_t(F2)});
            F = F2;
            i = j;
        }
        if (S.steps.empty() || F < D) S.steps.push_back({uint32_t(n_items), uint32_t(n_items), uint32_t(F), uint32_t(D)});
        // within a step, longest streams first (expected draws ~ p x units),
        // so the step's tail is short; order within a step does not change
        // the output (events XOR into the ring)
        std::vector<uint32_t> perm(n_items);
        for (size_t k = 0; k < n_items; k++) perm[k] = uint32_t(k);
        auto cost = [&](uint32_t k) {
            const NoiseDesc &nd = G.noise[items[2 * k]];
            const uint32_t units = std::min(kSegUnits, nd.n_units - items[2 * k + 1] * kSegUnits);
            return table_p[nd.table] * double(units);
        };
        for (const SigStep &st : S.steps)
            std::stable_sort(perm.begin() + st.item_begin, perm.begin() + st.item_end,
                             [&](uint32_t x, uint32_t y) { return cost(x) > cost(y); });
        for (size_t k = 0; k < n_items; k++) {
            S.items[2 * k] = items[2 * perm[k]];
            S.items[2 * k + 1] = items[2 * perm[k] + 1];
        }
        // expected events per chunk of each step: 64 trials per unit at the
        // op's probability (the decoupled kernel sizes its event regions)
        for (const SigStep &st : S.steps) {
            double ev = 0;
            for (uint32_t k = st.item_begin; k < st.item_end; k++) ev += 64.0 * cost(perm[k]);
            S.step_events.push_back(float(ev));
        }
        // walker descriptors of the decoupled kernel (see SigSchedule)
        for (uint32_t t = 0; t < S.steps.size(); t++)
            for (uint32_t k = S.steps[t].item_begin; k < S.steps[t].item_end; k++) {
                const uint32_t di = S.items[2 * k], sg = S.items[2 * k + 1];
                const NoiseDesc &nd = G.noise[di];
                const uint32_t units = std::min(kSegUnits, nd.n_units - sg * kSegUnits);
                const uint64_t m = uint64_t(0xCD9E8D57u) * nd.op_index;
                const uint32_t npauli = nd.kind == 3u ? 15u : nd.kind == 2u ? 3u : 1u;
                uint32_t inv_bits = G.tables[size_t(nd.table) * kTableWords + kGapLen];
                const uint32_t slot0 = G.ev_base[di] + sg * kSegUnits * sig_paulis(nd.kind);
                const uint32_t w[8] = {uint32_t(m >> 32), uint32_t(m), sg, slot0,
                                       nd.kind | (npauli << 3) | (sig_paulis(nd.kind) << 7) | ((units - 1) << 11) |
                                           (t << 17),
                                       nd.table | (di << 13), inv_bits,
                                       live_paulis(G, slot0, units, sig_paulis(nd.kind))};
                S.item_desc.insert(S.item_desc.end(), w, w + 8);
            }
        // device item records (the walk reads one 16-byte record per stream)
        for (size_t k = 0; k < n_items; k++) {
            const uint32_t di = S.items[2 * k], sg = S.items[2 * k + 1];
            const NoiseDesc &nd = G.noise[di];
            const uint32_t units = std::min(kSegUnits, nd.n_units - sg * kSegUnits);
            S.item_rec.push_back(nd.op_index);
            S.item_rec.push_back(sg);
            S.item_rec.push_back(G.ev_base[di] + sg * kSegUnits * sig_paulis(nd.kind));
            S.item_rec.push_back(nd.kind | (nd.table << 3) | ((units - 1) << 16) | (di << 22));
        }
        return true;
    };
    for (uint64_t W = W0; W >= Wmin && G.sched.size() < 3; W >>= 1) {
        G.sched.emplace_back();
        if (!build_schedule(W, G.sched.back())) {
            G.why = "internal: schedule";
            G.sched.clear();
            return TMCS_OK;
        }
        if (W == 1024) break;
    }

    // ---- pipelined schedules: steps of window Ws, up to L of them in
    // flight. The ring must hold, for every run of L consecutive steps (the
    // next tile's steps follow this tile's, D detectors further on), every
    // detector from the first step's flush point up to the highest detector
    // any of the L steps touches or flushes.
    auto ring_for = [&](const SigSchedule &S, uint32_t L) {
        const size_t ns = S.steps.size();
        std::vector<uint64_t> hi(ns);
        for (size_t t = 0; t < ns; t++) {
            hi[t] = S.steps[t].flush_hi;
            for (uint32_t i = S.steps[t].item_begin; i < S.steps[t].item_end; i++)
                if (dmin[i] != 0xFFFFFFFFu) hi[t] = std::max<uint64_t>(hi[t], uint64_t(dmax[i]) + 1);
        }
        uint64_t span = 0;
        for (size_t v = 0; v < 2 * ns; v++) {
            const size_t v0 = v + 1 >= L ? v + 1 - L : 0;
            uint64_t h = 0;
            for (size_t u = v0; u <= v; u++) h = std::max<uint64_t>(h, hi[u % ns] + (u / ns) * D);
            span = std::max<uint64_t>(span, h - (S.steps[v0 % ns].flush_lo + (v0 / ns) * D));
        }
        uint64_t R = 256;
        while (R < span) R <<= 1;
        return R;
    };
    uint64_t Wp = 256;
    while (Wp < need) Wp <<= 1;
    for (int w = 0; w < 2; w++, Wp <<= 1) {
        SigSchedule base;
        if (!build_schedule(Wp, base)) continue;
        for (uint32_t L = 2; L <= uint32_t(kSigMaxLag) && G.sched.size() < size_t(kSigMaxSchedules); L++) {
            if (L > base.steps.size() + 1) break;  // the two observable buffers need L <= steps + 1
            const uint64_t R = ring_for(base, L);
            if (R > 16384) break;
            G.sched.push_back(base);
            G.sched.back().window = uint32_t(R);
            G.sched.back().lag = L;
        }
    }
    // testing knob: plant one mistake before validation (the host-side
    // validator must then refuse the program; sampling uses the frame kernels)
    if (const char *v = std::getenv("TMCS_TEST_CORRUPT_SIG")) {
        const std::string what(v);
        if (what == "observable") {
            for (size_t k = 0; k + 1 < G.ev_ent.size(); k += 2)
                if (G.ev_ent[k] != kEvNone && !(G.ev_ent[k] & kEvOverflow)) {
                    G.ev_ent[k] = (1u << 29) | uint32_t(O);  // one past the last observable
                    break;
                }
        } else if (what == "record" && !G.sched.empty() && !G.sched[0].item_rec.empty()) {
            G.sched[0].item_rec[2] += 1;  // first item's event slot
        } else if (what == "window" && !G.sched.empty()) {
            G.sched[0].window = 256;  // steps cut for a larger ring
        } else if (what == "live" && !G.sched.empty()) {
            // drop a Pauli index that flips something from one item's mask
            std::vector<uint32_t> &wd = G.sched[0].item_desc;
            for (size_t k = 7; k < wd.size(); k += 8)
                if (wd[k]) {
                    wd[k] &= wd[k] - 1u;
                    break;
                }
        }
    }
    const std::string bad = validate_signature_program(G, D, O);
    if (!bad.empty()) {
        G.why = "internal: " + bad;
        G.sched.clear();
        return TMCS_OK;
    }
    G.ok = true;
    G.build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return TMCS_OK;
}

}  // namespace tmcs
