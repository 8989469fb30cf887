// Host side of libtmcs: op-list validation, the slot compiler, the gap
// tables of the sampling specification, the determinism audit and the
// reference-sample tableau. No CUDA calls in this file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "tmcs_internal.h"

namespace tmcs {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

static bool is_noise(uint32_t code) {
    return code == TMCS_X_ERROR || code == TMCS_Z_ERROR || code == TMCS_DEPOLARIZE1 ||
           code == TMCS_DEPOLARIZE2 || code == TMCS_PAULI_CHANNEL_1;
}

static bool is_pair(uint32_t code) {
    return code == TMCS_CX || code == TMCS_DEPOLARIZE2 || code == TMCS_XFEED || code == TMCS_ZFEED;
}

// ------------------------------------------------------------ gap table
//
// Sampling specification: the gap between consecutive noise events of a
// segment is G = #{g in 1..4096 : w < T[g]} for a uniform 32-bit word w, with
// T[g] = floor(2^32 (1-p)^g); P(G >= g) = T[g] / 2^32, so G is geometric with
// success probability p on every position a 4096-trial segment can reach.

static uint32_t frac_to_u32(double x) {
    double v = std::floor(std::ldexp(x, 32));
    if (!(v > 0.0)) return 0u;
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    return static_cast<uint32_t>(v);
}

int gap_table(double p, uint32_t *t) {
    if (!(p > 0.0 && p <= 1.0)) return fail(TMCS_E_INVALID, "gap table needs p in (0, 1]");
    const double lq = std::log1p(-p);
    for (uint32_t g = 1; g <= kGapLen; g++) t[g - 1] = frac_to_u32(std::exp(double(g) * lq));
    // The kernel locates the count by search, which equals it only for a
    // non-increasing table.
    for (uint32_t g = 1; g < kGapLen; g++)
        if (t[g] > t[g - 1]) return fail(TMCS_E_INVALID, "gap table not monotone (p too small)");
    return TMCS_OK;
}

size_t program_bytes(const Program &p) {
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    return al(p.layers.size() * sizeof(Layer)) + al(p.args.size() * 4) +
           al(p.noise.size() * sizeof(NoiseDesc)) + al(p.tables.size() * 4) + al(p.fault_base.size() * 8);
}

// -------------------------------------------------------------- compiler

namespace {

enum IRKind : uint8_t { I_ZERO, I_XOR, I_COPY, I_NOISE, I_DET, I_OBS, I_GAUGE, I_REC };

struct IRInst {
    uint8_t kind;
    uint32_t a, b;  // ZERO a | XOR a ^= b | COPY a = b | NOISE a = index | DET/OBS a = index
};

struct IRNoise {
    uint32_t op;
    uint32_t kind;
    double p;
    uint32_t t1 = 0, t2 = 0;
    std::vector<uint32_t> comp;  // (xv, zv) per target qubit
    std::vector<uint8_t> live;   // per comp entry
};

struct IRParity {
    uint32_t acc;  // accumulator vreg (OBS) or detector id (DET)
    std::vector<uint32_t> recs;
};

}  // namespace

// Checks every invariant the kernel relies on for memory safety: staged
// blocks 16-byte aligned and at most kStageWords words, every slot index
// below n_slots, list bounds inside their block, detector and observable ids
// in range, noise windows inside the event buffer. Runs after every compile.
static int validate_program(const Program &P, uint64_t n_det, uint64_t n_obs, uint64_t n_meas) {
    auto bad = [](const std::string &m) { return fail(TMCS_E_INVALID, "internal: program check failed: " + m); };
    if (P.args.size() % 4) return bad("args not padded");
    uint32_t staged = 0;
    for (size_t l = 0; l < P.layers.size(); l++) {
        const Layer &ly = P.layers[l];
        const std::string at = "layer " + std::to_string(l);
        if (ly.nwords && ly.seq != staged++) return bad(at + ": staged sequence number");
        if (ly.nwords) {
            if (ly.off % 4 || ly.nwords % 4 || ly.nwords > kStageWords || size_t(ly.off) + ly.nwords > P.args.size())
                return bad(at + ": staged block misaligned or out of range");
        }
        const uint32_t *b = P.args.data() + ly.off;
        switch (ly.kind) {
        case L_ZERO:
        case L_OBSOUT:
            if (!ly.nwords || ly.count > ly.nwords) return bad(at + ": block too small");
            for (uint32_t i = 0; i < ly.count; i++)
                if (b[i] >= P.n_slots) return bad(at + ": slot out of range");
            if (ly.kind == L_OBSOUT && ly.count > n_obs) return bad(at + ": observable out of range");
            break;
        case L_XOR:
        case L_COPY:
            if (!ly.nwords || ly.count > ly.nwords) return bad(at + ": block too small");
            for (uint32_t i = 0; i < ly.count; i++)
                if ((b[i] & 0xFFFFu) >= P.n_slots || (b[i] >> 16) >= P.n_slots) return bad(at + ": slot out of range");
            break;
        case L_DET:
        case L_OBS: {
            if (!ly.nwords || ly.count + 1 > ly.nwords) return bad(at + ": block too small");
            for (uint32_t d = 0; d < ly.count; d++) {
                const uint32_t lo = b[d], hi = b[d + 1];
                if (lo < ly.count + 1 || hi < lo || hi > ly.nwords) return bad(at + ": list bounds");
                if (ly.kind == L_OBS && hi == lo) return bad(at + ": observable list without accumulator");
                for (uint32_t t = lo; t < hi; t++)
                    if (b[t] >= P.n_slots) return bad(at + ": slot out of range");
            }
            if (ly.kind == L_DET && uint64_t(ly.aux) + ly.count > n_det) return bad(at + ": detector out of range");
            break;
        }
        case L_NGEN: {
            if (ly.nwords) return bad(at + ": generation layer with a block");
            uint64_t segs = 0;
            for (uint32_t i = 0; i < ly.count; i++) {
                if (size_t(ly.aux) + i >= P.noise.size()) return bad(at + ": noise descriptor out of range");
                segs += P.noise[ly.aux + i].n_seg;
            }
            if (segs != ly.aux2 || ly.aux2 > P.max_window_segs) return bad(at + ": window size");
            break;
        }
        case L_GAUGE:
            if (!ly.nwords || 3ull * ly.count > ly.nwords) return bad(at + ": block too small");
            for (uint32_t i = 0; i < ly.count; i++)
                if (b[3 * i] >= P.n_slots) return bad(at + ": slot out of range");
            break;
        case L_RECOUT:
            if (!ly.nwords || 2ull * ly.count > ly.nwords) return bad(at + ": block too small");
            for (uint32_t i = 0; i < ly.count; i++)
                if ((b[2 * i] & 0x7FFFFFFFu) >= P.n_slots || b[2 * i + 1] >= n_meas) return bad(at + ": record out of range");
            break;
        case L_NAPPLY: {
            if (ly.nwords || ly.aux >= P.noise.size()) return bad(at + ": apply layer");
            if (uint64_t(ly.aux2) + P.noise[ly.aux].n_seg > P.max_window_segs) return bad(at + ": window base");
            break;
        }
        default:
            return bad(at + ": unknown kind");
        }
    }
    for (size_t i = 0; i < P.noise.size(); i++) {
        const NoiseDesc &nd = P.noise[i];
        const uint64_t words = uint64_t(nd.kind == N_DEP2 ? 2 : 1) * nd.n_units;
        if (nd.kind > N_PC1 || (nd.kind == N_PC1 && nd.t1 > nd.t2) || nd.table >= P.table_p.size() || nd.n_seg != (nd.n_units + kSegUnits - 1) / kSegUnits ||
            uint64_t(nd.tgt_off) + words > P.args.size())
            return bad("noise descriptor " + std::to_string(i));
        for (uint64_t w = 0; w < words; w++) {
            const uint32_t v = P.args[nd.tgt_off + w];
            if (((v & 0xFFFFu) != kDeadSlot && (v & 0xFFFFu) >= P.n_slots) ||
                ((v >> 16) != kDeadSlot && (v >> 16) >= P.n_slots))
                return bad("noise target slot out of range");
        }
    }
    if (P.tables.size() != P.table_p.size() * kTableWords) return bad("table size");
    return TMCS_OK;
}

// meas = false: detector/observable program (c->prog). meas = true: raw
// measurement program (c->prog_meas): gauge Paulis XORed in after every reset
// and measurement (and on z at the start), every record emitted as
// reference XOR flip, detectors and observables left out.
int compile(tmcs_circuit *c, uint32_t flags, bool meas) {
    const bool prune = !(flags & TMCS_FLAG_NO_PRUNE);
    std::vector<std::pair<uint32_t, uint32_t>> gauges;  // (op index, target index) per I_GAUGE
    auto gauge = [&](uint32_t vreg, uint32_t op, uint32_t u, std::vector<IRInst> &irv) {
        irv.push_back({I_GAUGE, vreg, uint32_t(gauges.size())});
        gauges.push_back({op, u});
    };
    const uint64_t Q = c->n_qubits;
    uint32_t V = 0;
    std::vector<IRInst> ir;
    std::vector<IRNoise> noise;
    std::vector<IRParity> pars;
    std::vector<uint32_t> X(Q), Z(Q), rec(c->n_meas), acc(c->n_obs);
    ir.reserve(c->ops.size() * 4 + 2 * Q);

    auto newv = [&]() -> uint32_t { return V++; };
    for (uint64_t q = 0; q < Q; q++) {
        X[q] = newv();
        ir.push_back({I_ZERO, X[q], 0});
        Z[q] = newv();
        ir.push_back({I_ZERO, Z[q], 0});
    }
    if (meas)
        for (uint64_t q = 0; q < Q; q++) gauge(Z[q], uint32_t(c->ops.size()), uint32_t(q), ir);
    for (uint64_t o = 0; o < c->n_obs && !meas; o++) {
        acc[o] = newv();
        ir.push_back({I_ZERO, acc[o], 0});
    }
    uint64_t m = 0, d = 0;
    for (size_t i = 0; i < c->ops.size(); i++) {
        const HostOp &op = c->ops[i];
        const uint32_t *t = c->targets.data() + op.toff;
        switch (op.code) {
        case TMCS_R:
        case TMCS_RX:
            for (uint32_t a = 0; a < op.nt; a++) {
                X[t[a]] = newv();
                ir.push_back({I_ZERO, X[t[a]], 0});
                Z[t[a]] = newv();
                ir.push_back({I_ZERO, Z[t[a]], 0});
                if (meas) gauge(op.code == TMCS_R ? Z[t[a]] : X[t[a]], uint32_t(i), a, ir);
            }
            break;
        case TMCS_H:
            for (uint32_t a = 0; a < op.nt; a++) std::swap(X[t[a]], Z[t[a]]);
            break;
        case TMCS_S:
            for (uint32_t a = 0; a < op.nt; a++) ir.push_back({I_XOR, Z[t[a]], X[t[a]]});
            break;
        case TMCS_CX:
            for (uint32_t a = 0; a + 1 < op.nt; a += 2) {
                ir.push_back({I_XOR, X[t[a + 1]], X[t[a]]});
                ir.push_back({I_XOR, Z[t[a]], Z[t[a + 1]]});
            }
            break;
        case TMCS_M:
        case TMCS_MX:
            for (uint32_t a = 0; a < op.nt; a++) {
                std::vector<uint32_t> &P = (op.code == TMCS_M) ? X : Z;
                rec[m] = P[t[a]];
                uint32_t nv = newv();
                ir.push_back({I_COPY, nv, P[t[a]]});
                P[t[a]] = nv;
                if (meas) {
                    ir.push_back({I_REC, rec[m], uint32_t(m)});
                    gauge(op.code == TMCS_M ? Z[t[a]] : X[t[a]], uint32_t(i), a, ir);
                }
                m++;
            }
            break;
        case TMCS_X_ERROR:
        case TMCS_Z_ERROR:
        case TMCS_DEPOLARIZE1:
        case TMCS_DEPOLARIZE2:
        case TMCS_PAULI_CHANNEL_1: {
            if (!(op.p > 0.0) || op.nt == 0) break;
            IRNoise nz;
            nz.op = uint32_t(i);
            nz.kind = op.code == TMCS_X_ERROR ? N_XERR : op.code == TMCS_Z_ERROR ? N_ZERR
                      : op.code == TMCS_DEPOLARIZE1 ? N_DEP1 : op.code == TMCS_DEPOLARIZE2 ? N_DEP2 : N_PC1;
            nz.p = op.p;
            if (nz.kind == N_PC1) {
                nz.t1 = op.arg;
                nz.t2 = op.arg2;
            }
            nz.comp.reserve(2 * op.nt);
            for (uint32_t a = 0; a < op.nt; a++) {
                nz.comp.push_back(X[t[a]]);
                nz.comp.push_back(Z[t[a]]);
            }
            nz.live.assign(nz.comp.size(), 0);
            ir.push_back({I_NOISE, uint32_t(noise.size()), 0});
            noise.push_back(std::move(nz));
            break;
        }
        case TMCS_XFEED:
            for (uint32_t a = 0; a + 1 < op.nt; a += 2) ir.push_back({I_XOR, X[t[a + 1]], rec[t[a]]});
            break;
        case TMCS_ZFEED:
            for (uint32_t a = 0; a + 1 < op.nt; a += 2) ir.push_back({I_XOR, Z[t[a + 1]], rec[t[a]]});
            break;
        case TMCS_DETECTOR: {
            if (meas) break;
            IRParity p;
            p.acc = uint32_t(d++);
            for (uint32_t a = 0; a < op.nt; a++) p.recs.push_back(rec[t[a]]);
            ir.push_back({I_DET, uint32_t(pars.size()), 0});
            pars.push_back(std::move(p));
            break;
        }
        case TMCS_OBSERVABLE: {
            if (meas) break;
            IRParity p;
            p.acc = acc[op.arg];
            for (uint32_t a = 0; a < op.nt; a++) p.recs.push_back(rec[t[a]]);
            ir.push_back({I_OBS, uint32_t(pars.size()), 0});
            pars.push_back(std::move(p));
            break;
        }
        default:
            break;
        }
    }

    // ---- backward liveness: keep only updates that can reach an output
    std::vector<uint8_t> live(V, 0), keep(ir.size(), 0);
    for (uint64_t o = 0; o < c->n_obs && !meas; o++) live[acc[o]] = 1;
    uint64_t pruned = 0;
    for (size_t k = ir.size(); k-- > 0;) {
        const IRInst &in = ir[k];
        switch (in.kind) {
        case I_ZERO:
            if (live[in.a] || !prune) keep[k] = 1;
            live[in.a] = 0;
            break;
        case I_COPY:
            if (live[in.a] || !prune) {
                keep[k] = 1;
                live[in.b] = 1;
            } else {
                pruned++;
            }
            live[in.a] = 0;
            break;
        case I_XOR:
            if (live[in.a] || !prune) {
                keep[k] = 1;
                live[in.a] = 1;
                live[in.b] = 1;
            } else {
                pruned++;
            }
            break;
        case I_NOISE: {
            IRNoise &nz = noise[in.a];
            bool any = false;
            for (size_t e = 0; e < nz.comp.size(); e++) {
                const bool is_x = (e & 1) == 0;
                // X_ERROR touches only x components, Z_ERROR only z components
                if (nz.kind == N_XERR && !is_x) continue;
                if (nz.kind == N_ZERR && is_x) continue;
                if (live[nz.comp[e]] || !prune) {
                    nz.live[e] = 1;
                    live[nz.comp[e]] = 1;
                    any = true;
                }
            }
            if (any) keep[k] = 1;
            break;
        }
        case I_DET:
        case I_OBS:
            keep[k] = 1;
            for (uint32_t r : pars[in.a].recs) live[r] = 1;
            if (in.kind == I_OBS) live[pars[in.a].acc] = 1;
            break;
        case I_GAUGE:
            if (live[in.a] || !prune) {
                keep[k] = 1;
                live[in.a] = 1;
            }
            break;
        case I_REC:
            keep[k] = 1;
            live[in.a] = 1;
            break;
        }
    }

    // ---- layering: maximal runs of independent same-kind instructions
    std::vector<uint32_t> layer_of(ir.size(), 0xFFFFFFFFu);
    std::vector<uint32_t> wstamp(V, 0xFFFFFFFFu), rstamp(V, 0xFFFFFFFFu);
    std::vector<uint8_t> layer_kind;
    std::vector<std::vector<uint32_t>> layer_insts;
    int cur_kind = -1;
    uint32_t L = 0xFFFFFFFFu;
    auto open = [&](int kind) {
        layer_kind.push_back(uint8_t(kind));
        layer_insts.emplace_back();
        L = uint32_t(layer_kind.size() - 1);
        cur_kind = kind;
    };
    for (size_t k = 0; k < ir.size(); k++) {
        if (!keep[k]) continue;
        const IRInst &in = ir[k];
        bool ok = (cur_kind == int(in.kind)) && in.kind != I_NOISE;
        if (ok) {
            switch (in.kind) {
            case I_ZERO:
                ok = wstamp[in.a] != L && rstamp[in.a] != L;
                break;
            case I_XOR:
            case I_COPY:
                ok = wstamp[in.a] != L && rstamp[in.a] != L && wstamp[in.b] != L;
                break;
            case I_GAUGE:
                ok = wstamp[in.a] != L && rstamp[in.a] != L;
                break;
            case I_REC:
                ok = wstamp[in.a] != L;
                break;
            case I_DET:
                for (uint32_t r : pars[in.a].recs) ok = ok && wstamp[r] != L;
                break;
            case I_OBS:
                ok = wstamp[pars[in.a].acc] != L && rstamp[pars[in.a].acc] != L;
                for (uint32_t r : pars[in.a].recs) ok = ok && wstamp[r] != L;
                break;
            }
        }
        if (!ok) open(in.kind);
        layer_of[k] = L;
        layer_insts[L].push_back(uint32_t(k));
        switch (in.kind) {
        case I_ZERO:
            wstamp[in.a] = L;
            break;
        case I_XOR:
        case I_COPY:
            wstamp[in.a] = L;
            rstamp[in.b] = L;
            break;
        case I_DET:
            for (uint32_t r : pars[in.a].recs) rstamp[r] = L;
            break;
        case I_OBS:
            wstamp[pars[in.a].acc] = L;
            for (uint32_t r : pars[in.a].recs) rstamp[r] = L;
            break;
        case I_NOISE:
            cur_kind = -1;  // noise layers hold one op
            break;
        case I_GAUGE:
            wstamp[in.a] = L;
            break;
        case I_REC:
            rstamp[in.a] = L;
            break;
        }
    }
    const uint32_t n_layers_body = uint32_t(layer_kind.size());
    const uint32_t obsout_layer = n_layers_body;  // final layer writes observables

    // ---- live ranges in layers and interval slot allocation
    std::vector<uint32_t> def_layer(V, 0xFFFFFFFFu), last_layer(V, 0);
    std::vector<uint8_t> used(V, 0);
    auto touch = [&](uint32_t v, uint32_t l) {
        used[v] = 1;
        last_layer[v] = std::max(last_layer[v], l);
    };
    for (size_t k = 0; k < ir.size(); k++) {
        if (!keep[k]) continue;
        const IRInst &in = ir[k];
        const uint32_t l = layer_of[k];
        switch (in.kind) {
        case I_ZERO:
            def_layer[in.a] = l;
            touch(in.a, l);
            break;
        case I_COPY:
            def_layer[in.a] = l;
            touch(in.a, l);
            touch(in.b, l);
            break;
        case I_XOR:
            touch(in.a, l);
            touch(in.b, l);
            break;
        case I_NOISE: {
            const IRNoise &nz = noise[in.a];
            for (size_t e = 0; e < nz.comp.size(); e++)
                if (nz.live[e]) touch(nz.comp[e], l);
            break;
        }
        case I_DET:
        case I_OBS:
            for (uint32_t r : pars[in.a].recs) touch(r, l);
            if (in.kind == I_OBS) touch(pars[in.a].acc, l);
            break;
        case I_GAUGE:
        case I_REC:
            touch(in.a, l);
            break;
        }
    }
    for (uint64_t o = 0; o < c->n_obs && !meas; o++) touch(acc[o], obsout_layer);
    for (uint32_t v = 0; v < V; v++) {
        if (used[v] && def_layer[v] == 0xFFFFFFFFu)
            return fail(TMCS_E_INVALID, "internal: frame value used without definition");
    }
    std::vector<std::vector<uint32_t>> defs_at(n_layers_body + 1), frees_at(n_layers_body + 1);
    for (uint32_t v = 0; v < V; v++) {
        if (!used[v]) continue;
        defs_at[def_layer[v]].push_back(v);
        frees_at[last_layer[v]].push_back(v);
    }
    std::vector<uint32_t> slot(V, kDeadSlot), free_list;
    uint32_t n_slots = 0;
    for (uint32_t l = 0; l <= n_layers_body; l++) {
        for (uint32_t v : defs_at[l]) {
            if (!free_list.empty()) {
                slot[v] = free_list.back();
                free_list.pop_back();
            } else {
                slot[v] = n_slots++;
            }
        }
        for (uint32_t v : frees_at[l]) free_list.push_back(slot[v]);
    }
    if (n_slots > kMaxSlots)
        return fail(TMCS_E_INVALID, "circuit needs " + std::to_string(n_slots) +
                                        " frame slots; at most 65534 are supported");

    // ---- gap tables
    Program &P = meas ? c->prog_meas : c->prog;
    P = Program();
    std::unordered_map<uint64_t, uint32_t> table_id;
    auto table_for = [&](double p, uint32_t *out) -> int {
        uint64_t key;
        std::memcpy(&key, &p, 8);
        auto it = table_id.find(key);
        if (it != table_id.end()) {
            *out = it->second;
            return TMCS_OK;
        }
        uint32_t id = uint32_t(P.table_p.size());
        P.table_p.push_back(p);
        P.tables.resize(P.tables.size() + kTableWords, 0u);
        uint32_t *tab = &P.tables[size_t(id) * kTableWords];
        int rc = gap_table(p, tab);
        if (rc) return rc;
        const float inv = p >= 1.0 ? 0.0f : float(1.0 / std::log2(1.0 - p));
        std::memcpy(tab + kGapLen, &inv, 4);
        table_id[key] = id;
        *out = id;
        return TMCS_OK;
    };

    // ---- emission
    //
    // Every layer's arguments form one 16-byte-aligned block of at most
    // kStageWords words (larger layers are split; their items are
    // independent). Item order inside update layers cycles through the 16
    // residues of the destination slot, so the lanes of a warp tend to hit
    // distinct shared-memory banks.
    tmcs_stats S_meas{};
    tmcs_stats &S = meas ? S_meas : c->stats;
    S = tmcs_stats{};
    auto pad4 = [&]() {
        while (P.args.size() % 4) P.args.push_back(0u);
    };
    // off = start of the layer's block (4-word aligned, written by the caller
    // after pad4()); staged = false for layers without a block.
    auto push_layer = [&](uint32_t kind, uint32_t count, size_t off, uint32_t aux, uint32_t aux2,
                          bool staged) {
        Layer ly{};
        ly.kind = kind;
        ly.count = count;
        ly.aux = aux;
        ly.aux2 = aux2;
        if (staged) {
            pad4();
            ly.off = uint32_t(off);
            ly.nwords = uint32_t(P.args.size() - off);
        }
        P.layers.push_back(ly);
    };
    auto bank_order = [](std::vector<uint32_t> &w) {
        std::vector<std::vector<uint32_t>> bucket(16);
        for (uint32_t v : w) bucket[v & 15u].push_back(v);
        std::vector<uint32_t> out;
        out.reserve(w.size());
        for (size_t r = 0; out.size() < w.size(); r++)
            for (auto &bk : bucket)
                if (r < bk.size()) out.push_back(bk[r]);
        w.swap(out);
    };
    auto emit_words = [&](uint32_t kind, std::vector<uint32_t> &w, bool order) {
        if (order) bank_order(w);
        for (size_t b = 0; b < w.size(); b += kStageWords) {
            const size_t e = std::min(w.size(), b + kStageWords);
            pad4();
            const size_t off = P.args.size();
            P.args.insert(P.args.end(), w.begin() + b, w.begin() + e);
            push_layer(kind, uint32_t(e - b), off, 0, 0, true);
        }
    };
    // single-fault enumeration over the whole op list: noise ops with p > 0
    // in order, each target unit, Pauli index 1..K (K = 1, 1, 3, 15, 3 for
    // X_ERROR, Z_ERROR, DEPOLARIZE1, DEPOLARIZE2, PAULI_CHANNEL_1)
    std::vector<uint64_t> op_fault_base(c->ops.size(), 0);
    {
        uint64_t f = 0;
        for (size_t i = 0; i < c->ops.size(); i++) {
            const HostOp &op = c->ops[i];
            op_fault_base[i] = f;
            if (!is_noise(op.code) || !(op.p > 0.0)) continue;
            const uint64_t units = op.code == TMCS_DEPOLARIZE2 ? op.nt / 2 : op.nt;
            const uint64_t K = op.code == TMCS_DEPOLARIZE2 ? 15 : (op.code == TMCS_DEPOLARIZE1 ||
                                                                   op.code == TMCS_PAULI_CHANNEL_1) ? 3 : 1;
            f += units * K;
        }
        P.n_faults = f;
    }
    // noise descriptors (program order) and their generation windows
    std::vector<uint32_t> noise_layer_desc(n_layers_body, 0xFFFFFFFFu);
    std::vector<uint32_t> desc_win_first, desc_win_count, desc_win_segs, desc_win_base;
    for (uint32_t l = 0; l < n_layers_body; l++) {
        if (layer_kind[l] != I_NOISE) continue;
        const IRNoise &nz = noise[ir[layer_insts[l][0]].a];
        NoiseDesc nd{};
        nd.op_index = nz.op;
        nd.kind = nz.kind;
        nd.t1 = nz.t1;
        nd.t2 = nz.t2;
        int rc = table_for(nz.p, &nd.table);
        if (rc) return rc;
        const uint32_t nq = uint32_t(nz.comp.size() / 2);
        nd.n_units = nz.kind == N_DEP2 ? nq / 2 : nq;
        nd.n_seg = (nd.n_units + kSegUnits - 1) / kSegUnits;
        nd.tgt_off = uint32_t(P.args.size());
        for (uint32_t q = 0; q < nq; q++) {
            uint32_t xs = nz.live[2 * q] ? slot[nz.comp[2 * q]] : kDeadSlot;
            uint32_t zs = nz.live[2 * q + 1] ? slot[nz.comp[2 * q + 1]] : kDeadSlot;
            P.args.push_back(xs | (zs << 16));
            S.live_components += (xs != kDeadSlot) + (zs != kDeadSlot);
        }
        noise_layer_desc[l] = uint32_t(P.noise.size());
        P.noise.push_back(nd);
        P.fault_base.push_back(op_fault_base[nz.op]);
        S.n_noise_ops++;
        S.n_noise_units += nd.n_units;
        S.n_noise_segments += nd.n_seg;
    }
    {
        const uint32_t nd_count = uint32_t(P.noise.size());
        desc_win_first.assign(nd_count, 0);
        desc_win_count.assign(nd_count, 0);
        desc_win_segs.assign(nd_count, 0);
        desc_win_base.assign(nd_count, 0);
        uint32_t i = 0;
        while (i < nd_count) {
            uint32_t j = i, segs = 0;
            while (j < nd_count && (j == i || (segs + P.noise[j].n_seg <= kWindowSegs && j - i < kWindowOps))) {
                desc_win_base[j] = segs;
                segs += P.noise[j].n_seg;
                j++;
            }
            for (uint32_t k = i; k < j; k++) {
                desc_win_first[k] = i;
                desc_win_count[k] = j - i;
                desc_win_segs[k] = segs;
            }
            P.max_window_segs = std::max(P.max_window_segs, segs);
            i = j;
        }
    }
    for (uint32_t l = 0; l < n_layers_body; l++) {
        const std::vector<uint32_t> &ins = layer_insts[l];
        switch (layer_kind[l]) {
        case I_ZERO: {
            std::vector<uint32_t> w;
            w.reserve(ins.size());
            for (uint32_t k : ins) w.push_back(slot[ir[k].a]);
            emit_words(L_ZERO, w, true);
            S.n_zero += ins.size();
            break;
        }
        case I_XOR:
        case I_COPY: {
            std::vector<uint32_t> w;
            w.reserve(ins.size());
            for (uint32_t k : ins) w.push_back(slot[ir[k].a] | (slot[ir[k].b] << 16));
            emit_words(layer_kind[l] == I_XOR ? L_XOR : L_COPY, w, true);
            (layer_kind[l] == I_XOR ? S.n_xor : S.n_copy) += ins.size();
            break;
        }
        case I_NOISE: {
            const uint32_t d = noise_layer_desc[l];
            if (desc_win_first[d] == d) push_layer(L_NGEN, desc_win_count[d], 0, d, desc_win_segs[d], false);
            push_layer(L_NAPPLY, 1, 0, d, desc_win_base[d], false);
            break;
        }
        case I_GAUGE: {
            // 3 words per item: slot, op index, target index
            const size_t per = kStageWords / 3;
            for (size_t b0 = 0; b0 < ins.size(); b0 += per) {
                const size_t e0 = std::min(ins.size(), b0 + per);
                pad4();
                const size_t off = P.args.size();
                for (size_t e = b0; e < e0; e++) {
                    const auto &g = gauges[ir[ins[e]].b];
                    P.args.push_back(slot[ir[ins[e]].a]);
                    P.args.push_back(g.first);
                    P.args.push_back(g.second);
                }
                push_layer(L_GAUGE, uint32_t(e0 - b0), off, 0, 0, true);
            }
            break;
        }
        case I_REC: {
            // 2 words per item: slot | reference bit << 31, record index
            const size_t per = kStageWords / 2;
            for (size_t b0 = 0; b0 < ins.size(); b0 += per) {
                const size_t e0 = std::min(ins.size(), b0 + per);
                pad4();
                const size_t off = P.args.size();
                for (size_t e = b0; e < e0; e++) {
                    const uint32_t r = ir[ins[e]].b;
                    P.args.push_back(slot[ir[ins[e]].a] | (uint32_t(c->ref_bits[r] & 1u) << 31));
                    P.args.push_back(r);
                }
                push_layer(L_RECOUT, uint32_t(e0 - b0), off, 0, 0, true);
            }
            break;
        }
        case I_DET:
        case I_OBS: {
            const bool det = layer_kind[l] == I_DET;
            size_t e = 0;
            while (e < ins.size()) {
                // greedily take detectors while bounds + lists fit one stage block
                size_t f = e, words = 1;
                while (f < ins.size()) {
                    const size_t len = pars[ir[ins[f]].a].recs.size() + (det ? 0 : 1);
                    if (words + 1 + len > kStageWords && f > e) break;
                    words += 1 + len;
                    f++;
                }
                if (words > kStageWords)
                    return fail(TMCS_E_INVALID, "a detector or observable lists more than " +
                                                    std::to_string(kStageWords - 2) + " records");
                pad4();
                const size_t off = P.args.size();
                const size_t nb = f - e + 1;
                P.args.resize(off + nb);
                for (size_t i = e; i < f; i++) {
                    const IRParity &pp = pars[ir[ins[i]].a];
                    P.args[off + (i - e)] = uint32_t(P.args.size() - off);
                    if (!det) P.args.push_back(slot[pp.acc]);
                    for (uint32_t r : pp.recs) P.args.push_back(slot[r]);
                    S.n_parity_terms += pp.recs.size();
                }
                P.args[off + (f - e)] = uint32_t(P.args.size() - off);
                push_layer(det ? L_DET : L_OBS, uint32_t(f - e), off, det ? pars[ir[ins[e]].a].acc : 0, 0, true);
                e = f;
            }
            break;
        }
        }
    }
    if (c->n_obs && !meas) {
        std::vector<uint32_t> w;
        for (uint64_t o = 0; o < c->n_obs; o++) w.push_back(slot[acc[o]]);
        if (w.size() > kStageWords) return fail(TMCS_E_INVALID, "too many observables");
        emit_words(L_OBSOUT, w, false);
    }
    pad4();
    {
        uint32_t q = 0;
        for (Layer &ly : P.layers) ly.seq = ly.nwords ? q++ : 0u;
    }
    P.n_slots = n_slots;
    P.n_det = c->n_det;
    P.n_obs = c->n_obs;
    S.n_layers = P.layers.size();
    S.n_slots = n_slots;
    S.pruned_updates = pruned;
    return validate_program(P, c->n_det, c->n_obs, c->n_meas);
}

// ------------------------------------------------------------- audit
//
// 64-lane noiseless frame run with random gauge Paulis after every reset and
// measurement (random Z after R/M, random X after RX/MX): these leave the
// state unchanged, so every deterministic parity stays 0 in every lane while
// a random one is 1 in about half of them.

static uint64_t mix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int audit(const tmcs_circuit *c) {
    std::vector<uint64_t> x(c->n_qubits), z(c->n_qubits), rec(c->n_meas), obs(c->n_obs);
    for (int pass = 0; pass < 2; pass++) {
        uint64_t s = 0x5EEDull + 1000003ull * uint64_t(pass);
        std::fill(x.begin(), x.end(), 0);
        std::fill(z.begin(), z.end(), 0);
        std::fill(obs.begin(), obs.end(), 0);
        uint64_t m = 0, d = 0;
        for (const HostOp &op : c->ops) {
            const uint32_t *t = c->targets.data() + op.toff;
            switch (op.code) {
            case TMCS_R:
                for (uint32_t a = 0; a < op.nt; a++) { x[t[a]] = 0; z[t[a]] = mix64(s); }
                break;
            case TMCS_RX:
                for (uint32_t a = 0; a < op.nt; a++) { z[t[a]] = 0; x[t[a]] = mix64(s); }
                break;
            case TMCS_H:
                for (uint32_t a = 0; a < op.nt; a++) std::swap(x[t[a]], z[t[a]]);
                break;
            case TMCS_S:
                for (uint32_t a = 0; a < op.nt; a++) z[t[a]] ^= x[t[a]];
                break;
            case TMCS_CX:
                for (uint32_t a = 0; a + 1 < op.nt; a += 2) {
                    x[t[a + 1]] ^= x[t[a]];
                    z[t[a]] ^= z[t[a + 1]];
                }
                break;
            case TMCS_M:
                for (uint32_t a = 0; a < op.nt; a++) { rec[m++] = x[t[a]]; z[t[a]] ^= mix64(s); }
                break;
            case TMCS_MX:
                for (uint32_t a = 0; a < op.nt; a++) { rec[m++] = z[t[a]]; x[t[a]] ^= mix64(s); }
                break;
            case TMCS_XFEED:
                for (uint32_t a = 0; a + 1 < op.nt; a += 2) x[t[a + 1]] ^= rec[t[a]];
                break;
            case TMCS_ZFEED:
                for (uint32_t a = 0; a + 1 < op.nt; a += 2) z[t[a + 1]] ^= rec[t[a]];
                break;
            case TMCS_DETECTOR: {
                uint64_t v = 0;
                for (uint32_t a = 0; a < op.nt; a++) v ^= rec[t[a]];
                if (v)
                    return fail(TMCS_E_NONDETERMINISTIC,
                                "detector " + std::to_string(d) + " is not deterministic");
                d++;
                break;
            }
            case TMCS_OBSERVABLE:
                for (uint32_t a = 0; a < op.nt; a++) obs[op.arg] ^= rec[t[a]];
                break;
            default:
                break;
            }
        }
        for (uint64_t o = 0; o < c->n_obs; o++)
            if (obs[o])
                return fail(TMCS_E_NONDETERMINISTIC,
                            "observable " + std::to_string(o) + " is not deterministic");
    }
    return TMCS_OK;
}

// ------------------------------------------------------ reference sample
//
// CHP tableau (Aaronson & Gottesman, PRA 70, 052328, 2004): rows 0..n-1 are
// destabilizers, n..2n-1 stabilizers, row 2n is scratch; each row is packed
// x bits, z bits and a sign. Random outcomes resolve to 0.

namespace {

struct Tableau {
    size_t n, W;
    std::vector<uint64_t> x, z;
    std::vector<uint8_t> r;
    explicit Tableau(size_t n_) : n(n_), W((n_ + 63) / 64), x((2 * n_ + 1) * W), z((2 * n_ + 1) * W), r(2 * n_ + 1) {
        for (size_t i = 0; i < n; i++) {
            x[i * W + i / 64] |= 1ull << (i % 64);
            z[(n + i) * W + i / 64] |= 1ull << (i % 64);
        }
    }
    uint64_t *xr(size_t i) { return &x[i * W]; }
    uint64_t *zr(size_t i) { return &z[i * W]; }
    bool xb(size_t i, size_t a) const { return (x[i * W + a / 64] >> (a % 64)) & 1; }

    void h(size_t a) {
        const size_t w = a / 64;
        const uint64_t bit = 1ull << (a % 64);
        for (size_t i = 0; i < 2 * n; i++) {
            uint64_t &xw = x[i * W + w], &zw = z[i * W + w];
            const bool xi = xw & bit, zi = zw & bit;
            r[i] ^= uint8_t(xi && zi);
            if (xi != zi) { xw ^= bit; zw ^= bit; }
        }
    }
    void s(size_t a) {
        const size_t w = a / 64;
        const uint64_t bit = 1ull << (a % 64);
        for (size_t i = 0; i < 2 * n; i++) {
            uint64_t &xw = x[i * W + w], &zw = z[i * W + w];
            const bool xi = xw & bit, zi = zw & bit;
            r[i] ^= uint8_t(xi && zi);
            if (xi) zw ^= bit;
        }
    }
    void cx(size_t a, size_t b) {
        const size_t wa = a / 64, wb = b / 64;
        const uint64_t ba = 1ull << (a % 64), bb = 1ull << (b % 64);
        for (size_t i = 0; i < 2 * n; i++) {
            uint64_t *xw = &x[i * W], *zw = &z[i * W];
            const bool xa = xw[wa] & ba, za = zw[wa] & ba, xb_ = xw[wb] & bb, zb = zw[wb] & bb;
            r[i] ^= uint8_t(xa && zb && (xb_ == za));
            if (xa) xw[wb] ^= bb;
            if (zb) zw[wa] ^= ba;
        }
    }
    void pauli_x(size_t a) {
        for (size_t i = 0; i < 2 * n; i++) r[i] ^= uint8_t((z[i * W + a / 64] >> (a % 64)) & 1);
    }
    void pauli_z(size_t a) {
        for (size_t i = 0; i < 2 * n; i++) r[i] ^= uint8_t((x[i * W + a / 64] >> (a % 64)) & 1);
    }
    // row h <- row i * row h, with the sign rule of the tableau algorithm
    void rowsum(size_t h, size_t i) {
        int64_t sum = 2 * int64_t(r[h]) + 2 * int64_t(r[i]);
        uint64_t *x1 = xr(i), *z1 = zr(i), *x2 = xr(h), *z2 = zr(h);
        for (size_t w = 0; w < W; w++) {
            const uint64_t a = x1[w], b = z1[w], cx_ = x2[w], dz = z2[w];
            // g = +1 / -1 cases of the phase exponent of P1 * P2
            const uint64_t plus = (a & b & ~cx_ & dz) | (a & ~b & cx_ & dz) | (~a & b & cx_ & ~dz);
            const uint64_t minus = (a & b & cx_ & ~dz) | (a & ~b & ~cx_ & dz) | (~a & b & cx_ & dz);
            sum += int64_t(__builtin_popcountll(plus)) - int64_t(__builtin_popcountll(minus));
            x2[w] ^= a;
            z2[w] ^= b;
        }
        sum %= 4;
        if (sum < 0) sum += 4;
        r[h] = uint8_t(sum == 2);
    }
    int measure(size_t a) {
        size_t p = SIZE_MAX;
        for (size_t i = n; i < 2 * n; i++)
            if (xb(i, a)) { p = i; break; }
        if (p != SIZE_MAX) {
            for (size_t i = 0; i < 2 * n; i++)
                if (i != p && xb(i, a)) rowsum(i, p);
            std::memcpy(xr(p - n), xr(p), W * 8);
            std::memcpy(zr(p - n), zr(p), W * 8);
            r[p - n] = r[p];
            std::memset(xr(p), 0, W * 8);
            std::memset(zr(p), 0, W * 8);
            zr(p)[a / 64] |= 1ull << (a % 64);
            r[p] = 0;
            return 0;
        }
        const size_t sc = 2 * n;
        std::memset(xr(sc), 0, W * 8);
        std::memset(zr(sc), 0, W * 8);
        r[sc] = 0;
        for (size_t i = 0; i < n; i++)
            if (xb(i, a)) rowsum(sc, i + n);
        return r[sc];
    }
};

}  // namespace

// Noiseless run of the circuit on the stabilizer tableau: the reference
// measurement record (one byte per record, 0 or 1).
int reference_record(const tmcs_circuit *c, std::vector<uint8_t> *out) {
    try {
        Tableau T(c->n_qubits);
        std::vector<uint8_t> &rec = *out;
        rec.clear();
        rec.reserve(c->n_meas);
        for (const HostOp &op : c->ops) {
            const uint32_t *t = c->targets.data() + op.toff;
            switch (op.code) {
            case TMCS_R:
                for (uint32_t a = 0; a < op.nt; a++)
                    if (T.measure(t[a])) T.pauli_x(t[a]);
                break;
            case TMCS_RX:
                for (uint32_t a = 0; a < op.nt; a++) {
                    if (T.measure(t[a])) T.pauli_x(t[a]);
                    T.h(t[a]);
                }
                break;
            case TMCS_H:
                for (uint32_t a = 0; a < op.nt; a++) T.h(t[a]);
                break;
            case TMCS_S:
                for (uint32_t a = 0; a < op.nt; a++) T.s(t[a]);
                break;
            case TMCS_CX:
                for (uint32_t a = 0; a + 1 < op.nt; a += 2) T.cx(t[a], t[a + 1]);
                break;
            case TMCS_M:
                for (uint32_t a = 0; a < op.nt; a++) rec.push_back(uint8_t(T.measure(t[a])));
                break;
            case TMCS_MX:
                for (uint32_t a = 0; a < op.nt; a++) {
                    T.h(t[a]);
                    rec.push_back(uint8_t(T.measure(t[a])));
                    T.h(t[a]);
                }
                break;
            case TMCS_XFEED:
                for (uint32_t a = 0; a + 1 < op.nt; a += 2)
                    if (rec[t[a]]) T.pauli_x(t[a + 1]);
                break;
            case TMCS_ZFEED:
                for (uint32_t a = 0; a + 1 < op.nt; a += 2)
                    if (rec[t[a]]) T.pauli_z(t[a + 1]);
                break;
            default:
                break;
            }
        }
    } catch (const std::bad_alloc &) {
        return fail(TMCS_E_OOM, "out of host memory for the tableau");
    }
    return TMCS_OK;
}

// Builds, once, the program that emits raw measurement records: the
// reference record is XORed into the sampled frame bits, and every reset and
// measurement re-randomises the anticommuting frame component (gauge).
int build_measurement_program(tmcs_circuit *c) {
    if (c->meas_built) return TMCS_OK;
    try {
        int rc = reference_record(c, &c->ref_bits);
        if (rc) return rc;
        rc = compile(c, c->flags, true);
        if (rc) return rc;
    } catch (const std::bad_alloc &) {
        return fail(TMCS_E_OOM, "out of host memory while compiling");
    }
    c->meas_built = true;
    return TMCS_OK;
}

// Detector error model columns (Methods "Decoding"): single faults in the
// order of tmcs_fault_count, each read from the event-signature table the
// samplers apply, merged by signature. Faults of one noise unit are mutually
// exclusive and units are independent, so a column fires (an odd number of
// its faults occur) with probability (1 - prod_u (1 - 2 P_u)) / 2, P_u the
// summed probability of the unit's faults in the column.
namespace {
struct VecHash {
    size_t operator()(const std::vector<uint32_t> &v) const {
        uint64_t h = 0x9E3779B97F4A7C15ull ^ v.size();
        for (uint32_t x : v) h = (h ^ x) * 0x100000001B3ull;
        return size_t(h ^ (h >> 29));
    }
};
}  // namespace

// Output list of one event slot, as sorted ids (detector, or kSigObsFlag |
// observable); empty if the event flips nothing.
static void slot_outputs(const SigProgram &G, size_t slot, std::vector<uint32_t> &w) {
    w.clear();
    const uint32_t w0 = G.ev_ent[2 * slot], w1 = G.ev_ent[2 * slot + 1];
    if (w0 == kEvNone) return;
    if (w0 & kEvOverflow) {
        w.assign(G.ev_ent.begin() + (w0 & ~kEvOverflow), G.ev_ent.begin() + (w0 & ~kEvOverflow) + w1);
    } else {
        w.push_back(w0);
        if (w1 != kEvNone) w.push_back(w1);
    }
    for (uint32_t &e : w) e = (e & (1u << 29)) ? (kSigObsFlag | (e & 0x1FFFFFFFu)) : e;
    std::sort(w.begin(), w.end());
}

static void build_dem(const tmcs_circuit *c) {
    const SigProgram &G = c->sig;
    std::unordered_map<std::vector<uint32_t>, uint32_t, VecHash> index;
    std::vector<std::vector<uint32_t>> cols;
    std::vector<double> prod;
    std::vector<uint64_t> nf;
    struct UnitCol {
        std::vector<uint32_t> sig;
        double p;
        uint32_t n;
    };
    std::vector<UnitCol> unit;  // this unit's non-empty faults, by signature
    std::vector<uint32_t> w;
    for (uint32_t di = 0; di < G.noise.size(); di++) {
        const NoiseDesc &nd = G.noise[di];
        const uint32_t KP = sig_paulis(nd.kind);
        const double p = c->ops[nd.op_index].p;
        for (uint32_t u = 0; u < nd.n_units; u++) {
            unit.clear();
            for (uint32_t k = 1; k <= KP; k++) {
                slot_outputs(G, size_t(G.ev_base[di]) + size_t(u) * KP + (k - 1), w);
                if (w.empty()) continue;
                double pf = p / double(KP);
                if (nd.kind == N_PC1) {
                    // the sampled split: X below t1, Y in [t1, t2), Z from t2
                    // (Pauli index 1 = X, 3 = Y, 2 = Z)
                    const double lo = k == 1 ? 0.0 : k == 3 ? double(nd.t1) : double(nd.t2);
                    const double hi = k == 1 ? double(nd.t1) : k == 3 ? double(nd.t2) : 4294967296.0;
                    pf = p * (hi - lo) / 4294967296.0;
                }
                bool merged = false;
                for (UnitCol &e : unit)
                    if (e.sig == w) {
                        e.p += pf;
                        e.n++;
                        merged = true;
                        break;
                    }
                if (!merged) unit.push_back({w, pf, 1u});
            }
            for (const UnitCol &e : unit) {
                auto it = index.find(e.sig);
                uint32_t col;
                if (it == index.end()) {
                    col = uint32_t(cols.size());
                    index.emplace(e.sig, col);
                    cols.push_back(e.sig);
                    prod.push_back(1.0);
                    nf.push_back(0);
                } else {
                    col = it->second;
                }
                prod[col] *= 1.0 - 2.0 * e.p;
                nf[col] += e.n;
            }
        }
    }
    // canonical order: columns sorted by their entry lists
    std::vector<uint32_t> ord(cols.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = uint32_t(i);
    std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) { return cols[a] < cols[b]; });
    c->dem_off.assign(1, 0);
    c->dem_ent.clear();
    c->dem_p.clear();
    c->dem_nf.clear();
    for (uint32_t i : ord) {
        c->dem_ent.insert(c->dem_ent.end(), cols[i].begin(), cols[i].end());
        c->dem_off.push_back(c->dem_ent.size());
        c->dem_p.push_back((1.0 - prod[i]) / 2.0);
        c->dem_nf.push_back(nf[i]);
    }
    c->dem_built = true;
}

}  // namespace tmcs

using namespace tmcs;

extern "C" {

const char *tmcs_last_error(void) { return g_last_error.c_str(); }

int tmcs_debug_gap_table(double p, uint32_t *table) {
    if (!table) return fail(TMCS_E_INVALID, "null table pointer");
    return gap_table(p, table);
}

int tmcs_circuit_build(const tmcs_op *ops, size_t n_ops, uint32_t flags, tmcs_circuit **out) {
    if (!out) return fail(TMCS_E_INVALID, "out is NULL");
    *out = nullptr;
    if (n_ops && !ops) return fail(TMCS_E_INVALID, "ops is NULL");
    if (flags & ~uint32_t(TMCS_FLAG_NO_AUDIT | TMCS_FLAG_NO_PRUNE))
        return fail(TMCS_E_INVALID, "unknown flag bits");
    tmcs_circuit *c = new (std::nothrow) tmcs_circuit();
    if (!c) return fail(TMCS_E_OOM, "out of host memory");
    try {
        c->ops.reserve(n_ops);
        uint64_t m = 0, d = 0, q = 0, nobs = 0;
        for (size_t i = 0; i < n_ops; i++) {
            const tmcs_op &op = ops[i];
            const std::string where = "op " + std::to_string(i) + ": ";
            if (op.code > TMCS_PAULI_CHANNEL_1) { delete c; return fail(TMCS_E_INVALID, where + "unknown opcode"); }
            if (op.arg2 && op.code != TMCS_PAULI_CHANNEL_1) { delete c; return fail(TMCS_E_INVALID, where + "arg2 must be 0"); }
            if (op.code == TMCS_PAULI_CHANNEL_1 && op.arg > op.arg2) {
                delete c;
                return fail(TMCS_E_INVALID, where + "PAULI_CHANNEL_1 thresholds must satisfy arg <= arg2");
            }
            if (op.n_targets && !op.targets) { delete c; return fail(TMCS_E_INVALID, where + "targets is NULL"); }
            if (is_pair(op.code) && (op.n_targets & 1)) { delete c; return fail(TMCS_E_INVALID, where + "odd target count"); }
            if (is_noise(op.code)) {
                if (!(op.p >= 0.0 && op.p <= 1.0)) { delete c; return fail(TMCS_E_INVALID, where + "probability outside [0, 1]"); }
                if (op.p > 0.0 && op.p < 1e-12) { delete c; return fail(TMCS_E_INVALID, where + "probability below 1e-12"); }
            }
            if (c->targets.size() + op.n_targets > 0xFFFFFFFFull) { delete c; return fail(TMCS_E_INVALID, "too many targets"); }
            HostOp h{op.code, op.p, op.arg, uint32_t(c->targets.size()), op.n_targets, op.arg2};
            const uint32_t *t = op.targets;
            if (op.code == TMCS_DETECTOR || op.code == TMCS_OBSERVABLE) {
                for (uint32_t a = 0; a < op.n_targets; a++)
                    if (t[a] >= m) { delete c; return fail(TMCS_E_INVALID, where + "record index out of range"); }
                if (op.code == TMCS_DETECTOR) d++;
                else nobs = std::max<uint64_t>(nobs, uint64_t(op.arg) + 1);
            } else if (op.code == TMCS_XFEED || op.code == TMCS_ZFEED) {
                for (uint32_t a = 0; a + 1 < op.n_targets; a += 2) {
                    if (t[a] >= m) { delete c; return fail(TMCS_E_INVALID, where + "record index out of range"); }
                    q = std::max<uint64_t>(q, uint64_t(t[a + 1]) + 1);
                }
            } else if (op.code != TMCS_TICK) {
                for (uint32_t a = 0; a < op.n_targets; a++) q = std::max<uint64_t>(q, uint64_t(t[a]) + 1);
                if (op.code == TMCS_CX || op.code == TMCS_DEPOLARIZE2)
                    for (uint32_t a = 0; a + 1 < op.n_targets; a += 2)
                        if (t[a] == t[a + 1]) { delete c; return fail(TMCS_E_INVALID, where + "pair on one qubit"); }
            }
            if (op.code == TMCS_M || op.code == TMCS_MX) m += op.n_targets;
            c->targets.insert(c->targets.end(), t, t + op.n_targets);
            c->ops.push_back(h);
        }
        if (m > 0xFFFFFFFFull || q > 0xFFFFFFFFull || n_ops > 0xFFFFFFFFull) {
            delete c;
            return fail(TMCS_E_INVALID, "circuit too large");
        }
        // Noise ops must hit distinct qubits: the sampler applies events of
        // different target units concurrently.
        {
            std::vector<uint32_t> seen(q, 0xFFFFFFFFu);
            for (size_t i = 0; i < c->ops.size(); i++) {
                const HostOp &op = c->ops[i];
                if (!is_noise(op.code)) continue;
                for (uint32_t a = 0; a < op.nt; a++) {
                    uint32_t v = c->targets[op.toff + a];
                    if (seen[v] == uint32_t(i)) {
                        delete c;
                        return fail(TMCS_E_INVALID, "op " + std::to_string(i) + ": noise op repeats a qubit");
                    }
                    seen[v] = uint32_t(i);
                }
            }
        }
        c->n_qubits = q;
        c->n_meas = m;
        c->n_det = d;
        c->n_obs = nobs;
        if (!(flags & TMCS_FLAG_NO_AUDIT)) {
            int rc = audit(c);
            if (rc) { delete c; return rc; }
        }
        c->flags = flags;
        int rc = compile(c, flags, false);
        if (rc) { delete c; return rc; }
        const char *wenv = std::getenv("TMCS_SIG_WINDOW");
        const uint32_t max_window = (wenv && *wenv) ? uint32_t(std::atoi(wenv)) : 4096u;
        rc = build_signature_program(c, max_window);
        if (rc) { delete c; return rc; }
    } catch (const std::bad_alloc &) {
        delete c;
        return fail(TMCS_E_OOM, "out of host memory while compiling");
    }
    *out = c;
    set_error("");
    return TMCS_OK;
}

int tmcs_circuit_free(tmcs_circuit *c) {
    if (!c) return TMCS_OK;
    free_device_programs(c);
    delete c;
    return TMCS_OK;
}

int tmcs_circuit_info(const tmcs_circuit *c, uint64_t *n_qubits, uint64_t *n_meas, uint64_t *n_det,
                      uint64_t *n_obs, uint64_t *device_bytes) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    if (n_qubits) *n_qubits = c->n_qubits;
    if (n_meas) *n_meas = c->n_meas;
    if (n_det) *n_det = c->n_det;
    if (n_obs) *n_obs = c->n_obs;
    if (device_bytes) *device_bytes = program_bytes(c->prog);
    return TMCS_OK;
}

int tmcs_fault_count(const tmcs_circuit *c, uint64_t *n_faults) {
    if (!c || !n_faults) return fail(TMCS_E_INVALID, "NULL argument");
    *n_faults = c->prog.n_faults;
    return TMCS_OK;
}

int tmcs_circuit_stats(const tmcs_circuit *c, tmcs_stats *out) {
    if (!c || !out) return fail(TMCS_E_INVALID, "NULL argument");
    *out = c->stats;
    const SigProgram &G = c->sig;
    out->sig_ok = G.ok ? 1 : 0;
    out->sig_generators = G.gen_off.empty() ? 0 : G.gen_off.size() - 1;
    out->sig_entries = G.gen_ent.size();
    out->sig_build_us = uint64_t(G.build_seconds * 1e6);
    out->sig_window = out->sig_steps = out->sig_items = out->sig_max_step_items = 0;
    out->sig_schedules = out->sig_pipe_schedules = out->sig_min_window = 0;
    for (const SigSchedule &S : G.sched) {
        if (S.lag) {
            out->sig_pipe_schedules++;
            continue;
        }
        out->sig_schedules++;
        out->sig_min_window = S.window;
    }
    if (!G.sched.empty()) {
        const SigSchedule &S = G.sched[0];
        out->sig_window = S.window;
        out->sig_steps = S.steps.size();
        out->sig_items = S.items.size() / 2;
        for (const SigStep &st : S.steps)
            out->sig_max_step_items = std::max<uint64_t>(out->sig_max_step_items, st.item_end - st.item_begin);
    }
    return TMCS_OK;
}

int tmcs_dem_columns(const tmcs_circuit *c, uint64_t *n_cols, uint64_t *n_entries, uint64_t *col_off,
                     uint32_t *entries, double *col_p, uint64_t *col_faults) {
    if (!c || !n_cols || !n_entries) return fail(TMCS_E_INVALID, "NULL argument");
    const SigProgram &G = c->sig;
    if (!G.ok) return fail(TMCS_E_INVALID, "no event-signature table: " + G.why);
    std::lock_guard<std::mutex> lock(c->mu);
    if (!c->dem_built) {
        try {
            build_dem(c);
        } catch (const std::bad_alloc &) {
            return fail(TMCS_E_OOM, "detector error model: out of host memory");
        }
    }
    const uint64_t nc = c->dem_p.size(), ne = c->dem_ent.size();
    const bool fill = col_off || entries || col_p || col_faults;
    if (fill && (*n_cols < nc || *n_entries < ne))
        return fail(TMCS_E_BUFFER, "column buffers smaller than the model (" + std::to_string(nc) + " columns, " +
                                       std::to_string(ne) + " entries)");
    *n_cols = nc;
    *n_entries = ne;
    if (col_off) std::memcpy(col_off, c->dem_off.data(), (nc + 1) * sizeof(uint64_t));
    if (entries && ne) std::memcpy(entries, c->dem_ent.data(), ne * sizeof(uint32_t));
    if (col_p && nc) std::memcpy(col_p, c->dem_p.data(), nc * sizeof(double));
    if (col_faults && nc) std::memcpy(col_faults, c->dem_nf.data(), nc * sizeof(uint64_t));
    return TMCS_OK;
}

int tmcs_fault_outputs(const tmcs_circuit *c, uint64_t fault, uint32_t *out, uint32_t cap, uint32_t *n_out) {
    if (!c || !n_out || (cap && !out)) return fail(TMCS_E_INVALID, "NULL argument");
    const SigProgram &G = c->sig;
    if (!G.ok) return fail(TMCS_E_INVALID, "no event-signature table: " + G.why);
    // read from the device table the samplers apply (one slot per event, in
    // fault order), converted back to output ids
    uint64_t f = fault;
    for (uint32_t di = 0; di < G.noise.size(); di++) {
        const NoiseDesc &nd = G.noise[di];
        const uint64_t nf = uint64_t(nd.n_units) * sig_paulis(nd.kind);
        if (f >= nf) {
            f -= nf;
            continue;
        }
        const size_t slot = 2 * (size_t(G.ev_base[di]) + size_t(f));
        const uint32_t w0 = G.ev_ent[slot], w1 = G.ev_ent[slot + 1];
        std::vector<uint32_t> w;
        if (w0 == kEvNone) {
        } else if (w0 & kEvOverflow) {
            w.assign(G.ev_ent.begin() + (w0 & ~kEvOverflow), G.ev_ent.begin() + (w0 & ~kEvOverflow) + w1);
        } else {
            w.push_back(w0);
            if (w1 != kEvNone) w.push_back(w1);
        }
        for (uint32_t &e : w) e = (e & (1u << 29)) ? (kSigObsFlag | (e & 0x1FFFFFFFu)) : e;
        std::sort(w.begin(), w.end());
        *n_out = uint32_t(w.size());
        for (size_t i = 0; i < w.size() && i < cap; i++) out[i] = w[i];
        return TMCS_OK;
    }
    return fail(TMCS_E_INVALID, "fault index out of range");
}

int tmcs_reference_sample(const tmcs_circuit *c, uint8_t *meas_bits) {
    if (!c || (!meas_bits && c->n_meas)) return fail(TMCS_E_INVALID, "NULL argument");
    std::vector<uint8_t> rec;
    int rc = reference_record(c, &rec);
    if (rc) return rc;
    if (c->n_meas) std::memset(meas_bits, 0, (c->n_meas + 7) / 8);
    for (size_t i = 0; i < rec.size(); i++)
        if (rec[i]) meas_bits[i / 8] |= uint8_t(1u << (i % 8));
    return TMCS_OK;
}

}  // extern "C"
