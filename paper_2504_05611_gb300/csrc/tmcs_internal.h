// Internal definitions shared by the host compiler (tmcs_host.cpp) and the
// CUDA sampler (tmcs_sample.cu). Not part of the public ABI.
#pragma once

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tmcs.h"

namespace tmcs {

// ---------------------------------------------------------------- program
//
// A compiled circuit is a straight-line program over "slots": shared-memory
// rows that each hold one frame component (the x or z bit of one qubit over
// the CTA's shots) or one measurement record. Gates become slot XORs/copies
// (H is a renaming and costs nothing), resets become clears, noise ops become
// event streams XORed into slots, detectors/observables become parities of
// record slots. Layers group independent updates; the kernel runs one layer
// at a time with a barrier in between.

enum LayerKind : uint32_t {
    L_ZERO = 0,    // block[i] = slot                          -> slot = 0
    L_XOR = 1,     // block[i] = dst | src << 16               -> dst ^= src
    L_COPY = 2,    // block[i] = dst | src << 16               -> dst = src
    L_NGEN = 3,    // walk the event streams of noise descriptors aux .. aux+count-1
                   // (a window of aux2 segments in total) into the event buffer
    L_NAPPLY = 4,  // apply the buffered events of noise descriptor aux, whose
                   // segments start at window segment aux2
    L_DET = 5,     // block[0..count] = list bounds relative to the block; lists
                   // of record slots; detector ids aux .. aux+count-1
    L_OBS = 6,     // as L_DET; list[0] = accumulator slot, rest = record slots
    L_OBSOUT = 7,  // block[i] = accumulator slot of observable i (count = n_obs)
    L_GAUGE = 8,   // block[3i..3i+2] = slot, op index, target: slot ^= gauge word
    L_RECOUT = 9,  // block[2i..2i+1] = slot | reference bit << 31, record index
};

// A layer's arguments are one contiguous block args[off, off + nwords) that
// the kernel stages into shared memory with a bulk asynchronous copy while
// the previous layer runs: off and nwords are multiples of 4 words (16 bytes)
// and nwords <= kStageWords. nwords = 0: nothing staged.
struct Layer {
    uint32_t kind;
    uint32_t count;
    uint32_t off;
    uint32_t nwords;
    uint32_t aux;
    uint32_t aux2;
    uint32_t seq;   // index of this layer among the staged layers (nwords > 0)
    uint32_t pad1;
};

constexpr uint32_t kStageWords = 2048;  // 8 KB per staging buffer (two buffers)
constexpr uint32_t kEvCap = 8;          // events buffered per (segment, chunk)
constexpr uint32_t kWindowSegs = 192;   // noise segments per generation window
constexpr uint32_t kWindowOps = 16;     // noise ops per generation window

enum NoiseKind : uint32_t { N_XERR = 0, N_ZERR = 1, N_DEP1 = 2, N_DEP2 = 3, N_PC1 = 4 };

// Targets of a noise op live at args[tgt_off ...]: one word per qubit,
// x slot in the low 16 bits, z slot in the high 16 bits, 0xFFFF = component
// pruned (it cannot reach any output). DEPOLARIZE2 has two words per unit.
struct NoiseDesc {
    uint32_t op_index;  // index of the op in the user's op list (RNG counter word 2)
    uint32_t kind;      // NoiseKind
    uint32_t table;     // gap-table index
    uint32_t n_units;   // targets (pairs for DEPOLARIZE2)
    uint32_t n_seg;     // ceil(n_units / 64)
    uint32_t tgt_off;   // offset into args
    uint32_t t1, t2;    // PAULI_CHANNEL_1: X if w < t1, Y if w < t2, else Z
};

constexpr uint32_t kSegUnits = 64;     // units per noise segment
constexpr uint32_t kGapLen = 4096;     // T[1..4096]: a full segment has 4096 trials
// Per probability: words [0, 4096) = T[1..4096] = floor(2^32 (1-p)^g);
// word 4096 = float bits of 1/log2(1-p) (0 for p = 1), used only to guess the
// count before the exact table check; words 4097..4099 = 0.
constexpr uint32_t kTableWords = 4100;
constexpr uint32_t kDeadSlot = 0xFFFFu;
constexpr uint32_t kMaxSlots = 0xFFFEu;

struct Program {
    std::vector<Layer> layers;
    std::vector<uint32_t> args;
    std::vector<NoiseDesc> noise;
    std::vector<uint32_t> tables;   // kTableWords per distinct p (gap table + estimate constant)
    std::vector<uint64_t> fault_base;  // per noise descriptor: index of its first single fault
    std::vector<double> table_p;
    uint32_t n_slots = 0;
    uint32_t max_window_segs = 0;  // event-buffer size in segments
    uint64_t n_faults = 0;         // single faults of the whole op list (see tmcs_fault_count)
    uint64_t n_det = 0, n_obs = 0;
};

struct SigStep;
constexpr int kSigMaxSchedules = 9;  // schedules an event-signature program carries
constexpr int kSigMaxLag = 4;        // steps in flight in a pipelined schedule

struct FlowShape {
    int sched = 0;            // barrier schedule of the signature program
    int K = 4;                // chunks per tile
    int threads = 1024;
    int appliers = 8;         // applier warps (the other warps walk)
    int window = 3;           // Philox calls per walker window (2..4)
    uint32_t arena = 0;       // event arena entries (power of two)
    bool smem_tables = false; // gap tables staged in shared memory
    size_t smem = 0;          // dynamic shared memory
    bool global_arena = false;  // arena in a global scratch buffer (one slice of `arena` entries per CTA)
    uint32_t garena_ctas = 0;   // CTAs the scratch buffer has slices for (global arena)
};

// One device copy of a program.
struct DeviceProgram {
    int device = -1;
    void *base = nullptr;  // single allocation holding everything below
    size_t bytes = 0;
    const Layer *layers = nullptr;
    const uint32_t *args = nullptr;
    const NoiseDesc *noise = nullptr;
    const uint32_t *tables = nullptr;
    const uint64_t *fault_base = nullptr;
    int tuned_mode = 0;     // launch shape chosen by the autotuner (0: not tuned)
    int tuned_K = 0;
    int tuned_warps = 0;
    int tuned_group = 0;
    int tuned_threads = 0;
    int tuned_sched = 0;    // event-signature schedule the autotuner chose
    FlowShape tuned_flow;   // mode 7: the decoupled kernel's shape
};

// One device copy of an event-signature program.
struct DeviceSig {
    int device = -1;
    void *base = nullptr;
    size_t bytes = 0;
    const NoiseDesc *noise = nullptr;
    const uint32_t *tables = nullptr;
    const uint32_t *items[kSigMaxSchedules] = {};  // item records of each schedule
    const SigStep *steps[kSigMaxSchedules] = {};
    const float *step_events[kSigMaxSchedules] = {};
    const uint32_t *item_desc[kSigMaxSchedules] = {};
    const uint32_t *ev_ent = nullptr;
};

// ------------------------------------------ decoupled event-signature kernel
//
// flow_kernel (tmcs_flow.cu): walker warps append events to a shared-memory
// arena, applier warps apply whole steps to the detector ring. Runs barrier
// schedules (lag 0) of at most kFlowMaxSteps steps.
constexpr uint32_t kFlowMaxSteps = 1024;



struct FlowCall {
    uint32_t key0 = 0, key1 = 0, first_chunk = 0;
    uint64_t n_cols = 0, last_mask = 0;
    uint64_t *det = nullptr, *obs = nullptr;
    uint32_t *status = nullptr;
    uint32_t *scratch = nullptr;  // global arena slices (FlowShape::global_arena)
    size_t scratch_bytes = 0;
};

// Per-device scratch of the library: a status word that kernels set when a
// bounded wait expires (read and cleared by tmcs_check_device).
uint32_t *device_status_word(int device);

// ------------------------------------------------- event-signature program
//
// Detector and observable flips are GF(2)-linear in the noise events, so a
// fixed circuit can also be sampled without running its Clifford layers per
// shot: every noise unit has up to four generators (X and Z on each of its
// qubits), each with the list of outputs it flips (its signature); an event
// with Pauli index k flips the XOR of the lists of the generators in k. The
// lists come from one transposed frame pass per group of 64 outputs (host),
// and the kernel walks the same noise streams as the frame program and XORs
// each event's lists into a shared-memory ring of detector words.
//
// Items are the noise segments that flip anything, in op order; steps are
// runs of items whose detectors fit in the ring (window) above the step's
// flush point. After step s, detectors [flush_lo, flush_hi) are final and are
// written out; every detector is written by exactly one step.
struct SigStep {
    uint32_t item_begin, item_end;
    uint32_t flush_lo, flush_hi;
};

constexpr uint32_t kSigObsFlag = 0x80000000u;  // entry = observable index | flag
constexpr uint32_t kEvNone = 0xFFFFFFFFu;      // empty word of an event slot
constexpr uint32_t kEvOverflow = 0x80000000u;  // event slot word 0: list in the overflow area

// One schedule of a program: its items in walk order, its steps and the
// ring size they need. Schedules differ only in the window; the output is
// the same for every one of them.
struct SigSchedule {
    // Ring size in detectors (power of two). For a barrier schedule (lag 0)
    // every step's detectors lie in [flush_lo, flush_lo + window). For a
    // pipelined schedule (lag L > 0) up to L consecutive steps, of this tile
    // and the next, run at once; the ring then holds every detector that
    // such a run of steps touches or has yet to flush.
    uint32_t window = 0;
    uint32_t lag = 0;
    std::vector<uint32_t> items;     // (descriptor, segment) pairs, 2 words per item
    // Device item records, 4 words per item: op index, segment, event slot
    // of the segment's first unit and Pauli index 1, kind | table << 3 |
    // (units - 1) << 16 | descriptor << 22 (descriptor < 1024, table < 8192).
    std::vector<uint32_t> item_rec;
    std::vector<SigStep> steps;
    // Expected events per 64-shot chunk of each step (sum over its items of
    // 64 x units x p); the decoupled kernel sizes its event regions by it.
    std::vector<float> step_events;
    // Walker descriptors of the decoupled kernel, 8 words per item (no
    // dependence on the seed): hi and lo of 0xCD9E8D57 x op index (Philox
    // round 1), segment, first event slot, kind | npauli << 3 | paulis << 7
    // | (units - 1) << 11 | step << 17, table | descriptor << 13, float bits
    // of 1/log2(1-p) (the gap estimate), and the mask of Pauli indices that
    // flip an output in some unit of the segment (bit k - 1 for index k).
    std::vector<uint32_t> item_desc;
};

struct SigProgram {
    bool ok = false;
    std::string why;                 // reason the program is unusable (ok = false)
    std::vector<NoiseDesc> noise;    // every noise op with p > 0; tgt_off = first generator id
                                     // (host); the device copy carries ev_base there
    std::vector<uint32_t> tables;    // kTableWords per distinct p
    uint32_t n_det = 0;              // detectors of the circuit
    // Barrier schedules (lag 0) by decreasing window, then pipelined ones.
    // Schedule 0 has the largest window (fewest steps) and is the one the
    // batch sampler and the statistics use.
    std::vector<SigSchedule> sched;
    std::vector<uint32_t> gen_off;   // CSR offsets per generator (n_gens + 1)
    std::vector<uint32_t> gen_ent;   // detector index, or kSigObsFlag | observable index
    // Device layout: two words per event (unit, Pauli index), in fault order
    // from the descriptor's ev_base: word 0 = first entry, kEvNone (no
    // outputs) or kEvOverflow | offset of the list in the overflow area
    // that follows the slots (then word 1 = its length); word 1 = second
    // entry or kEvNone. An entry is observable flag << 29 | output index.
    std::vector<uint32_t> ev_base;   // per descriptor: index of its first event slot
    std::vector<uint32_t> ev_ent;
    uint32_t n_event_slots = 0;      // event slots (the overflow lists follow them in ev_ent)
    double build_seconds = 0;
};

// Generators of a noise unit: DEPOLARIZE2 has X, Z on its first qubit then X,
// Z on its second; the single-qubit kinds have X, Z.
#ifdef __CUDACC__
#define TMCS_HD __host__ __device__
#else
#define TMCS_HD
#endif
TMCS_HD inline uint32_t sig_gens(uint32_t kind) { return kind == 3u ? 4u : 2u; }
// Pauli indices (events) per unit: 15 for DEPOLARIZE2, 3 for DEPOLARIZE1 and
// PAULI_CHANNEL_1, 1 for X_ERROR and Z_ERROR.
TMCS_HD inline uint32_t sig_paulis(uint32_t kind) { return kind == 3u ? 15u : (kind == 2u || kind == 4u) ? 3u : 1u; }
// Generator mask of Pauli index pk (bit 0 = X part, bit 1 = Z part per qubit).
TMCS_HD inline uint32_t sig_mask(uint32_t kind, uint32_t pk) {
    return kind == 3u ? ((pk >> 2) | ((pk & 3u) << 2)) : kind == 0u ? 1u : kind == 1u ? 2u : pk;
}

// Host-side copy of one user op.
struct HostOp {
    uint32_t code;
    double p;
    uint32_t arg;
    uint32_t toff, nt;
    uint32_t arg2;
};

}  // namespace tmcs

struct tmcs_circuit {
    uint64_t n_qubits = 0, n_meas = 0, n_det = 0, n_obs = 0;
    std::vector<tmcs::HostOp> ops;
    std::vector<uint32_t> targets;
    tmcs::Program prog;
    tmcs_stats stats{};
    // raw-measurement program, built on first use (tmcs_sample_measurements)
    tmcs::Program prog_meas;
    std::vector<uint8_t> ref_bits;
    bool meas_built = false;
    uint32_t flags = 0;
    mutable std::map<int, tmcs::DeviceProgram> dev_meas;
    // event-signature program (built with the circuit; ok = false if unusable)
    tmcs::SigProgram sig;
    mutable std::map<int, tmcs::DeviceSig> dev_sig;
    // detector error model columns, built on the first tmcs_dem_columns call
    mutable bool dem_built = false;
    mutable std::vector<uint64_t> dem_off;   // column c's entries: dem_ent[dem_off[c] .. dem_off[c+1])
    mutable std::vector<uint32_t> dem_ent;   // detector id, or 0x80000000 | observable id
    mutable std::vector<double> dem_p;       // probability that an odd number of its faults occurs
    mutable std::vector<uint64_t> dem_nf;    // single faults merged into the column
    mutable std::mutex mu;
    mutable std::map<int, tmcs::DeviceProgram> dev;
};

namespace tmcs {

// Host side (tmcs_host.cpp)
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int compile(tmcs_circuit *c, uint32_t flags, bool meas);
int reference_record(const tmcs_circuit *c, std::vector<uint8_t> *rec);
int build_measurement_program(tmcs_circuit *c);
int gap_table(double p, uint32_t *t);
int audit(const tmcs_circuit *c);
size_t program_bytes(const Program &p);
int build_signature_program(tmcs_circuit *c, uint32_t max_window);
int table_for_p(std::vector<uint32_t> &tables, std::vector<double> &table_p, double p, uint32_t *out);

// Device side (tmcs_sample.cu)
void free_device_programs(tmcs_circuit *c);

// Decoupled event-signature kernel (tmcs_flow.cu). flow_shape fills *out for
// the given schedule, chunks per tile, CTA size, applier warps and walker
// window (Philox calls per pass, 2 to 4; 0: 3; TMCS_FLOW_WINDOW overrides)
// if that shape fits `budget` bytes of dynamic shared memory.
bool flow_shape(const tmcs_circuit *c, int sched, int K, int threads, int appliers, size_t budget, FlowShape *out,
                bool global_arena = false, int window = 0);
#ifdef __CUDACC__
cudaError_t flow_launch(const SigProgram &G, uint32_t n_obs, const DeviceSig *ds, const FlowShape &s,
                        const FlowCall &call, int sms, cudaStream_t st);
#endif

}  // namespace tmcs
