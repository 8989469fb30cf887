/*
 * tmcs.h -- C ABI of libtmcs.so, a GB300 (sm_103a) Pauli-frame Monte Carlo
 * sampler for noisy Clifford circuits: detection events and logical-observable
 * flips of syndrome-extraction circuits for distributed transversal
 * operations (arXiv 2504.05611: Methods "Simulation", "Non-local CNOT
 * circuit", "State teleportation circuit", "Decoding").
 *
 * Conventions shared by every entry point
 *   - Every function returns a tmcs_status; on failure a thread-local message
 *     is available from tmcs_last_error().
 *   - Device buffers are allocated and owned by the caller; the library never
 *     frees them. Host buffers are caller-owned too.
 *   - Sampling calls are asynchronous on the given CUDA stream (cudaStream_t
 *     passed as void*; NULL = legacy default stream). The caller synchronises
 *     the stream before reading results.
 *   - Output layout (detector-major, bit-packed): for n_det detectors and S
 *     shots, C = ceil(S/64) uint64 words per detector; word c of detector j
 *     holds shots 64c .. 64c+63, bit i (LSB first) = shot 64c+i; the value is
 *     the flip of the detector parity relative to the noiseless circuit.
 *     Pad bits of the last word are 0. Observables use the same layout.
 *   - Results depend only on (circuit, seed, global 64-shot chunk index):
 *     not on tile shape, batch composition, stream or GPU.
 */
#ifndef TMCS_ABI_H_
#define TMCS_ABI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TMCS_OK = 0,
    TMCS_E_INVALID = 1,          /* bad op, target, probability, record index or argument */
    TMCS_E_NONDETERMINISTIC = 2, /* a detector/observable is random in the noiseless circuit */
    TMCS_E_OOM = 3,              /* host or device allocation failed */
    TMCS_E_CUDA = 4,             /* a CUDA runtime call failed */
    TMCS_E_TIMEOUT = 5,          /* a bounded device wait expired */
    TMCS_E_BUFFER = 6            /* output buffer too small / misaligned */
} tmcs_status;

/*
 * Opcodes (Methods "Simulation" for the noise channels; Supplementary Note 1
 * for the symplectic Pauli encoding the frames use):
 *   R, RX          reset to |0> / |+> (frame cleared)
 *   H, S           single-qubit Cliffords (frame: swap x,z / z ^= x)
 *   CX             pairs (control, target): x_t ^= x_c, z_c ^= z_t
 *   M, MX          Z / X measurement; each target appends one record
 *   X_ERROR, Z_ERROR(p)          X / Z with probability p per target
 *   DEPOLARIZE1(p)               X, Y, Z each with p/3
 *   DEPOLARIZE2(p) on pairs      each of the 15 non-identity Paulis with p/15
 *   XFEED, ZFEED   pairs (record, qubit): X / Z on qubit if the record reads 1
 *                  (classically conditioned Paulis, Methods "Simulation")
 *   DETECTOR       XOR of the listed absolute record indices
 *   OBSERVABLE     XOR of the listed records into observable `arg`
 *   TICK           layer hint, no effect
 *   PAULI_CHANNEL_1 X, Y or Z with probabilities px, py, pz (Methods
 *                  "Decoherence"): p = px + py + pz; an event's Pauli is X if
 *                  its 32-bit Pauli word w < arg, Y if w < arg2, else Z, with
 *                  arg = floor(2^32 px / p), arg2 = floor(2^32 (px+py) / p)
 */
typedef enum {
    TMCS_R = 0, TMCS_RX, TMCS_H, TMCS_S, TMCS_CX, TMCS_M, TMCS_MX,
    TMCS_X_ERROR, TMCS_Z_ERROR, TMCS_DEPOLARIZE1, TMCS_DEPOLARIZE2,
    TMCS_XFEED, TMCS_ZFEED, TMCS_DETECTOR, TMCS_OBSERVABLE, TMCS_TICK,
    TMCS_PAULI_CHANNEL_1
} tmcs_opcode;

/* One instruction. `targets` points at n_targets uint32 (host memory, read
 * during tmcs_circuit_build only). `p` is used by the noise opcodes, `arg` by
 * OBSERVABLE (observable id) and PAULI_CHANNEL_1, `arg2` by PAULI_CHANNEL_1
 * only (must be 0 for every other opcode). 32 bytes on LP64. */
typedef struct {
    uint32_t code;
    uint32_t n_targets;
    double p;
    uint32_t arg;
    uint32_t arg2;
    const uint32_t *targets;
} tmcs_op;

typedef struct tmcs_circuit tmcs_circuit; /* opaque; owned by the library */

/* tmcs_circuit_build flags */
#define TMCS_FLAG_NO_AUDIT 0x1u   /* skip the determinism audit */
#define TMCS_FLAG_NO_PRUNE 0x2u   /* keep frame components that cannot reach an output */

/*
 * Validate and compile an op list (host only; no CUDA call).
 * Defining passages: the op list is the noisy circuit of Methods
 * "Simulation" (reset flips, 1- and 2-qubit depolarizing after gates,
 * measurement flips, depolarized ebit pairs, classically conditioned
 * operations) built for the protocols of Methods "Non-local CNOT circuit" and
 * "State teleportation circuit" (Fig. 1b, c); its DETECTOR and OBSERVABLE
 * ops are the rows and logical observables of Methods "Decoding".
 * Compiles to a straight-line program over frame-component slots: liveness
 * pruning drops every x/z component that cannot reach a detector or
 * observable, components get shared-memory slots by interval allocation, and
 * independent updates are grouped into layers. Unless TMCS_FLAG_NO_AUDIT is
 * set, a 64-lane gauge-randomised noiseless run checks that every detector and
 * observable is deterministic (TMCS_E_NONDETERMINISTIC otherwise).
 * On success *out owns the compiled circuit; free it with tmcs_circuit_free.
 * Errors: TMCS_E_INVALID (bad opcode, odd pair list, qubit/record index out of
 * range, p outside [0,1] or in (0, 1e-12), arg2 != 0 outside PAULI_CHANNEL_1,
 * PAULI_CHANNEL_1 thresholds with arg > arg2), TMCS_E_OOM.
 */
int tmcs_circuit_build(const tmcs_op *ops, size_t n_ops, uint32_t flags, tmcs_circuit **out);

/* Release a circuit and its device copies (all devices it was uploaded to).
 * The caller must ensure no sampling call using it is still in flight. */
int tmcs_circuit_free(tmcs_circuit *c);

/* Sizes of a compiled circuit; any pointer may be NULL. device_bytes is the
 * size of the compiled program one device copy occupies. */
int tmcs_circuit_info(const tmcs_circuit *c, uint64_t *n_qubits, uint64_t *n_meas,
                      uint64_t *n_det, uint64_t *n_obs, uint64_t *device_bytes);

/* Compiler statistics of a circuit (for tuning and reports). */
typedef struct {
    uint64_t n_layers;        /* synchronised layers of the device program */
    uint64_t n_slots;         /* frame-component slots (64 shots x 8 bytes each per chunk) */
    uint64_t n_xor;           /* slot XOR updates (gates, feeds) after pruning */
    uint64_t n_zero;          /* slot clears */
    uint64_t n_copy;          /* slot copies */
    uint64_t n_noise_ops;     /* noise ops with at least one live component */
    uint64_t n_noise_units;   /* noise targets (pairs) of those ops */
    uint64_t n_noise_segments;/* 64-unit segments of those ops */
    uint64_t n_parity_terms;  /* record reads of detectors and observables */
    uint64_t live_components; /* x/z components kept by pruning (of 2 * updates) */
    uint64_t pruned_updates;  /* slot updates removed by pruning */
    /* event-signature program (see tmcs_fault_outputs) */
    uint64_t sig_ok;          /* 1 if the signature sampler can run this circuit */
    uint64_t sig_window;      /* detector ring size of the main schedule (words per chunk) */
    uint64_t sig_steps;       /* flush steps of the main schedule */
    uint64_t sig_items;       /* noise segments walked per chunk */
    uint64_t sig_generators;  /* X/Z generators of all noise units */
    uint64_t sig_entries;     /* (generator, output) pairs */
    uint64_t sig_build_us;    /* host time to build it, microseconds */
    uint64_t sig_max_step_items; /* segments in the largest step */
    uint64_t sig_schedules;   /* barrier schedules carried (ring window halves each time) */
    uint64_t sig_min_window;  /* ring size of the smallest barrier schedule */
    uint64_t sig_pipe_schedules; /* pipelined schedules carried (several steps in flight) */
} tmcs_stats;
int tmcs_circuit_stats(const tmcs_circuit *c, tmcs_stats *out);

/*
 * Noiseless reference measurement record on the host (CHP stabilizer
 * tableau, Aaronson & Gottesman 2004); a random outcome resolves to 0.
 * meas_bits: host, ceil(n_meas/8) bytes, bit i of byte b = record 8b+i.
 * O(n_qubits^2) memory and time per measurement; not on the sampling path.
 */
int tmcs_reference_sample(const tmcs_circuit *c, uint8_t *meas_bits);

/*
 * Sample `shots` shots with global 64-shot chunks 0 .. ceil(shots/64)-1.
 * Defining passages: the Monte Carlo sampling of the noisy circuit in
 * Methods "Simulation" (each shot runs the circuit with independently drawn
 * noise), producing per shot the syndrome vector of detector values and the
 * logical-observable flips that Methods "Decoding" hands to the decoder.
 * detector_bits:   device, n_det * ceil(shots/64) uint64, 8-byte aligned
 * observable_bits: device, n_obs * ceil(shots/64) uint64 (may be NULL if n_obs == 0)
 * Asynchronous on `stream`, with two one-time exceptions per circuit and
 * device: the first call uploads the compiled programs (synchronously, before
 * the launch), and the first call with at least 16 chunks per SM times the
 * candidate launch shapes on the leading columns of its own output
 * (synchronously; skipped while `stream` is being captured) and keeps the
 * fastest. Make such a call before capturing a graph or timing steps.
 * Kernel choice: the event-signature sampler when the circuit has a usable
 * event-signature program (tmcs_circuit_stats sig_ok), else the frame
 * kernels; both give the same bits. Tuning knobs in the environment change
 * only the schedule: TMCS_KERNEL (3 CTA frame kernel, 4 warp-group frame
 * kernel, 5 event-signature kernel, 6 pipelined event-signature kernel,
 * 7 decoupled event-signature kernel: walker warps append events to a
 * shared-memory arena, applier warps apply whole steps), TMCS_TILE_K,
 * TMCS_THREADS, TMCS_SIG_SCHED (signature schedule index), TMCS_FLOW_APPLIERS
 * and TMCS_FLOW_ARENA (kernel 7: applier warps, arena entries),
 * TMCS_FLOW_WINDOW (kernel 7: Philox calls per walker pass, 2 to 4),
 * TMCS_FLOW_GLOBAL_ARENA=1 and TMCS_FLOW_GARENA (kernel 7: the arena in a
 * per-stream global scratch buffer, its entries per CTA), TMCS_FLOW_TMA
 * and TMCS_FLOW_TMA_ROWS (kernel 7 with 8 or more chunks per tile, or any
 * even number with TMCS_FLOW_TMA=1, writes finished detector rows as 2D
 * tensor stores, boxes of that many rows (default 64) by the tile's chunks,
 * when detector_bits is 16-byte aligned and ceil(shots/64) is even;
 * TMCS_FLOW_TMA=0 never; other outputs take plain stores),
 * TMCS_SIG_WINDOW (read by tmcs_circuit_build), TMCS_AUTOTUNE=0.
 * Testing: TMCS_TEST_STALL_FLUSH=1 makes the pipelined kernel's flusher wait
 * for a stream count that never arrives, so its bounded wait (2 s) expires,
 * every warp leaves and tmcs_check_device reports TMCS_E_TIMEOUT.
 * TMCS_TEST_FLOW_CAP=n gives every step of kernel 7 an arena region of n
 * events, so most events take its overflow path (same bits);
 * TMCS_TEST_FLOW_SLICE_TILES=n splits a kernel-7 call into launches of n
 * tiles (the path huge calls take to keep 32-bit stream counters).
 * Errors: TMCS_E_INVALID (NULL circuit/buffer, shots == 0), TMCS_E_CUDA,
 * TMCS_E_OOM (program upload).
 */
int tmcs_sample(const tmcs_circuit *c, uint64_t shots, uint64_t seed,
                uint64_t *detector_bits, uint64_t *observable_bits, void *stream);

/*
 * Resumable / shardable form: shots 64*first_chunk .. 64*first_chunk+shots-1
 * (Methods "Simulation": the paper spreads the shots of one circuit over
 * hundreds to thousands of CPU cores with MPI; a chunk range is that unit of
 * independent work, here one per GPU or per call)
 * of the stream defined by `seed`. Outputs have ceil(shots/64) words per
 * detector; word j is global chunk first_chunk + j. Concatenating the outputs
 * of disjoint ranges reproduces one tmcs_sample call bit for bit.
 * first_chunk + ceil(shots/64) must not exceed 2^32.
 */
int tmcs_sample_range(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                      uint64_t *detector_bits, uint64_t *observable_bits, void *stream);

/*
 * Allocation-free form of tmcs_sample_range (no counterpart in the paper; a
 * service entry point of this library). For callers that cannot allocate
 * device memory while running -- a service whose device memory belongs to
 * another allocator's pool, a real-time host that forbids allocation on its
 * request path, code that must not let cudaMalloc/cudaFree synchronise the
 * device -- it calls no cudaMalloc, cudaFree or other allocating routine.
 * Its scratch is one file-scope device array of 8 MiB (every GPU that loads
 * libtmcs.so holds it until the process exits): a status word (256 bytes)
 * followed by the circuit's compiled frame program, which each call copies
 * into it (stream-ordered on `stream`) before launching a frame kernel on it.
 * Every sampling kernel draws the same noise streams, so outputs are
 * bit-identical to tmcs_sample_range with the same arguments, whichever
 * kernel that call uses.
 *   - Circuits whose compiled program exceeds the array (device_bytes of
 *     tmcs_circuit_info plus 256) are rejected with TMCS_E_INVALID.
 *   - The first call on each device looks up the array's device address with
 *     that device current and clears the status word (synchronously); make
 *     that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents: calls
 *     that overlap on the GPU (other streams, other host threads) race; the
 *     caller must serialise them (e.g. one stream).
 *   - Launch shape: the frame kernels' heuristic, or the knobs TMCS_KERNEL=3/4,
 *     TMCS_TILE_K, TMCS_THREADS, TMCS_WARPS, TMCS_GROUP; no timing.
 *   - A device-side bounded wait that expires sets the array's status word,
 *     which stays set until tmcs_check_device reports TMCS_E_TIMEOUT and
 *     clears it. Testing: TMCS_TEST_NOALLOC_EXPIRED=1 sets that word as an
 *     expired wait would.
 * Arguments and errors as tmcs_sample_range.
 */
int tmcs_sample_noalloc(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                        uint64_t *detector_bits, uint64_t *observable_bits, void *stream);

/*
 * Detector error model by single-fault injection (Methods "Decoding": one
 * detector-error-model column per distinct error mechanism). Faults are
 * enumerated over the op list: every noise op with p > 0 in order, every
 * target unit (pair for DEPOLARIZE2), Pauli index k = 1..K (K = 1 for
 * X_ERROR/Z_ERROR, 3 for DEPOLARIZE1/PAULI_CHANNEL_1 with 1=X, 2=Z, 3=Y, 15
 * for DEPOLARIZE2 with k>>2 on the first and k&3 on the second target).
 * tmcs_fault_count gives the number of faults.
 * tmcs_fault_signatures propagates faults first_fault .. first_fault+n_faults-1
 * through the noiseless circuit, one fault per lane, with the sampling
 * kernels: lane l of word c of detector j (layout of tmcs_sample with
 * ceil(n_faults/64) words per detector) says whether fault first_fault+64c+l
 * flips detector j; observables likewise. first_fault must be a multiple of
 * 64. Errors: TMCS_E_INVALID (range), as tmcs_sample otherwise.
 */
int tmcs_fault_count(const tmcs_circuit *c, uint64_t *n_faults);

/*
 * Outputs flipped by elementary fault `fault` (enumeration of
 * tmcs_fault_count), read from the event table the signature samplers apply:
 * detector indices, then 0x80000000 | observable index, ascending. The table
 * holds, per event (noise unit and Pauli index, in fault order), the outputs
 * it flips (a DEM column, Methods "Decoding"): the XOR of the lists of X and
 * Z on each of its qubits, found by running the transposed frame maps
 * backwards over the op list.
 * out: host, cap entries; *n_out = number of outputs (may exceed cap, then
 * only cap are written). Errors: TMCS_E_INVALID (fault out of range, no
 * table: sig_ok = 0 in tmcs_circuit_stats).
 */
int tmcs_fault_outputs(const tmcs_circuit *c, uint64_t fault, uint32_t *out, uint32_t cap, uint32_t *n_out);

/*
 * Detector error model columns (Methods "Decoding": the parity-check matrix
 * derived from the detector error model has one row per detector and one
 * column per distinct error mechanism, a fault class that flips one or more
 * detectors and possibly observables; Table III "cols" counts them). Single
 * faults are enumerated as in tmcs_fault_count and read from the same
 * event-signature table the samplers apply (tmcs_fault_outputs); faults with
 * equal non-empty signatures merge into one column. Host only (no CUDA
 * call); built on the first call and kept with the circuit.
 *   n_cols, n_entries: in/out. Call with every array NULL to get the sizes;
 *     then pass arrays of at least those sizes (their capacities in *n_cols,
 *     *n_entries; TMCS_E_BUFFER if smaller).
 *   col_off:    n_cols + 1 uint64: column c's entries are
 *               entries[col_off[c] .. col_off[c+1]), sorted ascending
 *   entries:    detector id, or 0x80000000 | observable id
 *   col_p:      n_cols doubles: probability that an odd number of the
 *               column's faults occur in one shot (faults of one noise unit
 *               are mutually exclusive, units independent:
 *               (1 - prod_u (1 - 2 P_u)) / 2 with P_u the unit's share)
 *   col_faults: n_cols uint64: single faults merged into the column
 * Columns come in ascending order of their entry lists. Any of the four
 * arrays may be NULL. Errors: TMCS_E_INVALID (NULL circuit or sizes, no
 * event-signature program: tmcs_circuit_stats sig_ok = 0), TMCS_E_BUFFER,
 * TMCS_E_OOM.
 */
int tmcs_dem_columns(const tmcs_circuit *c, uint64_t *n_cols, uint64_t *n_entries, uint64_t *col_off,
                     uint32_t *entries, double *col_p, uint64_t *col_faults);

/*
 * Raw measurement records of noisy executions (Methods "Decoding": detector
 * values are parities of the measurement outcomes of one noisy run; this
 * returns the outcomes themselves). Shots 64*first_chunk .. +shots-1 of the
 * stream `seed`: the noise draws are those of tmcs_sample_range with the same
 * arguments, so every detector parity of these records, XORed with its value
 * on the reference record (tmcs_reference_sample), equals that call's
 * detector bit. Record i of a shot is reference bit XOR frame flip, where the
 * frame also carries a random gauge Pauli after every reset and measurement
 * (Z after R/M, X after RX/MX, Z on every qubit at the start): that leaves
 * the state unchanged but turns each non-deterministic outcome into a fair
 * coin. Gauge word of (op i, target u, chunk c): Philox4x32-10 with the
 * sampling key at counter (u/2, c, i, 2^31), words 0|1<<32 for even u, 2|3<<32
 * for odd u; the start uses op index n_ops and u = qubit.
 * meas_bits: device, n_meas * ceil(shots/64) uint64, 8-byte aligned; word j of
 * row i holds record i of shots 64(first_chunk+j) .. +63, bits past `shots` 0.
 * The first call per circuit builds a second compiled program on the host
 * (reference tableau run plus compile) and uploads it; asynchronous after
 * that. Errors: as tmcs_sample_range.
 */
int tmcs_sample_measurements(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                             uint64_t *meas_bits, void *stream);
int tmcs_fault_signatures(const tmcs_circuit *c, uint64_t first_fault, uint64_t n_faults, uint64_t *detector_bits,
                          uint64_t *observable_bits, void *stream);

/* One job of a batched launch: circuit, shots (from chunk 0), seed, outputs. */
typedef struct {
    const tmcs_circuit *c;
    uint64_t shots;
    uint64_t seed;
    uint64_t *det;
    uint64_t *obs;
} tmcs_job;

/*
 * Defining passages: the paper's results are sweeps of many circuits -- codes,
 * distances, rounds and physical error rates (Results "Distributed
 * operations thresholds and scaling", Methods "Simulation" and
 * "Statistics": each point needs enough shots to see logical errors) -- each
 * sampled as in tmcs_sample. This call samples such a set of jobs together.
 * Sample many circuits of uneven size on `stream`: the jobs share persistent
 * launches whose resident CTAs pull (job, tile) work items from a device
 * queue; a job that fills the GPU by itself (at least 16 chunks per SM) with
 * an event-signature program instead runs as its own tmcs_sample call, with
 * the launch shape tuned for its circuit (that call may tune synchronously,
 * as tmcs_sample does, unless the stream is being captured). Each job's
 * output equals its own tmcs_sample call bit for bit.
 * Errors: as tmcs_sample; TMCS_E_INVALID if any job is invalid.
 */
int tmcs_batch_sample(const tmcs_job *jobs, size_t n_jobs, void *stream);

/*
 * Synchronous device-side error check for the current device: returns
 * TMCS_E_TIMEOUT (and clears the flags) if any sampling kernel since the last
 * check gave up on a bounded wait (its outputs are then incomplete), else
 * TMCS_OK. It reads the library's per-device status word and, once
 * tmcs_sample_noalloc has run on the device, that entry point's status word
 * too. Blocks until prior work on the device's legacy stream is done. This
 * call stands in for a per-stream status query: the status words are per
 * device, so one check covers every stream.
 */
int tmcs_check_device(void);

/*
 * The launch shape the autotuner chose for this circuit on the current
 * device (for reports): *mode = 0 if it has not run yet (first large call),
 * 3 = CTA-wide frame kernel, 4 = warp-group frame kernel, 5 = event-signature
 * kernel, 6 = pipelined event-signature kernel, 7 = decoupled
 * event-signature kernel; *chunks = 64-shot chunks per CTA (modes 3, 5, 6,
 * 7) or per warp group (mode 4); *threads = CTA size; *ring_window =
 * detector ring of the chosen event-signature schedule (modes 5, 6, 7; 0
 * otherwise). Any pointer may be NULL.
 * Errors: TMCS_E_INVALID (NULL circuit), TMCS_E_CUDA (no current device).
 */
int tmcs_launch_shape(const tmcs_circuit *c, int *mode, int *chunks, int *threads, int *ring_window);

/*
 * The decoupled kernel's part of the chosen shape (mode 7; zeros otherwise):
 * applier warps, Philox calls per walker window, whether the event arena is
 * in global memory, and the arena's entries (per CTA). Together with
 * tmcs_launch_shape this fixes the launch (for reports and for forcing the
 * same shape with the tuning knobs). Any pointer may be NULL.
 * Errors: as tmcs_launch_shape.
 */
int tmcs_launch_flow_shape(const tmcs_circuit *c, int *appliers, int *window, int *global_arena, int *arena_entries);

/*
 * Measured non-HBM ceilings of the current device, for roofline reports (the
 * samplers do GF(2) bit work, so besides HBM their co-bounds are the shared
 * memory pipe and the integer pipe). Three compute-only microbenchmarks on
 * every SM: conflict-free 32-bit shared loads (one 128-byte wavefront per
 * warp-wide load), 32-bit shared atomic XORs, and chains of lop3.b32.
 * Synchronous; allocates and frees a small result buffer; about 0.1 s.
 * Errors: TMCS_E_INVALID (NULL), TMCS_E_OOM, TMCS_E_CUDA.
 */
typedef struct {
    double smem_load_bytes_per_s;      /* conflict-free shared loads, whole device */
    double smem_load_wavefronts_per_s;
    double smem_atomic_lanes_per_s;    /* 32-bit shared atomics, lanes per second */
    double lop3_lanes_per_s;           /* lop3.b32 per lane per second */
    double lop3_warp_inst_per_s;
    double sm_clock_mhz;               /* device attribute (not the live clock) */
    int sms;
} tmcs_peaks;
int tmcs_measure_peaks(tmcs_peaks *out);

/*
 * Sampling server (continuous batching). A host scheduler thread admits
 * submitted requests in arrival order as soon as their output words fit in a
 * device arena (admission by HBM footprint), cuts every admitted request into
 * slices of 64-shot chunks and issues slices round-robin over all admitted
 * requests on n_streams CUDA streams, so a request that arrives while others
 * run starts on the next free stream and its work overlaps theirs on the
 * GPU. Each slice is one tmcs_sample_range call, so every request's output is
 * bit-identical to a solo tmcs_sample of the same circuit, shots and seed.
 * Circuits stay device-resident (uploaded on first use) and must outlive their
 * requests. All functions are thread-safe; the server uses the device that is
 * current when it is opened.
 */
typedef struct tmcs_server tmcs_server;

typedef struct {
    uint32_t n_streams;         /* concurrent streams (0: 4) */
    uint32_t slice_chunks;      /* 64-shot chunks per slice (0: 4096) */
    uint64_t arena_bytes;       /* device bytes for outputs of admitted requests
                                   (0: half of the free device memory) */
} tmcs_server_config;

typedef struct {
    uint64_t submitted, completed, failed, queued, running;
    uint64_t arena_bytes, arena_in_use;
    double latency_p50_s, latency_p99_s, latency_mean_s; /* submit -> all slices done */
    double busy_seconds;        /* wall time with at least one request admitted */
    uint64_t shots_done;
} tmcs_server_stats;

enum { TMCS_REQ_QUEUED = 0, TMCS_REQ_RUNNING = 1, TMCS_REQ_DONE = 2, TMCS_REQ_FAILED = 3 };

/* Open a server on the current device (allocates the arena, starts the
 * scheduler thread). Errors: TMCS_E_OOM, TMCS_E_CUDA. */
int tmcs_server_open(const tmcs_server_config *cfg, tmcs_server **out);
/* Queue one request; *request_id identifies it. Fails with TMCS_E_BUFFER if
 * its outputs, (n_det + n_obs) * ceil(shots/64) * 8 bytes, exceed the arena. */
int tmcs_server_submit(tmcs_server *srv, const tmcs_circuit *c, uint64_t shots, uint64_t seed,
                       uint64_t *request_id);
/* State of a request (TMCS_REQ_*). */
int tmcs_server_poll(tmcs_server *srv, uint64_t request_id, int *state);
/* Wait for a request, copy its outputs to host memory in the tmcs_sample
 * layout (host_det: n_det * ceil(shots/64) words, host_obs: n_obs * ... ;
 * either may be NULL to skip), then release its arena space. */
int tmcs_server_fetch(tmcs_server *srv, uint64_t request_id, uint64_t *host_det, uint64_t *host_obs);
/* Wait for a request and release it without copying its outputs. */
int tmcs_server_release(tmcs_server *srv, uint64_t request_id);
int tmcs_server_get_stats(tmcs_server *srv, tmcs_server_stats *out);
/* Stop the scheduler (after in-flight slices finish) and free the arena. */
int tmcs_server_close(tmcs_server *srv);

/* Thread-local description of the last error of this thread ("" if none). */
const char *tmcs_last_error(void);

/*
 * Gap table of the sampling specification for probability p in (0, 1]:
 * table[g-1] = T[g] = floor(2^32 (1-p)^g), g = 1..4096, with (1-p)^g computed
 * as exp(g * log1p(-p)) in double precision. The gap between noise events is
 * G = #{g : w < T[g]} for a uniform 32-bit word w. Exported so tests can
 * compare it with an independent computation.
 */
int tmcs_debug_gap_table(double p, uint32_t *table);

/*
 * Gap counts G = #{g in 1..4096 : w < T[g]} of the table above for n words,
 * computed on the current device by the routines the sampling kernels use:
 * method 0 as the decoupled kernel's walkers count (one table read guided by
 * a float estimate when |1/log2(1-p)| < 32768, else method 1), 1 the
 * two-read count with neighbour walks, 2 the log estimate with neighbour
 * loops (kernels 3 to 6 count as method 0 does where one read is allowed,
 * else by method 2). words and counts are device pointers to n uint32
 * and n int32. Blocks until done (on `stream`). Exported so tests can check
 * every route against the definition, words at the table's boundaries
 * included. Errors: TMCS_E_INVALID (NULL pointer, p outside (0, 1], bad
 * method), TMCS_E_CUDA.
 */
int tmcs_debug_gap_counts(double p, const uint32_t *words, uint64_t n, int32_t *counts, int method, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TMCS_ABI_H_ */
