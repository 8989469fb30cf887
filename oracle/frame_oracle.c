/*
 * CPU oracle for the Pauli-frame sampler -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this file's library. The CUDA sampler shares no code with it.
 *
 * What it computes (arXiv 2504.05611, Methods "Simulation"; Supplementary
 * Note 1 for the symplectic (x, z) encoding of Paulis):
 *   one shot at a time, a Pauli frame (x[q], z[q]) in {0,1} per qubit is
 *   pushed through the op list; Clifford gates conjugate it (H swaps x and z,
 *   S sets z ^= x, CX c->t sets x_t ^= x_c and z_c ^= z_t), resets clear it,
 *   M records x (MX records z) as the flip of that measurement relative to
 *   the noiseless reference, conditioned Paulis XOR a record into x or z, and
 *   noise channels XOR sampled Paulis in. Detectors and observables are
 *   XORs of record flips.
 *
 * The random process (this project's sampling specification; the paper
 * samples with a third-party simulator and fixes no generator):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed low 32,
 *   seed high 32), counter = (j, chunk, op index, segment) for call j of the
 *   noise stream of one segment of one noise op in one 64-shot chunk. Call j
 *   yields words (w0, w1, w2, w3) = draws 2j (gap w0, Pauli w1) and 2j+1
 *   (gap w2, Pauli w3).
 *   A noise op with T units (targets; pairs for DEPOLARIZE2) has segments of
 *   64 units; segment s spans trials t = 64*u_local + lane, u_local < U_s.
 *   Walk: pos = -1; per draw, pos += 1 + G, stop when pos >= 64*U_s, else an
 *   event hits unit 64*s + pos/64 in lane pos%64 with Pauli index
 *   k = 1 + ((w_pauli * K) >> 32), K = 1, 3, 15 for *_ERROR, DEPOLARIZE1, 2.
 *   G = #{g in 1..4096 : w_gap < T[g]} with T[g] = floor(2^32 (1-p)^g),
 *   (1-p)^g evaluated as exp(g * log1p(-p)); so G is geometric with success
 *   probability p on every position a segment can reach (G is capped at
 *   4096, the trial count of a full segment).
 *   Pauli index bits: x = bit 0, z = bit 1 (X=1, Z=2, Y=3); DEPOLARIZE2 puts
 *   k>>2 on the first target and k&3 on the second. PAULI_CHANNEL_1 (event
 *   probability p = px + py + pz, Methods "Decoherence") picks X if
 *   w_pauli < t1, Y if w_pauli < t2, else Z, with t1 = floor(2^32 px / p),
 *   t2 = floor(2^32 (px + py) / p); the oracle derives p, t1 and t2 from
 *   (px, py, pz) itself (oracle_pauli_channel).
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC -pthread (see oracle/build.py).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Opcode numbering private to the oracle. */
enum {
    OR_R = 0, OR_RX, OR_H, OR_S, OR_CX, OR_M, OR_MX,
    OR_X_ERROR, OR_Z_ERROR, OR_DEP1, OR_DEP2,
    OR_XFEED, OR_ZFEED, OR_DETECTOR, OR_OBSERVABLE, OR_TICK,
    OR_PC1, /* PAULI_CHANNEL_1 */
    OR_N_CODES
};

#define SEG_UNITS 64
#define GAP_LEN 4096

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds: multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
 * increments 0x9E3779B9 / 0xBB67AE85; the key is bumped before every round
 * after the first. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* --------------------------------------------------------- gap tables */

static uint32_t to_u32_fraction(double x)
{
    /* floor(2^32 * x) clamped to [0, 2^32 - 1] */
    double v = floor(ldexp(x, 32));
    if (!(v > 0.0)) return 0u;
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)v;
}

/* PAULI_CHANNEL_1(px, py, pz) (Methods "Decoherence": X and Y with the
 * amplitude-damping share, Z with the dephasing share of an aged ebit): an
 * event happens with probability p = px + py + pz (a sum up to 1e-12 above 1
 * is rounding and is taken as 1); given an event, the uniform Pauli word w
 * of the sampling specification picks X when w < t1, Y when t1 <= w < t2
 * and Z otherwise, with t1 = floor(2^32 px / p) and t2 = floor(2^32 (px + py)
 * / p), so that X, Y, Z occur with probabilities px/p, py/p, pz/p up to
 * 2^-32. Returns -1 for probabilities outside [0, 1] or summing above 1. */
int oracle_pauli_channel(double px, double py, double pz, double *p, uint32_t *t1, uint32_t *t2)
{
    if (!(px >= 0.0 && px <= 1.0 && py >= 0.0 && py <= 1.0 && pz >= 0.0 && pz <= 1.0)) return -1;
    double sum = px + py + pz;
    if (sum > 1.0 + 1e-12) return -1;
    if (sum > 1.0) sum = 1.0;
    *p = sum;
    if (sum == 0.0) {
        *t1 = 0u;
        *t2 = 0u;
        return 0;
    }
    *t1 = to_u32_fraction(px / sum);
    *t2 = to_u32_fraction((px + py) / sum);
    return 0;
}

/* t[0..4095] hold T[1..4096] = floor(2^32 (1-p)^g). p must be in (0, 1]. */
void oracle_gap_table(double p, uint32_t *t)
{
    double lq = log1p(-p);
    for (int g = 1; g <= GAP_LEN; g++)
        t[g - 1] = to_u32_fraction(exp((double)g * lq));
}

/* ---------------------------------------------------------- op access */

typedef struct {
    int64_t n_ops;
    const int32_t *codes;
    const double *ps;
    const uint32_t *args;
    const uint32_t *args2; /* PAULI_CHANNEL_1 second threshold */
    const int64_t *toff; /* n_ops + 1 */
    const uint32_t *targets;
    int64_t n_qubits, n_meas, n_det, n_obs;
} oracle_circuit;

typedef struct {
    uint32_t t[GAP_LEN];
} gap_table;

static int is_noise(int code)
{
    return code == OR_X_ERROR || code == OR_Z_ERROR || code == OR_DEP1 || code == OR_DEP2 || code == OR_PC1;
}

/* #{i : w < t[i]} for a non-increasing table (checked when it is built):
 * the entries with w < t[i] form a prefix, found by bisection. */
static uint32_t count_below(uint32_t w, const uint32_t *t, int len)
{
    int lo = 0, hi = len; /* answer in [lo, hi] */
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (w < t[mid]) lo = mid + 1;
        else hi = mid;
    }
    return (uint32_t)lo;
}

/* ------------------------------------------------- one-shot sampler */

typedef struct {
    const oracle_circuit *c;
    const gap_table *const *tables; /* per op: table of its p (noise ops only) */
    uint64_t seed, first_chunk, shots;
    uint64_t col_begin, col_end; /* output columns (chunks) this worker owns */
    uint64_t n_cols;
    uint64_t *det, *obs;
    int status;
} shot_job;

static void apply_pauli(uint8_t *x, uint8_t *z, uint32_t q, uint32_t pauli)
{
    x[q] ^= (uint8_t)(pauli & 1u);
    z[q] ^= (uint8_t)((pauli >> 1) & 1u);
}

/* Run the noise streams of op `i` for chunk `chunk` and apply the events that
 * land in `lane`. Every segment's stream is walked from its start. */
static void noise_op_one_lane(const oracle_circuit *c, const gap_table *tab, int64_t i,
                              uint64_t seed, uint32_t chunk, uint32_t lane,
                              uint8_t *x, uint8_t *z)
{
    int code = c->codes[i];
    const uint32_t *t = c->targets + c->toff[i];
    int64_t nt = c->toff[i + 1] - c->toff[i];
    int64_t units = (code == OR_DEP2) ? nt / 2 : nt;
    uint32_t K = (code == OR_DEP2) ? 15u : (code == OR_DEP1) ? 3u : 1u;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t nseg = (units + SEG_UNITS - 1) / SEG_UNITS;
    for (int64_t s = 0; s < nseg; s++) {
        int64_t u_seg = units - s * SEG_UNITS;
        if (u_seg > SEG_UNITS) u_seg = SEG_UNITS;
        int64_t n_trials = 64 * u_seg;
        int64_t pos = -1;
        for (uint32_t d = 0;; d++) {
            uint32_t ctr[4] = {d / 2, chunk, (uint32_t)i, (uint32_t)s};
            uint32_t w[4];
            oracle_philox4x32_10(ctr, key, w);
            uint32_t w_gap = (d & 1) ? w[2] : w[0];
            uint32_t w_pauli = (d & 1) ? w[3] : w[1];
            int64_t G = count_below(w_gap, tab->t, GAP_LEN);
            pos += 1 + G;
            if (pos >= n_trials) break;
            if ((uint32_t)(pos & 63) != lane) continue;
            int64_t u = s * SEG_UNITS + (pos >> 6);
            uint32_t k = 1u + (uint32_t)(((uint64_t)w_pauli * (uint64_t)K) >> 32);
            switch (code) {
            case OR_X_ERROR: apply_pauli(x, z, t[u], 1u); break;
            case OR_Z_ERROR: apply_pauli(x, z, t[u], 2u); break;
            case OR_DEP1: apply_pauli(x, z, t[u], k); break;
            case OR_DEP2:
                apply_pauli(x, z, t[2 * u], k >> 2);
                apply_pauli(x, z, t[2 * u + 1], k & 3u);
                break;
            case OR_PC1: {
                uint32_t pauli = (w_pauli < c->args[i]) ? 1u : (w_pauli < c->args2[i]) ? 3u : 2u;
                apply_pauli(x, z, t[u], pauli);
                break;
            }
            }
        }
    }
}

static void *shot_worker(void *arg)
{
    shot_job *job = (shot_job *)arg;
    const oracle_circuit *c = job->c;
    uint8_t *x = calloc((size_t)c->n_qubits + 1, 1);
    uint8_t *z = calloc((size_t)c->n_qubits + 1, 1);
    uint8_t *rec = calloc((size_t)c->n_meas + 1, 1);
    uint8_t *obs = calloc((size_t)c->n_obs + 1, 1);
    if (!x || !z || !rec || !obs) {
        job->status = -2;
        free(x); free(z); free(rec); free(obs);
        return NULL;
    }
    for (uint64_t col = job->col_begin; col < job->col_end; col++) {
        uint32_t chunk = (uint32_t)(job->first_chunk + col);
        for (uint32_t lane = 0; lane < 64; lane++) {
            uint64_t shot = col * 64 + lane;
            if (shot >= job->shots) break;
            memset(x, 0, (size_t)c->n_qubits);
            memset(z, 0, (size_t)c->n_qubits);
            memset(obs, 0, (size_t)c->n_obs);
            int64_t m = 0, d = 0;
            for (int64_t i = 0; i < c->n_ops; i++) {
                int code = c->codes[i];
                const uint32_t *t = c->targets + c->toff[i];
                int64_t nt = c->toff[i + 1] - c->toff[i];
                switch (code) {
                case OR_R:
                case OR_RX:
                    for (int64_t a = 0; a < nt; a++) { x[t[a]] = 0; z[t[a]] = 0; }
                    break;
                case OR_H:
                    for (int64_t a = 0; a < nt; a++) { uint8_t v = x[t[a]]; x[t[a]] = z[t[a]]; z[t[a]] = v; }
                    break;
                case OR_S:
                    for (int64_t a = 0; a < nt; a++) z[t[a]] ^= x[t[a]];
                    break;
                case OR_CX:
                    for (int64_t a = 0; a + 1 < nt; a += 2) {
                        uint32_t cq = t[a], tq = t[a + 1];
                        x[tq] ^= x[cq];
                        z[cq] ^= z[tq];
                    }
                    break;
                case OR_M:
                    for (int64_t a = 0; a < nt; a++) rec[m++] = x[t[a]];
                    break;
                case OR_MX:
                    for (int64_t a = 0; a < nt; a++) rec[m++] = z[t[a]];
                    break;
                case OR_X_ERROR:
                case OR_Z_ERROR:
                case OR_DEP1:
                case OR_DEP2:
                case OR_PC1:
                    if (c->ps[i] > 0.0)
                        noise_op_one_lane(c, job->tables[i], i, job->seed, chunk, lane, x, z);
                    break;
                case OR_XFEED:
                    for (int64_t a = 0; a + 1 < nt; a += 2) x[t[a + 1]] ^= rec[t[a]];
                    break;
                case OR_ZFEED:
                    for (int64_t a = 0; a + 1 < nt; a += 2) z[t[a + 1]] ^= rec[t[a]];
                    break;
                case OR_DETECTOR: {
                    uint8_t v = 0;
                    for (int64_t a = 0; a < nt; a++) v ^= rec[t[a]];
                    if (v) job->det[(uint64_t)d * job->n_cols + col] |= (uint64_t)1 << lane;
                    d++;
                    break;
                }
                case OR_OBSERVABLE: {
                    uint8_t v = 0;
                    for (int64_t a = 0; a < nt; a++) v ^= rec[t[a]];
                    obs[c->args[i]] ^= v;
                    break;
                }
                default:
                    break;
                }
            }
            for (int64_t o = 0; o < c->n_obs; o++)
                if (obs[o]) job->obs[(uint64_t)o * job->n_cols + col] |= (uint64_t)1 << lane;
        }
    }
    free(x); free(z); free(rec); free(obs);
    return NULL;
}

static int validate(const oracle_circuit *c)
{
    int64_t m = 0, d = 0;
    for (int64_t i = 0; i < c->n_ops; i++) {
        int code = c->codes[i];
        if (code < 0 || code >= OR_N_CODES) return -1;
        int64_t nt = c->toff[i + 1] - c->toff[i];
        const uint32_t *t = c->targets + c->toff[i];
        if (is_noise(code) && !(c->ps[i] >= 0.0 && c->ps[i] <= 1.0)) return -1;
        if (code == OR_PC1 && c->args[i] > c->args2[i]) return -1;
        if ((code == OR_CX || code == OR_DEP2 || code == OR_XFEED || code == OR_ZFEED) && (nt & 1)) return -1;
        if (code == OR_XFEED || code == OR_ZFEED) {
            for (int64_t a = 0; a < nt; a += 2)
                if ((int64_t)t[a] >= m || (int64_t)t[a + 1] >= c->n_qubits) return -1;
        } else if (code == OR_DETECTOR || code == OR_OBSERVABLE) {
            for (int64_t a = 0; a < nt; a++)
                if ((int64_t)t[a] >= m) return -1;
            if (code == OR_DETECTOR) d++;
            if (code == OR_OBSERVABLE && (int64_t)c->args[i] >= c->n_obs) return -1;
        } else if (code != OR_TICK) {
            for (int64_t a = 0; a < nt; a++)
                if ((int64_t)t[a] >= c->n_qubits) return -1;
        }
        if (code == OR_M || code == OR_MX) m += nt;
    }
    if (m != c->n_meas || d != c->n_det) return -1;
    return 0;
}

/*
 * Sample `shots` shots starting at global chunk `first_chunk`.
 * det: [n_det][ceil(shots/64)] uint64, obs: [n_obs][ceil(shots/64)] uint64,
 * both zero-filled by the caller; bit `lane` of column `col` is shot
 * 64*col + lane. Returns 0, -1 on an invalid circuit, -2 on allocation failure.
 */
int oracle_sample(int64_t n_ops, const int32_t *codes, const double *ps, const uint32_t *args,
                  const uint32_t *args2, const int64_t *toff, const uint32_t *targets,
                  int64_t n_qubits, int64_t n_meas, int64_t n_det, int64_t n_obs,
                  uint64_t seed, uint64_t first_chunk, uint64_t shots,
                  uint64_t *det, uint64_t *obs, int threads)
{
    oracle_circuit c = {n_ops, codes, ps, args, args2, toff, targets, n_qubits, n_meas, n_det, n_obs};
    if (validate(&c) != 0) return -1;
    uint64_t n_cols = (shots + 63) / 64;
    if (first_chunk + n_cols > 0x100000000ull) return -1;
    /* one table per distinct probability */
    const gap_table **tables = calloc((size_t)n_ops + 1, sizeof(gap_table *));
    gap_table *distinct = calloc((size_t)n_ops + 1, sizeof(gap_table));
    double *distinct_p = calloc((size_t)n_ops + 1, sizeof(double));
    int64_t n_distinct = 0;
    if (!tables || !distinct || !distinct_p) { free(tables); free(distinct); free(distinct_p); return -2; }
    for (int64_t i = 0; i < n_ops; i++) {
        if (!is_noise(codes[i]) || !(ps[i] > 0.0)) continue;
        int64_t k = 0;
        while (k < n_distinct && distinct_p[k] != ps[i]) k++;
        if (k == n_distinct) {
            distinct_p[k] = ps[i];
            oracle_gap_table(ps[i], distinct[k].t);
            for (int g = 1; g < GAP_LEN; g++)
                if (distinct[k].t[g] > distinct[k].t[g - 1]) { free(tables); free(distinct); free(distinct_p); return -1; }
            n_distinct++;
        }
        tables[i] = &distinct[k];
    }
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > n_cols) threads = (int)(n_cols ? n_cols : 1);
    shot_job *jobs = calloc((size_t)threads, sizeof(shot_job));
    pthread_t *tid = calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(tables); free(distinct); free(distinct_p); free(jobs); free(tid); return -2; }
    for (int w = 0; w < threads; w++) {
        jobs[w] = (shot_job){&c, tables, seed, first_chunk, shots,
                             n_cols * (uint64_t)w / (uint64_t)threads,
                             n_cols * (uint64_t)(w + 1) / (uint64_t)threads,
                             n_cols, det, obs, 0};
    }
    int rc = 0;
    if (threads == 1) {
        shot_worker(&jobs[0]);
    } else {
        for (int w = 0; w < threads; w++) pthread_create(&tid[w], NULL, shot_worker, &jobs[w]);
        for (int w = 0; w < threads; w++) pthread_join(tid[w], NULL);
    }
    for (int w = 0; w < threads; w++)
        if (jobs[w].status) rc = jobs[w].status;
    free(tables); free(distinct); free(distinct_p); free(jobs); free(tid);
    return rc;
}

/* ---------------------------------------- raw measurement sampling */

/*
 * Measurement records of every shot (not only detector parities): the frame
 * additionally gets a random gauge Pauli wherever it is free to -- Z after R
 * and M, X after RX and MX, Z on every qubit at the start (an implicit R) --
 * which leaves the state unchanged but makes every non-deterministic outcome
 * a fair coin, and each record is reported as reference XOR flip.
 * Gauge word of (op i, target u, chunk c): Philox4x32-10 at counter
 * (u / 2, c, i, 2^31) with the sampling key; (w0 | w1 << 32) for even u,
 * (w2 | w3 << 32) for odd u; bit `lane` applies to shot 64 c + lane. The
 * implicit initial R uses op index n_ops and target u = qubit.
 */
static uint32_t gauge_bit(uint64_t seed, uint32_t op, uint32_t u, uint32_t chunk, uint32_t lane)
{
    uint32_t ctr[4] = {u / 2u, chunk, op, 0x80000000u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    uint64_t word = (u & 1u) ? ((uint64_t)w[2] | ((uint64_t)w[3] << 32)) : ((uint64_t)w[0] | ((uint64_t)w[1] << 32));
    return (uint32_t)((word >> lane) & 1u);
}

typedef struct {
    const oracle_circuit *c;
    const gap_table *const *tables;
    const uint8_t *ref;
    uint64_t seed, first_chunk, shots, col_begin, col_end, n_cols;
    uint64_t *meas;
    int status;
} meas_job;

static void *meas_worker(void *arg)
{
    meas_job *job = (meas_job *)arg;
    const oracle_circuit *c = job->c;
    uint8_t *x = calloc((size_t)c->n_qubits + 1, 1);
    uint8_t *z = calloc((size_t)c->n_qubits + 1, 1);
    uint8_t *rec = calloc((size_t)c->n_meas + 1, 1);
    if (!x || !z || !rec) {
        job->status = -2;
        free(x); free(z); free(rec);
        return NULL;
    }
    for (uint64_t col = job->col_begin; col < job->col_end; col++) {
        uint32_t chunk = (uint32_t)(job->first_chunk + col);
        for (uint32_t lane = 0; lane < 64; lane++) {
            uint64_t shot = col * 64 + lane;
            if (shot >= job->shots) break;
            for (int64_t q = 0; q < c->n_qubits; q++) {
                x[q] = 0;
                z[q] = (uint8_t)gauge_bit(job->seed, (uint32_t)c->n_ops, (uint32_t)q, chunk, lane);
            }
            int64_t m = 0;
            for (int64_t i = 0; i < c->n_ops; i++) {
                int code = c->codes[i];
                const uint32_t *t = c->targets + c->toff[i];
                int64_t nt = c->toff[i + 1] - c->toff[i];
                switch (code) {
                case OR_R:
                    for (int64_t a = 0; a < nt; a++) {
                        x[t[a]] = 0;
                        z[t[a]] = (uint8_t)gauge_bit(job->seed, (uint32_t)i, (uint32_t)a, chunk, lane);
                    }
                    break;
                case OR_RX:
                    for (int64_t a = 0; a < nt; a++) {
                        z[t[a]] = 0;
                        x[t[a]] = (uint8_t)gauge_bit(job->seed, (uint32_t)i, (uint32_t)a, chunk, lane);
                    }
                    break;
                case OR_H:
                    for (int64_t a = 0; a < nt; a++) { uint8_t v = x[t[a]]; x[t[a]] = z[t[a]]; z[t[a]] = v; }
                    break;
                case OR_S:
                    for (int64_t a = 0; a < nt; a++) z[t[a]] ^= x[t[a]];
                    break;
                case OR_CX:
                    for (int64_t a = 0; a + 1 < nt; a += 2) { x[t[a + 1]] ^= x[t[a]]; z[t[a]] ^= z[t[a + 1]]; }
                    break;
                case OR_M:
                    for (int64_t a = 0; a < nt; a++) {
                        rec[m++] = x[t[a]];
                        z[t[a]] ^= (uint8_t)gauge_bit(job->seed, (uint32_t)i, (uint32_t)a, chunk, lane);
                    }
                    break;
                case OR_MX:
                    for (int64_t a = 0; a < nt; a++) {
                        rec[m++] = z[t[a]];
                        x[t[a]] ^= (uint8_t)gauge_bit(job->seed, (uint32_t)i, (uint32_t)a, chunk, lane);
                    }
                    break;
                case OR_X_ERROR:
                case OR_Z_ERROR:
                case OR_DEP1:
                case OR_DEP2:
                case OR_PC1:
                    if (c->ps[i] > 0.0) noise_op_one_lane(c, job->tables[i], i, job->seed, chunk, lane, x, z);
                    break;
                case OR_XFEED:
                    for (int64_t a = 0; a + 1 < nt; a += 2) x[t[a + 1]] ^= rec[t[a]];
                    break;
                case OR_ZFEED:
                    for (int64_t a = 0; a + 1 < nt; a += 2) z[t[a + 1]] ^= rec[t[a]];
                    break;
                default:
                    break;
                }
            }
            for (int64_t r = 0; r < c->n_meas; r++)
                if (rec[r] ^ job->ref[r]) job->meas[(uint64_t)r * job->n_cols + col] |= (uint64_t)1 << lane;
        }
    }
    free(x); free(z); free(rec);
    return NULL;
}

/* meas: [n_meas][ceil(shots/64)] zero-filled; ref: n_meas reference bits. */
int oracle_sample_measurements(int64_t n_ops, const int32_t *codes, const double *ps, const uint32_t *args,
                               const uint32_t *args2, const int64_t *toff, const uint32_t *targets,
                               int64_t n_qubits, int64_t n_meas, int64_t n_det, int64_t n_obs,
                               const uint8_t *ref, uint64_t seed, uint64_t first_chunk, uint64_t shots,
                               uint64_t *meas, int threads)
{
    oracle_circuit c = {n_ops, codes, ps, args, args2, toff, targets, n_qubits, n_meas, n_det, n_obs};
    if (validate(&c) != 0) return -1;
    uint64_t n_cols = (shots + 63) / 64;
    if (first_chunk + n_cols > 0x100000000ull) return -1;
    const gap_table **tables = calloc((size_t)n_ops + 1, sizeof(gap_table *));
    gap_table *distinct = calloc((size_t)n_ops + 1, sizeof(gap_table));
    double *distinct_p = calloc((size_t)n_ops + 1, sizeof(double));
    int64_t n_distinct = 0;
    if (!tables || !distinct || !distinct_p) { free(tables); free(distinct); free(distinct_p); return -2; }
    for (int64_t i = 0; i < n_ops; i++) {
        if (!is_noise(codes[i]) || !(ps[i] > 0.0)) continue;
        int64_t k = 0;
        while (k < n_distinct && distinct_p[k] != ps[i]) k++;
        if (k == n_distinct) {
            distinct_p[k] = ps[i];
            oracle_gap_table(ps[i], distinct[k].t);
            n_distinct++;
        }
        tables[i] = &distinct[k];
    }
    if (threads < 1) threads = 1;
    if ((uint64_t)threads > n_cols) threads = (int)(n_cols ? n_cols : 1);
    meas_job *jobs = calloc((size_t)threads, sizeof(meas_job));
    pthread_t *tid = calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(tables); free(distinct); free(distinct_p); free(jobs); free(tid); return -2; }
    for (int w = 0; w < threads; w++)
        jobs[w] = (meas_job){&c, tables, ref, seed, first_chunk, shots,
                             n_cols * (uint64_t)w / (uint64_t)threads, n_cols * (uint64_t)(w + 1) / (uint64_t)threads,
                             n_cols, meas, 0};
    for (int w = 0; w < threads; w++) pthread_create(&tid[w], NULL, meas_worker, &jobs[w]);
    for (int w = 0; w < threads; w++) pthread_join(tid[w], NULL);
    int rc = 0;
    for (int w = 0; w < threads; w++)
        if (jobs[w].status) rc = jobs[w].status;
    free(tables); free(distinct); free(distinct_p); free(jobs); free(tid);
    return rc;
}

/* ------------------------------------- bit-parallel fault propagation */

/*
 * Noiseless propagation of 64 lanes at once, each lane carrying its own
 * injected Paulis. Used for single-fault detector-error-model enumeration and
 * for the gauge-randomised determinism audit.
 *
 * Injections: n_inj entries (op, target, pauli, lane), sorted by op, are
 * applied right AFTER op `op` executes (the position of a noise op): `pauli`
 * (bit0 = X, bit1 = Z) is XORed onto qubit `target` in lane `lane`.
 * gauge_seed != 0 additionally randomises z after R and M, and x after RX
 * and MX, in every lane (splitmix64 stream), which leaves every deterministic
 * measurement parity unchanged and randomises every non-deterministic one.
 * Outputs: det_words[n_det], obs_words[n_obs] (bit l = lane l).
 */
static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int oracle_propagate64(int64_t n_ops, const int32_t *codes, const double *ps, const uint32_t *args,
                       const uint32_t *args2, const int64_t *toff, const uint32_t *targets,
                       int64_t n_qubits, int64_t n_meas, int64_t n_det, int64_t n_obs,
                       int64_t n_inj, const int64_t *inj_op, const uint32_t *inj_target,
                       const uint32_t *inj_pauli, const uint32_t *inj_lane,
                       uint64_t gauge_seed, uint64_t *det_words, uint64_t *obs_words)
{
    oracle_circuit c = {n_ops, codes, ps, args, args2, toff, targets, n_qubits, n_meas, n_det, n_obs};
    if (validate(&c) != 0) return -1;
    uint64_t *x = calloc((size_t)n_qubits + 1, 8);
    uint64_t *z = calloc((size_t)n_qubits + 1, 8);
    uint64_t *rec = calloc((size_t)n_meas + 1, 8);
    if (!x || !z || !rec) { free(x); free(z); free(rec); return -2; }
    memset(det_words, 0, (size_t)n_det * 8);
    memset(obs_words, 0, (size_t)n_obs * 8);
    uint64_t gs = gauge_seed;
    int64_t m = 0, d = 0, k = 0;
    for (int64_t i = 0; i < n_ops; i++) {
        int code = codes[i];
        const uint32_t *t = targets + toff[i];
        int64_t nt = toff[i + 1] - toff[i];
        switch (code) {
        case OR_R:
            for (int64_t a = 0; a < nt; a++) { x[t[a]] = 0; z[t[a]] = gauge_seed ? splitmix64(&gs) : 0; }
            break;
        case OR_RX:
            for (int64_t a = 0; a < nt; a++) { z[t[a]] = 0; x[t[a]] = gauge_seed ? splitmix64(&gs) : 0; }
            break;
        case OR_H:
            for (int64_t a = 0; a < nt; a++) { uint64_t v = x[t[a]]; x[t[a]] = z[t[a]]; z[t[a]] = v; }
            break;
        case OR_S:
            for (int64_t a = 0; a < nt; a++) z[t[a]] ^= x[t[a]];
            break;
        case OR_CX:
            for (int64_t a = 0; a + 1 < nt; a += 2) { x[t[a + 1]] ^= x[t[a]]; z[t[a]] ^= z[t[a + 1]]; }
            break;
        case OR_M:
            for (int64_t a = 0; a < nt; a++) {
                rec[m++] = x[t[a]];
                if (gauge_seed) z[t[a]] ^= splitmix64(&gs);
            }
            break;
        case OR_MX:
            for (int64_t a = 0; a < nt; a++) {
                rec[m++] = z[t[a]];
                if (gauge_seed) x[t[a]] ^= splitmix64(&gs);
            }
            break;
        case OR_XFEED:
            for (int64_t a = 0; a + 1 < nt; a += 2) x[t[a + 1]] ^= rec[t[a]];
            break;
        case OR_ZFEED:
            for (int64_t a = 0; a + 1 < nt; a += 2) z[t[a + 1]] ^= rec[t[a]];
            break;
        case OR_DETECTOR: {
            uint64_t v = 0;
            for (int64_t a = 0; a < nt; a++) v ^= rec[t[a]];
            det_words[d++] = v;
            break;
        }
        case OR_OBSERVABLE: {
            uint64_t v = 0;
            for (int64_t a = 0; a < nt; a++) v ^= rec[t[a]];
            obs_words[args[i]] ^= v;
            break;
        }
        default:
            break;
        }
        /* injections are sorted by op by the caller; apply those at op i */
        while (k < n_inj && inj_op[k] < i) k++;
        while (k < n_inj && inj_op[k] == i) {
            uint64_t bit = (uint64_t)1 << (inj_lane[k] & 63u);
            if (inj_pauli[k] & 1u) x[inj_target[k]] ^= bit;
            if (inj_pauli[k] & 2u) z[inj_target[k]] ^= bit;
            k++;
        }
    }
    free(x); free(z); free(rec);
    return 0;
}
