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

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tmcs_internal.h"

namespace tmcs {

// ------------------------------------------------------------ device code

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
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
    while (g < int(kGapLen) && w < __ldg(T + g)) g++;
    while (g > 0 && w >= __ldg(T + g - 1)) g--;
    return g;
}

struct KernelArgs {
    const Layer *layers;
    const uint32_t *args;
    const NoiseDesc *noise;
    const uint32_t *tables;
    uint32_t n_layers;
    uint32_t n_slots;
    uint32_t key0, key1;
    uint32_t first_chunk;  // global chunk of output column 0
    uint64_t n_cols;       // output columns (chunks) of this call
    uint64_t last_mask;    // valid-shot mask of the last column
    uint64_t *det;
    uint64_t *obs;
};

__device__ __forceinline__ void xor_bit(uint64_t *F, uint32_t slot, uint32_t K, int k, unsigned long long bit) {
    if (slot != kDeadSlot) atomicXor(reinterpret_cast<unsigned long long *>(&F[slot * K + k]), bit);
}

// One event of a noise op: Pauli index from the word, applied to the live
// frame components of the unit's target(s).
template <int K>
__device__ __forceinline__ void apply_event(uint64_t *F, const uint32_t *__restrict__ tg, const NoiseDesc &nd,
                                            uint32_t npauli, uint32_t s, int pos, uint32_t w_pauli, int k) {
    const uint32_t unit = s * kSegUnits + uint32_t(pos >> 6);
    const unsigned long long bit = 1ull << (pos & 63);
    const uint32_t pk = 1u + __umulhi(w_pauli, npauli);
    if (nd.kind == N_DEP2) {
        const uint32_t c0 = __ldg(tg + 2 * unit), c1 = __ldg(tg + 2 * unit + 1);
        const uint32_t pa = pk >> 2, pb = pk & 3u;
        if (pa & 1u) xor_bit(F, c0 & 0xFFFFu, K, k, bit);
        if (pa & 2u) xor_bit(F, c0 >> 16, K, k, bit);
        if (pb & 1u) xor_bit(F, c1 & 0xFFFFu, K, k, bit);
        if (pb & 2u) xor_bit(F, c1 >> 16, K, k, bit);
    } else {
        const uint32_t c0 = __ldg(tg + unit);
        const uint32_t pa = nd.kind == N_XERR ? 1u : nd.kind == N_ZERR ? 2u : pk;
        if (pa & 1u) xor_bit(F, c0 & 0xFFFFu, K, k, bit);
        if (pa & 2u) xor_bit(F, c0 >> 16, K, k, bit);
    }
}

// Noise layer: one thread per (64-unit segment, chunk) walks the segment's
// event stream; each Philox4x32-10 call yields two draws (gap word, Pauli
// word).
template <int K>
__device__ __forceinline__ void noise_layer(uint64_t *F, const uint32_t *__restrict__ tables, const NoiseDesc nd,
                                            const uint32_t *__restrict__ args, uint32_t key0,
                                            uint32_t key1, uint32_t chunk0, int nvalid) {
    const uint32_t *T = tables + size_t(nd.table) * kTableWords;
    const float inv = __uint_as_float(__ldg(T + kGapLen));
    const uint32_t npauli = nd.kind == N_DEP2 ? 15u : nd.kind == N_DEP1 ? 3u : 1u;
    const uint32_t *tg = args + nd.tgt_off;
    const uint32_t work = nd.n_seg * K;
    for (uint32_t u = threadIdx.x; u < work; u += blockDim.x) {
        const uint32_t s = u / K;
        const int k = int(u % K);
        if (k >= nvalid) continue;
        const uint32_t chunk = chunk0 + uint32_t(k);
        const int n_trials = 64 * int(min(kSegUnits, nd.n_units - s * kSegUnits));
        int pos = -1;
        for (uint32_t j = 0;; j++) {
            const uint4 w = philox4x32_10(j, chunk, nd.op_index, s, key0, key1);
            pos += 1 + gap_count(T, inv, w.x);
            if (pos >= n_trials) break;
            apply_event<K>(F, tg, nd, npauli, s, pos, w.y, k);
            pos += 1 + gap_count(T, inv, w.z);
            if (pos >= n_trials) break;
            apply_event<K>(F, tg, nd, npauli, s, pos, w.w, k);
        }
    }
}

// Runs the whole program for one tile of K chunks starting at output column col0.
template <int K>
__device__ __forceinline__ void run_tile(const KernelArgs &P, uint64_t *F, uint64_t col0) {
    const uint64_t rem = P.n_cols - col0;
    const int nvalid = rem < uint64_t(K) ? int(rem) : K;
    const uint32_t chunk0 = P.first_chunk + uint32_t(col0);
    const uint32_t nt = blockDim.x;
    for (uint32_t L = 0; L < P.n_layers; L++) {
        const Layer ly = P.layers[L];
        const uint32_t *__restrict__ a = P.args + ly.off;
        switch (ly.kind) {
        case L_ZERO:
            for (uint32_t i = threadIdx.x; i < ly.count * K; i += nt) F[__ldg(a + i / K) * K + i % K] = 0ull;
            break;
        case L_XOR:
            for (uint32_t i = threadIdx.x; i < ly.count * K; i += nt) {
                const uint32_t w = __ldg(a + i / K);
                F[(w & 0xFFFFu) * K + i % K] ^= F[(w >> 16) * K + i % K];
            }
            break;
        case L_COPY:
            for (uint32_t i = threadIdx.x; i < ly.count * K; i += nt) {
                const uint32_t w = __ldg(a + i / K);
                F[(w & 0xFFFFu) * K + i % K] = F[(w >> 16) * K + i % K];
            }
            break;
        case L_NOISE:
            noise_layer<K>(F, P.tables, P.noise[ly.aux], P.args, P.key0, P.key1, chunk0, nvalid);
            break;
        case L_DET:
            for (uint32_t i = threadIdx.x; i < ly.count * K; i += nt) {
                const uint32_t d = i / K;
                const int k = int(i % K);
                if (k >= nvalid) continue;
                const uint32_t b = __ldg(a + d), e = __ldg(a + d + 1);
                uint64_t v = 0;
                for (uint32_t t = b; t < e; t++) v ^= F[__ldg(P.args + t) * K + k];
                const uint64_t col = col0 + uint64_t(k);
                if (col == P.n_cols - 1) v &= P.last_mask;
                P.det[uint64_t(ly.aux + d) * P.n_cols + col] = v;
            }
            break;
        case L_OBS:
            for (uint32_t i = threadIdx.x; i < ly.count * K; i += nt) {
                const uint32_t d = i / K;
                const int k = int(i % K);
                const uint32_t b = __ldg(a + d), e = __ldg(a + d + 1);
                uint64_t v = 0;
                for (uint32_t t = b + 1; t < e; t++) v ^= F[__ldg(P.args + t) * K + k];
                F[__ldg(P.args + b) * K + k] ^= v;
            }
            break;
        case L_OBSOUT:
            for (uint32_t i = threadIdx.x; i < ly.count * K; i += nt) {
                const uint32_t o = i / K;
                const int k = int(i % K);
                if (k >= nvalid) continue;
                uint64_t v = F[__ldg(a + o) * K + k];
                const uint64_t col = col0 + uint64_t(k);
                if (col == P.n_cols - 1) v &= P.last_mask;
                P.obs[uint64_t(o) * P.n_cols + col] = v;
            }
            break;
        default:
            break;
        }
        __syncthreads();
    }
}

template <int K>
__global__ void __launch_bounds__(1024) frame_kernel(const KernelArgs P) {
    extern __shared__ uint64_t smem[];
    run_tile<K>(P, smem, uint64_t(blockIdx.x) * K);
}

// ------------------------------------------------------------- host code

static int cuda_fail(cudaError_t e, const char *what) {
    return fail(TMCS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Upload (once per device) and return the device copy of a program.
static int device_program(const tmcs_circuit *c, const DeviceProgram **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(c->mu);
    auto it = c->dev.find(dev);
    if (it != c->dev.end()) {
        *out = &it->second;
        return TMCS_OK;
    }
    const Program &P = c->prog;
    const size_t b_layers = align256(P.layers.size() * sizeof(Layer));
    const size_t b_args = align256(P.args.size() * 4);
    const size_t b_noise = align256(P.noise.size() * sizeof(NoiseDesc));
    const size_t b_tables = align256(P.tables.size() * 4);
    const size_t total = std::max<size_t>(b_layers + b_args + b_noise + b_tables, 256);
    std::vector<uint8_t> host(total, 0);
    std::memcpy(host.data(), P.layers.data(), P.layers.size() * sizeof(Layer));
    std::memcpy(host.data() + b_layers, P.args.data(), P.args.size() * 4);
    std::memcpy(host.data() + b_layers + b_args, P.noise.data(), P.noise.size() * sizeof(NoiseDesc));
    std::memcpy(host.data() + b_layers + b_args + b_noise, P.tables.data(), P.tables.size() * 4);
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
    auto ins = c->dev.emplace(dev, dp);
    *out = &ins.first->second;
    return TMCS_OK;
}

void free_device_programs(tmcs_circuit *c) {
    std::lock_guard<std::mutex> lock(c->mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : c->dev) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second.base);
    }
    cudaSetDevice(cur);
    c->dev.clear();
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
    int K = 1;
    int threads = 256;
    size_t smem = 0;
    uint64_t tiles = 0;
};

// Tile shape: as many chunks per CTA as shared memory allows (fewer program
// re-reads, wider detector stores), but enough tiles to fill every SM.
static int env_int(const char *name, int dflt) {
    const char *v = std::getenv(name);
    return (v && *v) ? std::atoi(v) : dflt;
}

// Tuning knobs (autotuner / sweeps): TMCS_TILE_K caps the chunks per CTA,
// TMCS_THREADS fixes the CTA size. Both only change the launch shape, never
// the output bits.
static LaunchShape choose_shape(const Program &P, uint64_t n_cols, const DeviceLimits &lim) {
    const size_t tbytes = 0;  // gap tables are read through L1, not staged
    LaunchShape s;
    int K = 16;
    const int kcap = env_int("TMCS_TILE_K", 16);
    while (K > 1 && K > kcap) K >>= 1;
    while (K > 1 && size_t(P.n_slots) * 8 * K + tbytes > lim.smem_optin) K >>= 1;
    while (K > 1 && (n_cols + K - 1) / K < uint64_t(2 * lim.sms)) K >>= 1;
    s.K = K;
    s.smem = size_t(P.n_slots) * 8 * K + tbytes;
    s.tiles = (n_cols + K - 1) / K;
    const size_t per_sm = std::max<size_t>(1, lim.smem_per_sm / std::max<size_t>(s.smem + 1024, 1));
    int threads = int(2048 / std::min<size_t>(per_sm, 8));
    threads = std::max(128, std::min(1024, threads));
    const int tforce = env_int("TMCS_THREADS", 0);
    if (tforce >= 32 && tforce <= 1024 && tforce % 32 == 0) threads = tforce;
    s.threads = threads;
    return s;
}

template <int K>
static cudaError_t launch_k(const KernelArgs &a, const LaunchShape &s, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(frame_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(s.smem));
    if (e != cudaSuccess) return e;
    frame_kernel<K><<<unsigned(s.tiles), s.threads, s.smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch(const KernelArgs &a, const LaunchShape &s, cudaStream_t st) {
    switch (s.K) {
    case 16: return launch_k<16>(a, s, st);
    case 8: return launch_k<8>(a, s, st);
    case 4: return launch_k<4>(a, s, st);
    case 2: return launch_k<2>(a, s, st);
    default: return launch_k<1>(a, s, st);
    }
}

static int sample_range(const tmcs_circuit *c, uint64_t first_chunk, uint64_t shots, uint64_t seed,
                        uint64_t *det, uint64_t *obs, void *stream) {
    if (!c) return fail(TMCS_E_INVALID, "circuit is NULL");
    if (shots == 0) return fail(TMCS_E_INVALID, "shots must be positive");
    if ((c->n_det && !det) || (c->n_obs && !obs)) return fail(TMCS_E_INVALID, "output buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(det) & 7) || (reinterpret_cast<uintptr_t>(obs) & 7))
        return fail(TMCS_E_BUFFER, "output buffers must be 8-byte aligned");
    const uint64_t n_cols = (shots + 63) / 64;
    if (first_chunk + n_cols > (uint64_t(1) << 32)) return fail(TMCS_E_INVALID, "chunk range beyond 2^32");
    const DeviceProgram *dp = nullptr;
    int rc = device_program(c, &dp);
    if (rc) return rc;
    DeviceLimits lim;
    if ((rc = device_limits(&lim))) return rc;
    const Program &P = c->prog;
    if (size_t(P.n_slots) * 8 > lim.smem_optin)
        return fail(TMCS_E_INVALID, "circuit needs " + std::to_string(P.n_slots) +
                                        " frame slots; one 64-shot chunk does not fit in shared memory");
    if (P.layers.empty()) return TMCS_OK;
    LaunchShape s = choose_shape(P, n_cols, lim);
    KernelArgs a{};
    a.layers = dp->layers;
    a.args = dp->args;
    a.noise = dp->noise;
    a.tables = dp->tables;
    a.n_layers = uint32_t(P.layers.size());
    a.n_slots = P.n_slots;
    a.key0 = uint32_t(seed);
    a.key1 = uint32_t(seed >> 32);
    a.first_chunk = uint32_t(first_chunk);
    a.n_cols = n_cols;
    a.last_mask = (shots % 64) ? ((uint64_t(1) << (shots % 64)) - 1) : ~uint64_t(0);
    a.det = det;
    a.obs = obs;
    cudaError_t e = launch(a, s, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "frame kernel launch");
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

int tmcs_batch_sample(const tmcs_job *jobs, size_t n_jobs, void *stream) {
    if (n_jobs && !jobs) return fail(TMCS_E_INVALID, "jobs is NULL");
    for (size_t j = 0; j < n_jobs; j++) {
        int rc = sample_range(jobs[j].c, 0, jobs[j].shots, jobs[j].seed, jobs[j].det, jobs[j].obs, stream);
        if (rc) return rc;
    }
    return TMCS_OK;
}

}  // extern "C"
