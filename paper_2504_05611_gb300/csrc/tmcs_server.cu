// Sampling server: continuous batching of sampling requests on one GPU.
//
// A scheduler thread owns all device work. Requests are admitted in arrival
// order when their output words fit in a device arena allocated once at
// open (admission by HBM footprint). Every admitted request is cut into
// slices of 64-shot chunks; slices are issued round-robin across all admitted
// requests onto n_streams non-blocking streams (at most two in flight per
// stream), so a newly admitted request starts on the next free stream and its
// slices run concurrently with those of older requests. Each slice is one
// tmcs_sample_range call writing its own [n_det][cols] and [n_obs][cols]
// block in the request's arena space; fetching copies the blocks into the
// caller's host arrays with strided copies, which reproduces the layout (and
// the bits) of one solo tmcs_sample call.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tmcs_internal.h"

namespace tmcs {
namespace {

using Clock = std::chrono::steady_clock;

struct Slice {
    uint64_t first_chunk;  // relative to the request (chunk 0 = its first chunk)
    uint64_t cols;
    uint64_t shots;
    size_t offset_words;   // start of this slice's block in the request's space
};

struct Request {
    uint64_t id = 0;
    const tmcs_circuit *c = nullptr;
    uint64_t shots = 0, seed = 0, n_cols = 0, n_det = 0, n_obs = 0;
    int state = TMCS_REQ_QUEUED;
    std::string error;
    size_t bytes = 0;
    size_t arena_off = 0;
    uint64_t *buf = nullptr;
    std::vector<Slice> slices;
    size_t next_slice = 0, slices_done = 0;
    bool released = false;
    Clock::time_point t_submit, t_admit, t_done;
};

struct InFlight {
    Request *r;
    size_t slice;
    cudaEvent_t ev;
};

// First-fit allocator over [0, size) with coalescing of freed blocks.
class Arena {
public:
    void init(size_t size) {
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t len, size_t *off) {
        len = (len + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                const size_t rest = it->second - len, at = it->first + len;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += len;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len) {
        len = (len + 255) & ~size_t(255);
        used_ -= len;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

private:
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace
}  // namespace tmcs

using namespace tmcs;

struct tmcs_server {
    int device = 0;
    uint32_t n_streams = 4;
    uint64_t slice_chunks = 4096;
    std::vector<cudaStream_t> streams;
    std::vector<std::deque<InFlight>> inflight;
    std::vector<cudaEvent_t> event_pool;
    uint8_t *arena_base = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> active;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_id = 1;
    size_t rr = 0;
    bool stop = false;
    std::thread thr;
    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, shots_done = 0;
    std::vector<double> latencies;
    double busy_seconds = 0.0;
    Clock::time_point busy_since;
    bool busy = false;
};

namespace {

void finish_request(tmcs_server *s, Request *r, bool ok) {
    r->state = ok ? TMCS_REQ_DONE : TMCS_REQ_FAILED;
    r->t_done = Clock::now();
    if (ok) {
        s->completed++;
        s->shots_done += r->shots;
        s->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
    } else {
        s->failed++;
    }
    s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
    if (s->busy && s->active.empty()) {
        s->busy_seconds += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
        s->busy = false;
    }
    s->cv_done.notify_all();
}

// Scheduler thread: admit, issue slices, retire completed slices.
void scheduler(tmcs_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool any_inflight = false;
        for (auto &q : s->inflight) any_inflight = any_inflight || !q.empty();
        if (s->stop && !any_inflight) break;
        // admission in arrival order, by arena footprint
        while (!s->stop && !s->pending.empty()) {
            Request *r = s->pending.front();
            size_t off = 0;
            if (!s->arena.alloc(r->bytes, &off)) break;
            r->arena_off = off;
            r->buf = reinterpret_cast<uint64_t *>(s->arena_base + off);
            r->state = TMCS_REQ_RUNNING;
            r->t_admit = Clock::now();
            s->pending.pop_front();
            s->active.push_back(r);
            if (!s->busy) {
                s->busy = true;
                s->busy_since = Clock::now();
            }
        }
        // issue slices round-robin over admitted requests
        bool issued = false;
        for (uint32_t si = 0; si < s->n_streams && !s->stop; si++) {
            while (s->inflight[si].size() < 2) {
                Request *r = nullptr;
                for (size_t k = 0; k < s->active.size(); k++) {
                    Request *cand = s->active[(s->rr + k) % s->active.size()];
                    if (cand->state == TMCS_REQ_RUNNING && cand->next_slice < cand->slices.size()) {
                        r = cand;
                        s->rr = (s->rr + k + 1) % s->active.size();
                        break;
                    }
                }
                if (!r) break;
                const size_t idx = r->next_slice++;
                const Slice &sl = r->slices[idx];
                cudaEvent_t ev = nullptr;
                if (!s->event_pool.empty()) {
                    ev = s->event_pool.back();
                    s->event_pool.pop_back();
                } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                    cudaGetLastError();
                    r->error = "cannot create a CUDA event";
                    finish_request(s, r, false);
                    break;
                }
                uint64_t *det = r->buf + sl.offset_words;
                uint64_t *obs = det + r->n_det * sl.cols;
                int rc = tmcs_sample_range(r->c, sl.first_chunk, sl.shots, r->seed, det, r->n_obs ? obs : nullptr,
                                           s->streams[si]);
                if (rc == TMCS_OK && cudaEventRecord(ev, s->streams[si]) != cudaSuccess) rc = TMCS_E_CUDA;
                if (rc != TMCS_OK) {
                    r->error = tmcs_last_error();
                    s->event_pool.push_back(ev);
                    r->next_slice = r->slices.size();
                    bool busy_r = false;
                    for (auto &q : s->inflight)
                        for (auto &f : q) busy_r = busy_r || f.r == r;
                    if (!busy_r) finish_request(s, r, false);
                    else r->state = TMCS_REQ_FAILED;
                    break;
                }
                s->inflight[si].push_back({r, idx, ev});
                issued = true;
            }
        }
        // retire completed slices (in issue order per stream)
        bool retired = false;
        for (auto &q : s->inflight) {
            while (!q.empty()) {
                const cudaError_t st = cudaEventQuery(q.front().ev);
                if (st == cudaErrorNotReady) break;
                InFlight f = q.front();
                q.pop_front();
                s->event_pool.push_back(f.ev);
                retired = true;
                Request *r = f.r;
                if (st != cudaSuccess) {
                    cudaGetLastError();
                    r->error = cudaGetErrorString(st);
                    r->state = TMCS_REQ_FAILED;
                }
                r->slices_done++;
                bool r_inflight = false;
                for (auto &q2 : s->inflight)
                    for (auto &g : q2) r_inflight = r_inflight || g.r == r;
                if (r->state == TMCS_REQ_FAILED && !r_inflight) {
                    finish_request(s, r, false);
                } else if (r->state == TMCS_REQ_RUNNING && r->slices_done == r->slices.size()) {
                    finish_request(s, r, true);
                }
            }
        }
        if (!issued && !retired) {
            bool inflight_now = false;
            for (auto &q : s->inflight) inflight_now = inflight_now || !q.empty();
            if (inflight_now)
                s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
    // drop what was never issued
    for (Request *r : s->pending) {
        r->error = "server closed";
        r->state = TMCS_REQ_FAILED;
        s->failed++;
    }
    s->pending.clear();
    for (Request *r : std::vector<Request *>(s->active))
        if (r->state == TMCS_REQ_RUNNING) {
            r->error = "server closed";
            finish_request(s, r, false);
        }
    s->cv_done.notify_all();
}

int wait_done(tmcs_server *s, std::unique_lock<std::mutex> &lk, Request *r) {
    s->cv_done.wait(lk, [&] { return r->state == TMCS_REQ_DONE || r->state == TMCS_REQ_FAILED; });
    if (r->state == TMCS_REQ_FAILED) return fail(TMCS_E_CUDA, "request failed: " + r->error);
    return TMCS_OK;
}

void release_locked(tmcs_server *s, Request *r) {
    if (r->buf) s->arena.release(r->arena_off, r->bytes);
    r->buf = nullptr;
    s->all.erase(r->id);
    s->cv_work.notify_all();
}

}  // namespace

extern "C" {

int tmcs_server_open(const tmcs_server_config *cfg, tmcs_server **out) {
    if (!out) return fail(TMCS_E_INVALID, "out is NULL");
    *out = nullptr;
    std::unique_ptr<tmcs_server> s(new (std::nothrow) tmcs_server());
    if (!s) return fail(TMCS_E_OOM, "out of host memory");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) return fail(TMCS_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    s->n_streams = (cfg && cfg->n_streams) ? std::min<uint32_t>(cfg->n_streams, 32) : 4;
    s->slice_chunks = (cfg && cfg->slice_chunks) ? cfg->slice_chunks : 4096;
    size_t bytes = cfg ? size_t(cfg->arena_bytes) : 0;
    if (!bytes) {
        size_t freeb = 0, total = 0;
        if ((e = cudaMemGetInfo(&freeb, &total)) != cudaSuccess)
            return fail(TMCS_E_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
        bytes = freeb / 2;
    }
    bytes &= ~size_t(255);
    void *base = nullptr;
    if ((e = cudaMalloc(&base, bytes)) != cudaSuccess) {
        cudaGetLastError();
        return fail(TMCS_E_OOM, std::string("cudaMalloc of the server arena: ") + cudaGetErrorString(e));
    }
    s->arena_base = static_cast<uint8_t *>(base);
    s->arena.init(bytes);
    s->streams.resize(s->n_streams);
    s->inflight.resize(s->n_streams);
    for (auto &st : s->streams) {
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
            for (auto &x : s->streams)
                if (x) cudaStreamDestroy(x);
            cudaFree(base);
            return fail(TMCS_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
    }
    tmcs_server *raw = s.get();
    try {
        s->thr = std::thread(scheduler, raw);
    } catch (...) {
        for (auto &x : s->streams) cudaStreamDestroy(x);
        cudaFree(base);
        return fail(TMCS_E_OOM, "cannot start the scheduler thread");
    }
    *out = s.release();
    return TMCS_OK;
}

int tmcs_server_submit(tmcs_server *s, const tmcs_circuit *c, uint64_t shots, uint64_t seed, uint64_t *request_id) {
    if (!s || !c || !request_id) return fail(TMCS_E_INVALID, "NULL argument");
    if (shots == 0) return fail(TMCS_E_INVALID, "shots must be positive");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(TMCS_E_OOM, "out of host memory");
    r->c = c;
    r->shots = shots;
    r->seed = seed;
    r->n_cols = (shots + 63) / 64;
    if (r->n_cols > (uint64_t(1) << 32)) return fail(TMCS_E_INVALID, "too many shots");
    r->n_det = c->n_det;
    r->n_obs = c->n_obs;
    size_t off = 0;
    for (uint64_t c0 = 0; c0 < r->n_cols; c0 += s->slice_chunks) {
        Slice sl;
        sl.first_chunk = c0;
        sl.cols = std::min<uint64_t>(s->slice_chunks, r->n_cols - c0);
        sl.shots = std::min<uint64_t>(64 * sl.cols, shots - 64 * c0);
        sl.offset_words = off;
        off += (r->n_det + r->n_obs) * sl.cols;
        r->slices.push_back(sl);
    }
    r->bytes = std::max<size_t>(off * 8, 256);
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->bytes > s->arena.size())
        return fail(TMCS_E_BUFFER, "request outputs (" + std::to_string(r->bytes) + " bytes) exceed the arena (" +
                                       std::to_string(s->arena.size()) + ")");
    if (s->stop) return fail(TMCS_E_INVALID, "server is closing");
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    *request_id = r->id;
    s->pending.push_back(r.get());
    s->all[r->id] = std::move(r);
    s->submitted++;
    s->cv_work.notify_all();
    return TMCS_OK;
}

int tmcs_server_poll(tmcs_server *s, uint64_t request_id, int *state) {
    if (!s || !state) return fail(TMCS_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end()) return fail(TMCS_E_INVALID, "unknown request");
    *state = it->second->state;
    return TMCS_OK;
}

int tmcs_server_fetch(tmcs_server *s, uint64_t request_id, uint64_t *host_det, uint64_t *host_obs) {
    if (!s) return fail(TMCS_E_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end()) return fail(TMCS_E_INVALID, "unknown request");
    Request *r = it->second.get();
    int rc = wait_done(s, lk, r);
    if (rc) {
        release_locked(s, r);
        return rc;
    }
    // copy every slice block into its columns of the caller's arrays
    cudaSetDevice(s->device);
    for (const Slice &sl : r->slices) {
        const uint64_t *det = r->buf + sl.offset_words;
        const uint64_t *obs = det + r->n_det * sl.cols;
        cudaError_t e = cudaSuccess;
        if (host_det && r->n_det)
            e = cudaMemcpy2D(host_det + sl.first_chunk, r->n_cols * 8, det, sl.cols * 8, sl.cols * 8, r->n_det,
                             cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && host_obs && r->n_obs)
            e = cudaMemcpy2D(host_obs + sl.first_chunk, r->n_cols * 8, obs, sl.cols * 8, sl.cols * 8, r->n_obs,
                             cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            release_locked(s, r);
            return fail(TMCS_E_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
        }
    }
    release_locked(s, r);
    return TMCS_OK;
}

int tmcs_server_release(tmcs_server *s, uint64_t request_id) {
    if (!s) return fail(TMCS_E_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(request_id);
    if (it == s->all.end()) return fail(TMCS_E_INVALID, "unknown request");
    Request *r = it->second.get();
    int rc = wait_done(s, lk, r);
    release_locked(s, r);
    return rc;
}

int tmcs_server_get_stats(tmcs_server *s, tmcs_server_stats *out) {
    if (!s || !out) return fail(TMCS_E_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = s->pending.size();
    out->running = s->active.size();
    out->arena_bytes = s->arena.size();
    out->arena_in_use = s->arena.used();
    out->shots_done = s->shots_done;
    out->busy_seconds = s->busy_seconds +
                        (s->busy ? std::chrono::duration<double>(Clock::now() - s->busy_since).count() : 0.0);
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, size_t(f * double(v.size() - 1) + 0.5))]; };
        out->latency_p50_s = q(0.50);
        out->latency_p99_s = q(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->latency_mean_s = sum / double(v.size());
    }
    return TMCS_OK;
}

int tmcs_server_close(tmcs_server *s) {
    if (!s) return TMCS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(s->device);
    for (auto &q : s->inflight)
        for (auto &f : q) cudaEventDestroy(f.ev);
    for (cudaEvent_t ev : s->event_pool) cudaEventDestroy(ev);
    for (auto &st : s->streams) cudaStreamDestroy(st);
    cudaFree(s->arena_base);
    delete s;
    return TMCS_OK;
}

}  // extern "C"
