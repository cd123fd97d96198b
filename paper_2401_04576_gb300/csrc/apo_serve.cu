// Continuous-batching server over apo_solve_batch (include/apo.h, "Serving").
//
// Fixed batch slots (stream + device workspace + pinned host staging) are created once and
// stay resident.  One scheduling thread harvests finished slots and fills free ones with
// the events that have arrived since, so batches overlap on the device and a new event
// waits only for the next free slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/apo.h"
#include "kernels.cuh"

using namespace apo;

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id;
    std::vector<int32_t> wid;
    std::vector<double> drift;
    Clock::time_point t_submit;   // when apo_serve_submit accepted it
};

struct Result {
    uint64_t id;
    int32_t n_tracks;
    std::vector<apo_track> tracks;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t finished = nullptr;
    unsigned char *dev = nullptr;     // workspace + device inputs / outputs
    unsigned char *host = nullptr;    // pinned staging
    size_t ws_bytes = 0;
    // device views
    int32_t *d_off = nullptr, *d_wid = nullptr, *d_nt = nullptr;
    double *d_dr = nullptr;
    apo_track *d_tr = nullptr;
    // pinned host views
    int32_t *h_off = nullptr, *h_wid = nullptr, *h_nt = nullptr;
    double *h_dr = nullptr;
    apo_track *h_tr = nullptr;
    unsigned *h_status = nullptr;     // the workspace's status word, copied back per batch
    std::vector<uint64_t> ids;
    std::vector<Clock::time_point> t_submit;
    bool busy = false;
};

}  // namespace

struct apo_server {
    const apo_geometry *g = nullptr;
    apo_serve_opts o;
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> pending;
    std::deque<Result> done;
    long long submitted = 0, finished = 0;
    int batches = 0, busy_now = 0, max_busy = 0;
    std::vector<double> latency_ms;   // per finished event: accepted -> batch seen complete
    bool stop = false;
    int error = APO_OK;
    std::string msg;
    std::thread worker;
};

namespace {

int fail_msg(int code, const char *m) {
    set_last_error(m);
    return code;
}

// Extra device / pinned bytes of one slot besides the search workspace.
size_t slot_io_bytes(int B, int max_tracks) {
    return a256(sizeof(int32_t) * (B + 1)) + a256(sizeof(int32_t) * (size_t)B * APO_HIT_CAP) +
           a256(sizeof(double) * (size_t)B * APO_HIT_CAP) +
           a256(sizeof(apo_track) * (size_t)B * max_tracks) + a256(sizeof(int32_t) * B) + 256;
}

template <typename P> void carve(unsigned char *&p, P *&out, size_t bytes) {
    out = reinterpret_cast<P *>(p);
    p += a256(bytes);
}

void free_slot(Slot &s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.finished) cudaEventDestroy(s.finished);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.dev) cudaFree(s.dev);
    if (s.host) cudaFreeHost(s.host);
    s = Slot();
}

// Packs the pending events into a free slot and queues their search.  Called with mu held.
int launch_slot(apo_server *sv, Slot &s) {
    const int B = sv->o.batch_events, mt = sv->o.solve.max_tracks;
    int n = 0, off = 0;
    s.ids.clear();
    s.t_submit.clear();
    s.h_off[0] = 0;
    while (n < B && !sv->pending.empty()) {
        Req &r = sv->pending.front();
        std::memcpy(s.h_wid + off, r.wid.data(), sizeof(int32_t) * r.wid.size());
        std::memcpy(s.h_dr + off, r.drift.data(), sizeof(double) * r.drift.size());
        off += (int)r.wid.size();
        s.h_off[++n] = off;
        s.ids.push_back(r.id);
        s.t_submit.push_back(r.t_submit);
        sv->pending.pop_front();
    }
    if (n == 0) return APO_OK;
    sv->batches++;
    if (sv->o.inject_error_after > 0 && sv->batches == sv->o.inject_error_after)
        return fail_msg(APO_ECUDA, "apo_serve: injected batch failure");
    cudaError_t e = cudaMemcpyAsync(s.d_off, s.h_off, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess && off > 0)
        e = cudaMemcpyAsync(s.d_wid, s.h_wid, sizeof(int32_t) * off, cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess && off > 0)
        e = cudaMemcpyAsync(s.d_dr, s.h_dr, sizeof(double) * off, cudaMemcpyHostToDevice, s.stream);
    if (e != cudaSuccess) return fail_msg(APO_ECUDA, cudaGetErrorString(e));
    apo_hits h{n, s.d_off, s.d_wid, s.d_dr};
    apo_solve_opts so = sv->o.solve;
    so.use_graph = 0;
    int rc = apo_solve_batch(sv->g, &h, &so, s.d_tr, s.d_nt, s.dev, s.ws_bytes, s.stream);
    if (rc != APO_OK) return rc;
    e = cudaMemcpyAsync(s.h_tr, s.d_tr, sizeof(apo_track) * (size_t)n * mt, cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_nt, s.d_nt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s.stream);
    // the search's status word is the first word of the workspace
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_status, s.dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.finished, s.stream);
    if (e != cudaSuccess) return fail_msg(APO_ECUDA, cudaGetErrorString(e));
    s.busy = true;
    return APO_OK;
}

void worker_loop(apo_server *sv) {
    cudaSetDevice(sv->device);
    const int mt = sv->o.solve.max_tracks;
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // harvest finished batches
        for (Slot &s : sv->slots) {
            if (!s.busy) continue;
            cudaError_t q = cudaEventQuery(s.finished);
            if (q == cudaErrorNotReady) continue;
            s.busy = false;
            sv->busy_now--;
            if (q != cudaSuccess) {
                sv->error = APO_ECUDA;
                sv->msg = cudaGetErrorString(q);
                continue;
            }
            if (*s.h_status & ST_TIMEOUT) {
                sv->error = APO_ETIMEOUT;
                sv->msg = "apo_serve: a device wait ran out of its poll limit";
                sv->cv_done.notify_all();
                continue;
            }
            const Clock::time_point now = Clock::now();
            for (size_t i = 0; i < s.ids.size(); i++) {
                sv->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - s.t_submit[i]).count());
                Result r;
                r.id = s.ids[i];
                r.n_tracks = s.h_nt[i];
                r.tracks.assign(s.h_tr + i * mt, s.h_tr + (i + 1) * mt);
                sv->done.push_back(std::move(r));
            }
            sv->finished += (long long)s.ids.size();
            sv->cv_done.notify_all();
        }
        // fill free slots with the events that have arrived
        if (sv->error == APO_OK)
            for (Slot &s : sv->slots) {
                if (s.busy || sv->pending.empty()) continue;
                int rc = launch_slot(sv, s);
                if (rc != APO_OK) {
                    sv->error = rc;
                    sv->msg = apo_last_error();
                    sv->cv_done.notify_all();
                    break;
                }
                if (s.busy) {
                    sv->busy_now++;
                    if (sv->busy_now > sv->max_busy) sv->max_busy = sv->busy_now;
                }
            }
        if (sv->stop && sv->busy_now == 0) break;
        if (sv->busy_now == 0 && (sv->pending.empty() || sv->error != APO_OK))
            sv->cv_work.wait(lk, [&] { return sv->stop || (!sv->pending.empty() && sv->error == APO_OK); });
        else
            sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

void apo_serve_opts_default(apo_serve_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    apo_solve_opts_default(&o->solve);
    o->batch_events = 64;
    o->max_slots = 4;
    o->device_bytes = 0;
    o->max_pending = 4096;
    o->inject_error_after = 0;
}

size_t apo_serve_slot_bytes(const apo_geometry *g, const apo_serve_opts *opts) {
    if (!g || !opts || opts->batch_events < 1 || opts->solve.max_tracks < 1) return 0;
    size_t ws = 0;
    if (apo_workspace_bytes(g, opts->batch_events, &opts->solve, &ws) != APO_OK) return 0;
    return a256(ws) + slot_io_bytes(opts->batch_events, opts->solve.max_tracks);
}

int apo_serve_create(const apo_geometry *g, const apo_serve_opts *opts, apo_server **out) {
    if (!out) return fail_msg(APO_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g) return fail_msg(APO_EINVAL, "geometry is NULL");
    apo_serve_opts o;
    apo_serve_opts_default(&o);
    if (opts) o = *opts;
    if (o.batch_events < 1 || o.max_slots < 1 || o.max_pending < 1)
        return fail_msg(APO_EINVAL, "batch_events, max_slots and max_pending must be >= 1");
    if (o.solve.max_tracks < 1 || o.solve.max_tracks > APO_MAX_TRACKS)
        return fail_msg(APO_EINVAL, "solve.max_tracks out of range");
    if (o.solve.hit_track || o.solve.trace_keys || o.solve.trace_votes || o.solve.trace_count ||
        o.solve.final_level || o.solve.n_final)
        return fail_msg(APO_EINVAL, "the server takes no per-batch device outputs (hit_track, trace)");
    int gdev = -1;
    geometry_device_tables(g, &gdev);
    if (cudaSetDevice(gdev) != cudaSuccess) return fail_msg(APO_ECUDA, "cannot select the geometry's device");
    size_t ws = 0;
    int rc = apo_workspace_bytes(g, o.batch_events, &o.solve, &ws);
    if (rc != APO_OK) return rc;
    const size_t io = slot_io_bytes(o.batch_events, o.solve.max_tracks);
    const size_t slot_bytes = a256(ws) + io;
    int n_slots = o.max_slots;
    if (o.device_bytes > 0) {   // admission by device memory: as many slots as the budget holds
        size_t fit = o.device_bytes / slot_bytes;
        if (fit == 0) return fail_msg(APO_ENOMEM, "apo_serve: device budget below one batch slot");
        if ((size_t)n_slots > fit) n_slots = (int)fit;
    }
    apo_server *sv = new apo_server();
    sv->g = g;
    sv->o = o;
    sv->device = gdev;
    sv->slots.resize(n_slots);
    for (Slot &s : sv->slots) {
        const int B = o.batch_events, mt = o.solve.max_tracks;
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.finished, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&s.dev, slot_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&s.host, io);
        if (e != cudaSuccess) {
            for (Slot &t : sv->slots) free_slot(t);
            delete sv;
            return fail_msg(e == cudaErrorMemoryAllocation ? APO_ENOMEM : APO_ECUDA, cudaGetErrorString(e));
        }
        s.ws_bytes = a256(ws);
        unsigned char *p = s.dev + s.ws_bytes;
        carve(p, s.d_off, sizeof(int32_t) * (B + 1));
        carve(p, s.d_wid, sizeof(int32_t) * (size_t)B * APO_HIT_CAP);
        carve(p, s.d_dr, sizeof(double) * (size_t)B * APO_HIT_CAP);
        carve(p, s.d_tr, sizeof(apo_track) * (size_t)B * mt);
        carve(p, s.d_nt, sizeof(int32_t) * B);
        unsigned char *q = s.host;
        carve(q, s.h_off, sizeof(int32_t) * (B + 1));
        carve(q, s.h_wid, sizeof(int32_t) * (size_t)B * APO_HIT_CAP);
        carve(q, s.h_dr, sizeof(double) * (size_t)B * APO_HIT_CAP);
        carve(q, s.h_tr, sizeof(apo_track) * (size_t)B * mt);
        carve(q, s.h_nt, sizeof(int32_t) * B);
        carve(q, s.h_status, sizeof(unsigned));
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return APO_OK;
}

int32_t apo_serve_slots(const apo_server *sv) { return sv ? (int32_t)sv->slots.size() : 0; }

int apo_serve_submit(apo_server *sv, const int32_t *wire_id, const double *drift, int32_t n_hits,
                     uint64_t request_id) {
    if (!sv) return fail_msg(APO_EINVAL, "server is NULL");
    if (n_hits < 0 || n_hits > APO_HIT_CAP) return fail_msg(APO_EINVAL, "n_hits out of [0, APO_HIT_CAP]");
    if (n_hits > 0 && (!wire_id || !drift)) return fail_msg(APO_EINVAL, "hit arrays are NULL");
    Req r;
    r.id = request_id;
    r.wid.assign(wire_id, wire_id + n_hits);
    r.drift.assign(drift, drift + n_hits);
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->error != APO_OK) return fail_msg(sv->error, sv->msg.c_str());
        if ((int)sv->pending.size() >= sv->o.max_pending) return fail_msg(APO_EBUSY, "apo_serve: queue full");
        sv->pending.push_back(std::move(r));
        sv->submitted++;
    }
    sv->cv_work.notify_one();
    return APO_OK;
}

int apo_serve_poll(apo_server *sv, apo_track *tracks, int32_t *n_tracks, uint64_t *request_id,
                   int32_t max, int32_t *n_done) {
    if (!sv || !n_done) return fail_msg(APO_EINVAL, "server / n_done is NULL");
    *n_done = 0;
    if (max > 0 && (!tracks || !n_tracks || !request_id)) return fail_msg(APO_EINVAL, "output arrays are NULL");
    const int mt = sv->o.solve.max_tracks;
    std::lock_guard<std::mutex> lk(sv->mu);
    int k = 0;
    while (k < max && !sv->done.empty()) {
        Result &r = sv->done.front();
        std::memcpy(tracks + (size_t)k * mt, r.tracks.data(), sizeof(apo_track) * mt);
        n_tracks[k] = r.n_tracks;
        request_id[k] = r.id;
        sv->done.pop_front();
        k++;
    }
    *n_done = k;
    if (sv->error != APO_OK) return fail_msg(sv->error, sv->msg.c_str());
    return APO_OK;
}

int apo_serve_drain(apo_server *sv, int32_t timeout_ms) {
    if (!sv) return fail_msg(APO_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    bool ok = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                   [&] { return sv->finished == sv->submitted || sv->error != APO_OK; });
    if (sv->error != APO_OK) return fail_msg(sv->error, sv->msg.c_str());
    if (!ok) return fail_msg(APO_ETIMEOUT, "apo_serve_drain: timed out");
    return APO_OK;
}

int apo_serve_stats(const apo_server *sv, int32_t *batches, int32_t *max_busy_slots) {
    if (!sv) return fail_msg(APO_EINVAL, "server is NULL");
    apo_server *m = const_cast<apo_server *>(sv);
    std::lock_guard<std::mutex> lk(m->mu);
    if (batches) *batches = m->batches;
    if (max_busy_slots) *max_busy_slots = m->max_busy;
    return APO_OK;
}

int apo_serve_latency(const apo_server *sv, double *p50_ms, double *p99_ms, int64_t *n_events) {
    if (!sv) return fail_msg(APO_EINVAL, "server is NULL");
    apo_server *m = const_cast<apo_server *>(sv);
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(m->mu);
        v = m->latency_ms;
    }
    std::sort(v.begin(), v.end());
    auto rank = [&](double p) -> double {   // nearest rank: the ceil(p n)-th smallest
        if (v.empty()) return 0.0;
        size_t k = (size_t)std::ceil(p * (double)v.size());
        if (k < 1) k = 1;
        return v[k - 1];
    };
    if (p50_ms) *p50_ms = rank(0.50);
    if (p99_ms) *p99_ms = rank(0.99);
    if (n_events) *n_events = (int64_t)v.size();
    return APO_OK;
}

void apo_serve_destroy(apo_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    for (Slot &s : sv->slots) free_slot(s);
    delete sv;
}

}  // extern "C"
