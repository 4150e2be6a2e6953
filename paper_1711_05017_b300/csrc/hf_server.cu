// hf_server.cu -- the serving runtime of include/hf.h: the restricted-
// orientation mode of Section 4.2 (fields precomputed per permitted
// orientation, queried during motion) for many assembly sessions at once.
//
//   * sessions own a stationary and a moving part and the field set most
//     recently published for them;
//   * build requests queue first-in first-out; a scheduler thread admits the
//     head while its field set fits the context's HBM budget and fewer than
//     max_inflight builds run, launching it on one of max_inflight build
//     streams (continuous batching: builds admitted mid-flight overlap on the
//     device with those already running);
//   * a completed build replaces the session's set atomically; readers hold
//     a reference, so a set retired while a query uses it is freed afterwards;
//   * queries run on a pool of high-priority lanes.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <unordered_map>
#include <vector>

#include "hf.h"
#include "hf_internal.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

hf_status srv_fail(hf_status s, const char *fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    hf::set_last_error(msg);
    return s;
}

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_SUPERSEDED = 4 };

// Retired field sets wait here until the scheduler frees them, so that no
// query thread and no holder of the server mutex ever runs a free.
struct Graveyard {
    std::mutex mu;
    std::vector<hf_fieldset *> sets;
    void put(hf_fieldset *fs) {
        std::lock_guard<std::mutex> g(mu);
        sets.push_back(fs);
    }
    std::vector<hf_fieldset *> take() {
        std::lock_guard<std::mutex> g(mu);
        std::vector<hf_fieldset *> out;
        out.swap(sets);
        return out;
    }
};

struct SetHolder {  // a published field set; retired when the last reader lets go
    hf_fieldset *fs;
    Graveyard *gy;
    SetHolder(hf_fieldset *f, Graveyard *g) : fs(f), gy(g) {}
    ~SetHolder() { gy->put(fs); }
};

struct Request {
    int64_t id = 0;
    int session = -1;
    std::vector<float> quats;
    int R = 0;
    unsigned flags = 0;
    int state = RQ_QUEUED;
    double t_submit = 0, t_done = 0;
    hf_fieldset *fs = nullptr;
    cudaEvent_t done = nullptr;
    int stream = -1;
    std::string error;  // why it failed
};

struct Session {
    bool open = false;
    const hf_part *s1 = nullptr, *s2 = nullptr;
    int n = 0;
    std::shared_ptr<SetHolder> current;
    double last_use = 0;
};

struct Lane {
    cudaStream_t st = nullptr;
    float *h_out = nullptr, *d_out = nullptr;  // mapped pinned answer mailbox and its device alias
};

}  // namespace

struct hf_server {
    hf_ctx *ctx = nullptr;
    int device = 0;
    int max_inflight = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> running;
    std::unordered_map<int64_t, std::shared_ptr<Request>> requests;
    std::vector<Session> sessions;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;
    int64_t next_id = 1;
    bool stop = false;
    std::thread sched;
    hf_server_stats stats = {};
    Graveyard graveyard;
    std::mutex lat_mu;
    std::vector<float> lat_us;  // ring of query latencies
    size_t lat_head = 0, lat_count = 0;
    std::mutex lane_mu;
    std::vector<Lane> lanes;
    std::vector<int> free_lanes;
    std::condition_variable lane_cv;
};

static void publish(hf_server *s, const std::shared_ptr<Request> &r) {
    Session &ss = s->sessions[r->session];
    if (ss.open) ss.current = std::make_shared<SetHolder>(r->fs, &s->graveyard);
    else s->graveyard.put(r->fs);
    r->fs = nullptr;
}

// evict the published set of the least recently used other session
static bool evict_one(hf_server *s, int keep) {
    int best = -1;
    for (int i = 0; i < (int)s->sessions.size(); ++i) {
        const Session &ss = s->sessions[i];
        if (i == keep || !ss.current) continue;
        if (best < 0 || ss.last_use < s->sessions[best].last_use) best = i;
    }
    if (best < 0) return false;
    s->sessions[best].current.reset();
    s->stats.evicted++;
    return true;
}

static void free_retired(hf_server *s) {
    for (hf_fieldset *fs : s->graveyard.take()) hf_fieldset_release(fs);
}

// Scheduler: the server mutex guards only the queues and session table;
// allocation, the host set-up and the launches of a build, and every free,
// happen outside it, so queries (which take the mutex briefly) never wait
// for them.
static void scheduler(hf_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::shared_ptr<Request> cand;
        const hf_part *p1 = nullptr, *p2 = nullptr;
        int n = 0, si = -1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            // completions
            for (size_t i = 0; i < s->running.size();) {
                auto &r = s->running[i];
                const cudaError_t q = cudaEventQuery(r->done);
                if (q == cudaErrorNotReady) { ++i; continue; }
                r->t_done = now_ms();
                if (q == cudaSuccess) {
                    publish(s, r);
                    r->state = RQ_DONE;
                    s->stats.completed++;
                    s->stats.rotations_completed += r->R;
                } else {
                    s->graveyard.put(r->fs);
                    r->fs = nullptr;
                    r->state = RQ_FAILED;
                    s->stats.failed++;
                }
                cudaEventDestroy(r->done);
                r->done = nullptr;
                s->stream_busy[r->stream] = 0;
                s->running.erase(s->running.begin() + i);
            }
            // next admissible request, first-in first-out
            while (!s->queue.empty() && (int)s->running.size() < s->max_inflight) {
                auto r = s->queue.front();
                s->queue.pop_front();
                if (r->state == RQ_SUPERSEDED) continue;
                Session &ss = s->sessions[r->session];
                if (!ss.open) {
                    r->state = RQ_FAILED;
                    s->stats.failed++;
                    continue;
                }
                si = 0;
                while (si < (int)s->streams.size() && s->stream_busy[si]) ++si;
                cand = r;
                p1 = ss.s1;
                p2 = ss.s2;
                n = ss.n;
                s->stream_busy[si] = 1;  // reserved while this thread prepares the build
                break;
            }
            s->stats.queued = (int)s->queue.size();
            s->stats.running = (int)s->running.size();
            if (!cand) {
                const bool idle = s->running.empty();
                lk.unlock();
                free_retired(s);
                lk.lock();
                if (!s->stop) s->cv.wait_for(lk, std::chrono::microseconds(idle ? 5000 : 200));
                continue;
            }
        }
        free_retired(s);
        // allocate and launch outside the mutex
        hf_fieldset *fs = nullptr;
        hf_status st = hf_fieldset_create_stream_ordered(s->ctx, n, cand->R, cand->flags, s->streams[si], &fs);
        if (st == HF_EBUDGET) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->stream_busy[si] = 0;
            if (s->running.empty()) {
                // nothing in flight will free memory: make room from other sessions' sets
                if (evict_one(s, cand->session)) {
                    s->queue.push_front(cand);  // keep its place; retry once the set is freed
                } else {
                    cand->state = RQ_FAILED;  // can never fit next to the resident parts
                    s->stats.failed++;
                    s->stats.rejected++;
                }
                continue;
            }
            s->queue.push_front(cand);  // keep its place and wait for a running build
            s->cv.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        if (st == HF_OK) {
            st = hf_fieldset_compute(s->ctx, p1, p2, cand->quats.data(), cand->R, fs, s->streams[si]);
            // a rank-deficient torque neighbourhood is flagged (NaN torque), not fatal
            if (st == HF_EINVAL && hf_fieldset_is_ready(fs)) st = HF_OK;
            if (st != HF_OK) cand->error = hf_last_error();
        }
        cudaEvent_t ev = nullptr;
        if (st == HF_OK && (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventRecord(ev, s->streams[si]) != cudaSuccess))
            st = HF_ECUDA;
        std::lock_guard<std::mutex> g(s->mu);
        if (st == HF_OK) {
            cand->fs = fs;
            cand->done = ev;
            cand->stream = si;
            cand->state = RQ_RUNNING;
            s->running.push_back(cand);
        } else {
            if (fs) s->graveyard.put(fs);
            if (ev) cudaEventDestroy(ev);
            s->stream_busy[si] = 0;
            cand->state = RQ_FAILED;
            s->stats.failed++;
        }
    }
    // drain: wait for everything in flight, then release
    for (auto &r : s->running) {
        cudaEventSynchronize(r->done);
        cudaEventDestroy(r->done);
        s->graveyard.put(r->fs);
        r->fs = nullptr;
        r->state = RQ_FAILED;
    }
    s->running.clear();
    free_retired(s);
}

extern "C" hf_status hf_server_create(hf_ctx *ctx, int max_inflight, int query_lanes, hf_server **out) {
    if (!ctx || !out) return srv_fail(HF_EINVAL, "hf_server_create: NULL argument");
    *out = nullptr;
    if (max_inflight < 1 || max_inflight > 16 || query_lanes < 1 || query_lanes > 64)
        return srv_fail(HF_EINVAL, "hf_server_create: max_inflight %d, query_lanes %d", max_inflight, query_lanes);
    hf_server *s = new hf_server();
    s->ctx = ctx;
    s->max_inflight = max_inflight;
    cudaGetDevice(&s->device);
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int i = 0; i < max_inflight && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo);
        s->streams.push_back(st);
        s->stream_busy.push_back(0);
    }
    s->lanes.resize(query_lanes);
    for (int i = 0; i < query_lanes && e == cudaSuccess; ++i) {
        Lane &L = s->lanes[i];
        e = cudaStreamCreateWithPriority(&L.st, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaHostAlloc(&L.h_out, 8 * sizeof(float), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&L.d_out, L.h_out, 0);
        s->free_lanes.push_back(i);
    }
    if (e != cudaSuccess) {
        hf_server_destroy(s);
        return srv_fail(HF_ECUDA, "hf_server_create: %s", cudaGetErrorString(e));
    }
    s->sched = std::thread(scheduler, s);
    *out = s;
    return HF_OK;
}

extern "C" void hf_server_destroy(hf_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->sched.joinable()) s->sched.join();
    for (auto &ss : s->sessions) ss.current.reset();
    cudaDeviceSynchronize();
    free_retired(s);
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto &L : s->lanes) {
        if (L.st) cudaStreamDestroy(L.st);
        if (L.h_out) cudaFreeHost(L.h_out);
    }
    delete s;
}

extern "C" hf_status hf_server_session_open(hf_server *s, const hf_part *s1, const hf_part *s2, int *session) {
    if (!s || !s1 || !s2 || !session) return srv_fail(HF_EINVAL, "hf_server_session_open: NULL argument");
    // the pair is validated by the first build (roles, sizes)
    std::lock_guard<std::mutex> g(s->mu);
    Session ss;
    ss.open = true;
    ss.s1 = s1;
    ss.s2 = s2;
    ss.n = hf_part_n(s1);
    ss.last_use = now_ms();
    if (ss.n <= 0 || ss.n != hf_part_n(s2)) return srv_fail(HF_EINVAL, "hf_server_session_open: part sizes differ");
    s->sessions.push_back(ss);
    *session = (int)s->sessions.size() - 1;
    s->stats.sessions++;
    return HF_OK;
}

extern "C" hf_status hf_server_session_close(hf_server *s, int session) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_session_close: NULL server");
    std::lock_guard<std::mutex> g(s->mu);
    if (session < 0 || session >= (int)s->sessions.size() || !s->sessions[session].open)
        return srv_fail(HF_EINVAL, "hf_server_session_close: session %d", session);
    s->sessions[session].open = false;
    s->sessions[session].current.reset();
    s->stats.sessions--;
    return HF_OK;
}

extern "C" hf_status hf_server_submit(hf_server *s, int session, const float *h_quat, int R, unsigned flags,
                                      int64_t *request) {
    if (!s || !h_quat || !request) return srv_fail(HF_EINVAL, "hf_server_submit: NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    if (session < 0 || session >= (int)s->sessions.size() || !s->sessions[session].open)
        return srv_fail(HF_EINVAL, "hf_server_submit: session %d", session);
    if (R <= 0) return srv_fail(HF_EINVAL, "hf_server_submit: R=%d", R);
    const size_t need = hf_fieldset_bytes(s->sessions[session].n, R, flags);
    const size_t budget = hf_ctx_budget_bytes(s->ctx);
    if (budget && need > budget) {
        s->stats.rejected++;
        return srv_fail(HF_EBUDGET, "hf_server_submit: %zu bytes exceed the budget of %zu", need, budget);
    }
    // a newer request supersedes this session's still-queued one
    for (auto &q : s->queue)
        if (q->session == session && q->state == RQ_QUEUED) {
            q->state = RQ_SUPERSEDED;
            s->stats.superseded++;
        }
    auto r = std::make_shared<Request>();
    r->id = s->next_id++;
    r->session = session;
    r->quats.assign(h_quat, h_quat + 4 * (size_t)R);
    r->R = R;
    r->flags = flags;
    r->t_submit = now_ms();
    s->queue.push_back(r);
    s->requests[r->id] = r;
    s->stats.submitted++;
    *request = r->id;
    s->cv.notify_all();
    return HF_OK;
}

extern "C" hf_status hf_server_request_state(hf_server *s, int64_t request, int *state, double *latency_ms) {
    if (!s || !state) return srv_fail(HF_EINVAL, "hf_server_request_state: NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->requests.find(request);
    if (it == s->requests.end()) return srv_fail(HF_EINVAL, "hf_server_request_state: request %lld", (long long)request);
    *state = it->second->state;
    if (it->second->state == RQ_FAILED) hf::set_last_error(it->second->error.c_str());
    if (latency_ms) *latency_ms = it->second->state == RQ_DONE ? it->second->t_done - it->second->t_submit : -1.0;
    return HF_OK;
}

static std::shared_ptr<SetHolder> current_set(hf_server *s, int session, hf_status *st) {
    std::lock_guard<std::mutex> g(s->mu);
    if (session < 0 || session >= (int)s->sessions.size() || !s->sessions[session].open) {
        *st = srv_fail(HF_EINVAL, "hf_server: session %d", session);
        return nullptr;
    }
    Session &ss = s->sessions[session];
    ss.last_use = now_ms();
    if (!ss.current) {
        *st = srv_fail(HF_ENOTREADY, "hf_server: session %d has no field set yet", session);
        return nullptr;
    }
    *st = HF_OK;
    return ss.current;
}

constexpr size_t kLatRing = 1u << 20;

extern "C" hf_status hf_server_query(hf_server *s, int session, const float t[3], const float q[4], int k,
                                     float out7[7]) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_query: NULL server");
    const double t0 = now_ms();
    hf_status st = HF_OK;
    std::shared_ptr<SetHolder> set = current_set(s, session, &st);
    if (!set) return st;
    int li;
    {
        std::unique_lock<std::mutex> g(s->lane_mu);
        s->lane_cv.wait(g, [&] { return !s->free_lanes.empty(); });
        li = s->free_lanes.back();
        s->free_lanes.pop_back();
    }
    Lane &L = s->lanes[li];
    st = hf_query_on_lane(set->fs, t, q, k, out7, L.st, L.h_out, L.d_out);
    {
        std::lock_guard<std::mutex> g(s->lane_mu);
        s->free_lanes.push_back(li);
    }
    s->lane_cv.notify_one();
    if (st == HF_OK) {
        const float us = (float)((now_ms() - t0) * 1000.0);
        std::lock_guard<std::mutex> g(s->lat_mu);
        if (s->lat_us.size() < kLatRing) s->lat_us.resize(kLatRing);
        s->lat_us[s->lat_head] = us;
        s->lat_head = (s->lat_head + 1) % kLatRing;
        s->lat_count = std::min(s->lat_count + 1, kLatRing);
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stats.queries++;
    }
    return st;
}

extern "C" int hf_server_query_latencies(hf_server *s, float *out, int max) {
    if (!s || !out || max <= 0) return 0;
    std::lock_guard<std::mutex> g(s->lat_mu);
    const size_t n = std::min(s->lat_count, (size_t)max);
    size_t start = (s->lat_head + kLatRing - s->lat_count) % kLatRing;
    start = (start + (s->lat_count - n)) % kLatRing;  // the newest n
    for (size_t i = 0; i < n; ++i) out[i] = s->lat_us[(start + i) % kLatRing];
    s->lat_count = 0;
    return (int)n;
}

extern "C" hf_status hf_server_field_ptr(hf_server *s, int session, int rot, int field, const float **d_ptr) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_field_ptr: NULL server");
    hf_status st = HF_OK;
    std::shared_ptr<SetHolder> set = current_set(s, session, &st);
    if (!set) return st;
    return hf_fieldset_field_ptr(set->fs, rot, field, d_ptr);
}

extern "C" hf_status hf_server_field_get(hf_server *s, int session, int rot, int field, float *d_dst,
                                         hf_stream stream) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_field_get: NULL server");
    hf_status st = HF_OK;
    std::shared_ptr<SetHolder> set = current_set(s, session, &st);
    if (!set) return st;
    st = hf_fieldset_get(set->fs, rot, field, d_dst, stream);
    // keep the set alive until the copy has run
    if (st == HF_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return srv_fail(HF_ECUDA, "hf_server_field_get: synchronise failed");
    return st;
}

extern "C" hf_status hf_server_stats_get(hf_server *s, hf_server_stats *out) {
    if (!s || !out) return srv_fail(HF_EINVAL, "hf_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    out->reserved_bytes = hf_ctx_reserved_bytes(s->ctx);
    out->budget_bytes = hf_ctx_budget_bytes(s->ctx);
    return HF_OK;
}

extern "C" hf_status hf_server_drive_queries(hf_server *s, int nsess, const int *sessions, const float *poses,
                                             int steps, double rate_hz, int k, int64_t *answered,
                                             int64_t *not_ready, int64_t *late) {
    if (!s || nsess <= 0 || !sessions || !poses || steps <= 0 || !(rate_hz > 0))
        return srv_fail(HF_EINVAL, "hf_server_drive_queries: bad arguments");
    std::atomic<int64_t> ok{0}, nr{0}, lt{0};
    std::mutex err_mu;
    std::string first_err;
    hf_status first_st = HF_OK;
    const double period = 1000.0 / rate_hz;  // ms
    std::vector<std::thread> th;
    for (int i = 0; i < nsess; ++i) {
        th.emplace_back([&, i] {
            cudaSetDevice(s->device);
            const float *p = poses + (size_t)i * steps * 7;
            const double t0 = now_ms();
            for (int j = 0; j < steps; ++j) {
                const double due = t0 + j * period;
                double now = now_ms();
                while (now < due) {  // sleep most of the wait, then spin the last 50 us
                    const double left = due - now;
                    if (left > 0.1) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)((left - 0.05) * 1000)));
                    now = now_ms();
                }
                if (now - due > period) lt++;
                float out[7];
                const hf_status st = hf_server_query(s, sessions[i], p + 7 * (size_t)j, p + 7 * (size_t)j + 3, k, out);
                if (st == HF_OK) {
                    ok++;
                } else {
                    nr++;
                    std::lock_guard<std::mutex> g(err_mu);
                    if (first_st == HF_OK) {
                        first_st = st;
                        first_err = hf_last_error();
                    }
                }
            }
        });
    }
    for (auto &t : th) t.join();
    if (answered) *answered = ok;
    if (not_ready) *not_ready = nr;
    if (late) *late = lt;
    if (first_st != HF_OK && ok == 0)
        return srv_fail(first_st, "hf_server_drive_queries: no query answered; first failure: %s", first_err.c_str());
    return HF_OK;
}
