// hf_server.cu -- the serving runtime of include/hf.h: the restricted-
// orientation mode of Section 4.2 (fields precomputed per permitted
// orientation, queried during motion) for many assembly sessions at once.
//
//   * sessions own a stationary and a moving part and the field data most
//     recently published for them;
//   * a build request whose field set exceeds the server's chunk limit is
//     split into rotation chunks (hf_rotation_chunks: compact groups on
//     SO(3), each built with its torque neighbours so that the least-squares
//     torque is the whole set's); each chunk is a job;
//   * jobs queue first-in first-out; a scheduler thread admits the head while
//     its field set fits the context's HBM budget and fewer than max_inflight
//     jobs run, launching it on one of max_inflight build streams
//     (continuous batching: jobs admitted mid-flight overlap on the device
//     with those already running, and a large request's chunks are admitted
//     one by one as memory frees);
//   * a completed chunk is published at once: the request's first chunk
//     replaces the session's previous data atomically, later chunks fill in;
//     readers hold a reference, so data retired while a query uses it is
//     freed afterwards;
//   * when the head job does not fit and nothing runs, a published chunk is
//     evicted: the least recently queried idle one, else the largest;
//   * queries run on a pool of high-priority lanes, against the chunk that
//     owns the query's nearest rotation.  The query path takes no lock that
//     the scheduler or a submitting thread holds: the session table has a
//     fixed capacity, and the published data and its chunk slots are read
//     and replaced as atomic shared pointers, so a query never waits for a
//     thread that the OS has descheduled inside a critical section.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/resource.h>

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
    size_t bytes;
    SetHolder(hf_fieldset *f, Graveyard *g, size_t b) : fs(f), gy(g), bytes(b) {}
    ~SetHolder() { gy->put(fs); }
};

// A build request.  Fixed after submission except for the state fields,
// which the server mutex guards.
struct Request {
    int64_t id = 0;
    int session = -1;
    int n = 0;
    int R = 0;
    unsigned flags = 0;
    std::vector<float> quats;        // R x 4 as submitted
    std::vector<double> q;           // R x 4, normalised (routing)
    std::vector<int> owner, local;   // rotation -> chunk, index in that chunk's set
    int nchunks = 1;
    // guarded by the server mutex
    int state = RQ_QUEUED;
    int chunks_done = 0;
    double t_submit = 0, t_done = 0;
    std::string error;  // why it failed
};

struct Job {  // one chunk of a request
    std::shared_ptr<Request> req;
    int chunk = 0;
    std::vector<float> quats;  // the chunk's build set, global index order
    int R = 0;
    bool superseded = false;   // server mutex
    hf_fieldset *fs = nullptr;
    cudaEvent_t done = nullptr;
    int stream = -1;
    const hf_part *p1 = nullptr, *p2 = nullptr;  // held from launch to completion
};

// A session's published field data: one set per chunk of one request.  The
// request (routing tables) is fixed; the slots are atomic shared pointers
// and the use times atomics, so readers take no lock.
// The published pointers are std::atomic<std::shared_ptr>: each guards itself
// with a spin bit held for a reference-count update, so readers of different
// sessions never share a lock (the free-function atomic_load/atomic_store on
// a shared_ptr share a small pool of mutexes across all objects).
struct Published {
    std::shared_ptr<Request> req;
    std::unique_ptr<std::atomic<std::shared_ptr<SetHolder>>[]> chunk;
    std::unique_ptr<std::atomic<double>[]> last_use;
    explicit Published(const std::shared_ptr<Request> &r)
        : req(r),
          chunk(new std::atomic<std::shared_ptr<SetHolder>>[r->nchunks]),
          last_use(new std::atomic<double>[r->nchunks]) {
        for (int c = 0; c < r->nchunks; ++c) last_use[c].store(0.0);
    }
    std::shared_ptr<SetHolder> get(int c) const { return chunk[c].load(); }
    void set(int c, std::shared_ptr<SetHolder> h) { chunk[c].store(std::move(h)); }
};

struct Session {
    std::atomic<bool> open{false};
    const hf_part *s1 = nullptr, *s2 = nullptr;  // held while open; fixed once the session is visible
    int n = 0;
    std::atomic<std::shared_ptr<Published>> current_;
    std::atomic<int64_t> answered{0}, not_ready{0};
    std::shared_ptr<Published> current() const { return current_.load(); }
    void set_current(std::shared_ptr<Published> p) { current_.store(std::move(p)); }
};

struct Lane {
    cudaStream_t st = nullptr;
    float *h_out = nullptr, *d_out = nullptr;  // mapped pinned answer mailbox and its device alias
    // the lane's mailbox of the resident query kernel: the last request number
    // posted; the set the kernel may still read for it; whether a request
    // timed out and is still outstanding (the mailbox is then not written
    // again until the kernel has answered it)
    unsigned seq = 0;
    std::shared_ptr<SetHolder> hold;
    bool outstanding = false;
};

// fixed-size ring of diagnostic rows (slow queries, slow scheduler calls)
struct TraceRing {
    static constexpr int kRows = 4096, kCols = 9;
    std::mutex mu;
    std::vector<double> rows = std::vector<double>((size_t)kRows * kCols);
    int head = 0, count = 0;
    void put(const double *v) {
        std::lock_guard<std::mutex> g(mu);
        memcpy(&rows[(size_t)head * kCols], v, sizeof(double) * kCols);
        head = (head + 1) % kRows;
        count = std::min(count + 1, kRows);
    }
};

// Lock-free latency histogram on a log scale (8 bins per octave from 1 us,
// to about 71 minutes), for the metrics log's per-period percentiles; a
// percentile is reported as its bin's upper edge (within 9%).
struct LogHist {
    static constexpr int kPerOctave = 8, kBins = 8 * 32;
    std::atomic<uint32_t> bin[kBins];
    std::atomic<uint64_t> max_bits{0};  // largest sample since the last take_max (bits of a positive double)
    LogHist() {
        for (auto &b : bin) b.store(0, std::memory_order_relaxed);
    }
    static int index(double us) {
        if (!(us > 1.0)) return 0;
        return std::min((int)ceil(log2(us) * kPerOctave), kBins - 1);
    }
    static double upper(int i) { return exp2((double)i / kPerOctave); }
    void add(double us) {
        bin[index(us)].fetch_add(1, std::memory_order_relaxed);
        uint64_t bits;
        memcpy(&bits, &us, 8);
        uint64_t cur = max_bits.load(std::memory_order_relaxed);
        while (bits > cur && !max_bits.compare_exchange_weak(cur, bits, std::memory_order_relaxed)) {
        }
    }
    double take_max() {
        const uint64_t bits = max_bits.exchange(0, std::memory_order_relaxed);
        double v;
        memcpy(&v, &bits, 8);
        return v;
    }
};

// the JSON-lines metrics log: one line per period from its own thread
struct MetricsLog {
    FILE *f = nullptr;
    int period_ms = 1000;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint32_t prev_q[LogHist::kBins] = {}, prev_b[LogHist::kBins] = {};
    double t_last = 0;
};

constexpr size_t kLatRing = 1u << 20;
constexpr size_t kStageBytes = (size_t)4 << 20;  // a build's uploads: 308 bytes per rotation
constexpr int kMaxSessions = 4096;
constexpr double kSlowQueryUs = 500.0, kSlowCallUs = 1000.0;
constexpr double kIdleMs = 20.0;  // a chunk unqueried this long is idle (first to evict)

}  // namespace

struct hf_server {
    hf_ctx *ctx = nullptr;
    int device = 0;
    int max_inflight = 1;
    size_t chunk_bytes = 0;  // 0: never split a request (server mutex)
    double t0 = 0;           // creation time (trace timestamps)
    std::mutex mu;           // queue, requests, request states, stats; never taken by queries
    std::condition_variable cv;
    std::deque<std::shared_ptr<Job>> queue;
    std::vector<std::shared_ptr<Job>> running;  // the scheduler thread's own
    std::unordered_map<int64_t, std::shared_ptr<Request>> requests;
    std::unique_ptr<Session[]> sessions{new Session[kMaxSessions]};
    std::atomic<int> nsessions{0};
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;
    std::vector<void *> stage;  // per build stream: pinned staging of a build's uploads (kStageBytes)
    int64_t next_id = 1;
    bool stop = false;
    std::thread sched;
    hf_server_stats stats = {};
    std::atomic<int64_t> queries{0};
    Graveyard graveyard;
    std::mutex lat_mu;
    std::vector<float> lat_us;  // ring of query latencies
    size_t lat_head = 0, lat_count = 0;
    LogHist query_hist, build_hist;  // answered queries (us), finished requests submit -> published (us)
    std::mutex log_mu;               // the metrics log's open and close
    std::unique_ptr<MetricsLog> log;
    std::vector<Lane> lanes;
    std::atomic<uint64_t> free_lanes{0};  // bit i: lane i is free (at most 64 lanes)
    TraceRing slow_queries, slow_calls;
    void *arena_mem = nullptr;  // the field-set arena's device region (null: the pool serves)
    hf::Arena arena;
    // the resident query kernel (its host side) and what it has answered
    hf::ResidentQueries res;
    std::atomic<int64_t> res_answered{0}, res_timeouts{0};
};

// a request not answered by the resident query kernel within this long goes
// to the launch path instead
constexpr double kResidentWaitMs = 20.0;

// A query through the resident kernel on lane li: post the request, wait
// (spinning, bounded) for its answer.  *posted receives the time the request
// was posted.  After kResidentWaitMs the query runs by launch instead, and the
// lane's mailbox stays untouched until the kernel has answered the request.
static hf_status resident_query(hf_server *s, int li, Lane &L, const std::shared_ptr<SetHolder> &set,
                                const float t[3], const float q[4], int k, float out7[7], double *posted) {
    hf::QueryReq rq;
    hf_status st = hf_query_request(set->fs, t, q, k, &rq);
    if (st != HF_OK) return st;
    L.hold = set;  // the set outlives the kernel's reads of it
    if (!s->res.query(li, rq, &L.seq, out7, kResidentWaitMs, posted)) {
        L.outstanding = true;
        s->res_timeouts++;
        return hf_query_on_lane(set->fs, t, q, k, out7, L.st, L.h_out, L.d_out);
    }
    L.hold.reset();
    s->res_answered++;
    return HF_OK;
}

static Session *session_at(hf_server *s, int session) {
    if (session < 0 || session >= s->nsessions.load(std::memory_order_acquire)) return nullptr;
    Session *ss = &s->sessions[session];
    return ss->open.load() ? ss : nullptr;
}

static void trace_call(hf_server *s, int kind, double t_start, double t_end) {
    const double us = (t_end - t_start) * 1000.0;
    if (us < kSlowCallUs) return;
    const double row[TraceRing::kCols] = {t_start - s->t0, us, (double)kind, 0, 0, 0, 0, 0, 0};
    s->slow_calls.put(row);
}

// publish a finished chunk (server mutex held); false if it is stale (its
// request is older than the data the session already shows)
static bool publish(hf_server *s, const std::shared_ptr<Job> &j) {
    Session &ss = s->sessions[j->req->session];
    std::shared_ptr<Published> cur = ss.current();
    if (!ss.open.load() || (cur && cur->req->id > j->req->id)) {
        s->graveyard.put(j->fs);
        j->fs = nullptr;
        return false;
    }
    if (!cur || cur->req->id != j->req->id) {
        cur = std::make_shared<Published>(j->req);
        cur->last_use[j->chunk].store(now_ms());
        cur->set(j->chunk, std::make_shared<SetHolder>(j->fs, &s->graveyard,
                                                       hf_fieldset_bytes(j->req->n, j->R, j->req->flags)));
        ss.set_current(cur);  // the previous data is retired once its readers let go
    } else {
        cur->last_use[j->chunk].store(now_ms());
        cur->set(j->chunk, std::make_shared<SetHolder>(j->fs, &s->graveyard,
                                                       hf_fieldset_bytes(j->req->n, j->R, j->req->flags)));
    }
    j->fs = nullptr;
    return true;
}

// evict one published chunk (server mutex held): the least recently queried
// idle one; if every resident chunk was queried within kIdleMs, the largest
// (the fewest sessions lose their data per byte freed).  for_range: the
// budget had room but the arena had no free range of the size wanted, so
// among idle (else all) chunks the one whose release makes the largest free
// range goes first
static bool evict_one(hf_server *s, bool for_range = false) {
    const double now = now_ms();
    Published *bp = nullptr;
    int bc = -1;
    bool b_idle = false;
    double bt = 0;
    size_t bb = 0;
    const int ns = s->nsessions.load();
    for (int i = 0; i < ns; ++i) {
        std::shared_ptr<Published> cur = s->sessions[i].current();
        if (!cur) continue;
        for (int c = 0; c < cur->req->nchunks; ++c) {
            std::shared_ptr<SetHolder> h = cur->get(c);
            if (!h) continue;
            const double t = cur->last_use[c].load();
            const bool idle = now - t > kIdleMs;
            // the size that ranks it: its bytes, or the free range its release makes
            const size_t sz = for_range ? s->arena.merged_if_released(hf_fieldset_arena_block(h->fs)) : h->bytes;
            bool better;
            if (!bp) better = true;
            else if (idle != b_idle) better = idle;
            else if (for_range) better = sz > bb || (sz == bb && t < bt);
            else if (idle) better = t < bt;
            else better = sz > bb || (sz == bb && t < bt);
            if (better) {
                bp = cur.get();
                bc = c;
                b_idle = idle;
                bt = t;
                bb = sz;
            }
        }
    }
    if (!bp) return false;
    bp->set(bc, nullptr);
    s->stats.evicted++;
    return true;
}

static void free_retired(hf_server *s) {
    for (hf_fieldset *fs : s->graveyard.take()) {
        const double a = now_ms();
        hf_fieldset_release(fs);
        trace_call(s, 2, a, now_ms());
    }
}

// server mutex held
static void finish_job(hf_server *s, const std::shared_ptr<Job> &j, bool ok) {
    Request &r = *j->req;
    if (!ok) {
        if (r.state != RQ_SUPERSEDED) r.state = RQ_FAILED;
        s->stats.failed++;
        return;
    }
    s->stats.chunks_completed++;
    int owned = 0;
    for (int i = 0; i < r.R; ++i) owned += r.owner[i] == j->chunk;
    s->stats.rotations_completed += owned;
    if (++r.chunks_done == r.nchunks && r.state != RQ_FAILED && r.state != RQ_SUPERSEDED) {
        r.state = RQ_DONE;
        r.t_done = now_ms();
        s->stats.completed++;
        s->build_hist.add((r.t_done - r.t_submit) * 1000.0);
    }
}

// Scheduler: the server mutex guards only the queue, the requests and the
// statistics; allocation, the host set-up and the launches of a build, the
// event polls and every free happen outside it.
static void scheduler(hf_server *s) {
    cudaSetDevice(s->device);
    std::vector<std::pair<std::shared_ptr<Job>, bool>> finished;
    for (;;) {
        // completions, polled outside the mutex (the running list is this thread's)
        finished.clear();
        for (size_t i = 0; i < s->running.size();) {
            auto &j = s->running[i];
            const cudaError_t q = cudaEventQuery(j->done);
            if (q == cudaErrorNotReady) { ++i; continue; }
            finished.push_back({j, q == cudaSuccess});
            cudaEventDestroy(j->done);
            j->done = nullptr;
            hf_part_drop(j->p1);
            hf_part_drop(j->p2);
            j->p1 = j->p2 = nullptr;
            s->stream_busy[j->stream] = 0;
            s->running.erase(s->running.begin() + i);
        }
        std::shared_ptr<Job> cand;
        const hf_part *p1 = nullptr, *p2 = nullptr;
        int n = 0, si = -1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            for (auto &f : finished) {
                if (f.second) {
                    publish(s, f.first);
                } else {
                    s->graveyard.put(f.first->fs);
                    f.first->fs = nullptr;
                }
                finish_job(s, f.first, f.second);
            }
            // next admissible job, first-in first-out
            while (!s->queue.empty() && (int)s->running.size() < s->max_inflight) {
                auto j = s->queue.front();
                s->queue.pop_front();
                if (j->superseded) continue;
                Session &ss = s->sessions[j->req->session];
                if (!ss.open.load()) {
                    finish_job(s, j, false);
                    continue;
                }
                si = 0;
                while (si < (int)s->streams.size() && s->stream_busy[si]) ++si;
                cand = j;
                p1 = ss.s1;
                p2 = ss.s2;
                hf_part_retain(p1);  // a session closed from here on leaves the build its parts
                hf_part_retain(p2);
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
        const int64_t refusals0 = s->arena.failures();
        double a = now_ms();
        // one pipeline per build (the server runs builds side by side), its
        // uploads staged in the stream's pinned buffer: a stream takes its
        // next build only after the last one has completed
        hf_status st = hf_fieldset_create_stream_ordered(s->ctx, n, cand->R, cand->req->flags, s->streams[si], &fs,
                                                         s->stage[si], kStageBytes, 1,
                                                         s->arena_mem ? &s->arena : nullptr);
        trace_call(s, 0, a, now_ms());
        if (st == HF_EBUDGET) {
            hf_part_drop(p1);
            hf_part_drop(p2);
            std::unique_lock<std::mutex> lk(s->mu);
            s->stream_busy[si] = 0;
            if (s->running.empty()) {
                // nothing in flight will free memory: make room from published chunks
                if (evict_one(s, s->arena.failures() > refusals0)) {
                    s->queue.push_front(cand);  // keep its place; retry once the set is freed
                } else {
                    cand->req->error = "the chunk cannot fit next to the resident parts";
                    finish_job(s, cand, false);
                    s->stats.rejected++;
                }
                continue;
            }
            s->queue.push_front(cand);  // keep its place and wait for a running build
            s->cv.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        std::string err;
        if (st == HF_OK) {
            a = now_ms();
            st = hf_fieldset_compute(s->ctx, p1, p2, cand->quats.data(), cand->R, fs, s->streams[si]);
            trace_call(s, 1, a, now_ms());
            // a rank-deficient torque neighbourhood is flagged (NaN torque), not fatal
            if (st == HF_EINVAL && hf_fieldset_is_ready(fs)) st = HF_OK;
            if (st != HF_OK) err = hf_last_error();
        } else {
            err = hf_last_error();
        }
        cudaEvent_t ev = nullptr;
        if (st == HF_OK && (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventRecord(ev, s->streams[si]) != cudaSuccess))
            st = HF_ECUDA;
        if (st == HF_OK) {
            cand->fs = fs;
            cand->done = ev;
            cand->stream = si;
            cand->p1 = p1;
            cand->p2 = p2;
            s->running.push_back(cand);
            std::lock_guard<std::mutex> g(s->mu);
            if (cand->req->state == RQ_QUEUED) cand->req->state = RQ_RUNNING;
        } else {
            if (fs) s->graveyard.put(fs);
            if (ev) cudaEventDestroy(ev);
            cudaStreamSynchronize(s->streams[si]);  // a partial enqueue may still read the parts
            hf_part_drop(p1);
            hf_part_drop(p2);
            std::lock_guard<std::mutex> g(s->mu);
            s->stream_busy[si] = 0;
            cand->req->error = err;
            finish_job(s, cand, false);
        }
    }
    // drain: wait for everything in flight, then release
    for (auto &j : s->running) {
        cudaEventSynchronize(j->done);
        cudaEventDestroy(j->done);
        s->graveyard.put(j->fs);
        j->fs = nullptr;
        hf_part_drop(j->p1);
        hf_part_drop(j->p2);
        j->p1 = j->p2 = nullptr;
        std::lock_guard<std::mutex> g(s->mu);
        if (j->req->state != RQ_DONE) j->req->state = RQ_FAILED;
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
    hf_ctx_retain(ctx);
    s->max_inflight = max_inflight;
    s->chunk_bytes = hf_ctx_budget_bytes(ctx) / 3;
    s->t0 = now_ms();
    s->lat_us.resize(kLatRing);  // no allocation on the query path
    cudaGetDevice(&s->device);
    // every kernel the builds and queries can launch, loaded now: a kernel
    // loaded lazily at its first launch held up all query lanes' launches
    // while the driver loaded it (a driver without per-function loading
    // keeps lazy loading)
    (void)hf_ctx_preload(ctx, nullptr);
    // The builds' field sets come from one device arena of the context's
    // remaining budget (up to the free memory less 4 GB), carved by host
    // bookkeeping: a build then maps no memory while queries launch (pool
    // growth and remapping held up other threads' launches for milliseconds).
    // Without a budget, or without room for the arena, they allocate
    // stream-ordered from the device's default pool, which keeps what it has
    // reserved instead of handing it back at every synchronisation.
    // The arena holds half again the budget it serves (HF_ARENA_SLACK,
    // percent): the budget caps the live field data, and the slack absorbs
    // the gaps that sets of mixed sizes leave between them (at a quarter,
    // 14 times as many chunks found no free range in a 60 s serving run)
    cudaError_t e = cudaSuccess;
    const size_t budget = hf_ctx_budget_bytes(ctx), held = hf_ctx_reserved_bytes(ctx);
    size_t free_b = 0, total_b = 0;
    if (budget > held && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t margin = (size_t)4 << 30;
        const char *ev = getenv("HF_ARENA_SLACK");
        const long slack = ev ? std::max(0L, std::min(400L, atol(ev))) : 50L;
        const size_t span = budget - held, with_slack = span + span / 100 * (size_t)slack;
        const size_t want = std::min(with_slack, free_b > margin ? free_b - margin : 0);
        if (want > 0 && hf::dmalloc(&s->arena_mem, want) == cudaSuccess) s->arena.reset((uintptr_t)s->arena_mem, want);
        else s->arena_mem = nullptr;
        (void)cudaGetLastError();  // an arena that does not fit is not an error: the pool serves
    }
    if (!s->arena_mem) {
        cudaMemPool_t pool = nullptr;
        e = cudaDeviceGetDefaultMemPool(&pool, s->device);
        if (e == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    int lo = 0, hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int i = 0; i < max_inflight && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo);
        s->streams.push_back(st);
        s->stream_busy.push_back(0);
        void *h = nullptr;
        if (e == cudaSuccess) e = cudaHostAlloc(&h, kStageBytes, cudaHostAllocDefault);
        s->stage.push_back(h);
    }
    s->lanes.resize(query_lanes);
    for (int i = 0; i < query_lanes && e == cudaSuccess; ++i) {
        Lane &L = s->lanes[i];
        e = cudaStreamCreateWithPriority(&L.st, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaHostAlloc(&L.h_out, 8 * sizeof(float), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&L.d_out, L.h_out, 0);
        s->free_lanes.fetch_or(uint64_t(1) << i);
    }
    if (e != cudaSuccess) {
        hf_server_destroy(s);
        return srv_fail(HF_ECUDA, "hf_server_create: %s", cudaGetErrorString(e));
    }
    // the resident query kernel (HF_RESIDENT_QUERIES=0: every query by launch);
    // without its memory or stream the queries launch, which is not an error
    const char *rev = getenv("HF_RESIDENT_QUERIES");
    if (!(rev && atoi(rev) == 0)) (void)s->res.start(s->device, query_lanes);
    (void)cudaGetLastError();
    s->sched = std::thread(scheduler, s);
    *out = s;
    return HF_OK;
}

namespace {
void log_stop(hf_server *s);
}

extern "C" void hf_server_destroy(hf_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->log_mu);
        log_stop(s);
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->sched.joinable()) s->sched.join();
    s->res.stop();  // no instance runs after this
    for (auto &L : s->lanes) L.hold.reset();
    for (int i = 0; i < s->nsessions.load(); ++i) s->sessions[i].set_current(nullptr);
    cudaDeviceSynchronize();
    free_retired(s);
    for (int i = 0; i < s->nsessions.load(); ++i) {
        Session &ss = s->sessions[i];
        if (!ss.open.exchange(false)) continue;
        hf_part_drop(ss.s1);
        hf_part_drop(ss.s2);
    }
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto h : s->stage)
        if (h) cudaFreeHost(h);
    for (auto &L : s->lanes) {
        if (L.st) cudaStreamDestroy(L.st);
        if (L.h_out) cudaFreeHost(L.h_out);
    }

    if (s->arena_mem) {
        cudaFree(s->arena_mem);  // every set carved from it was released above
    } else {
        cudaMemPool_t pool = nullptr;
        if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
            cudaDeviceSynchronize();
            cudaMemPoolTrimTo(pool, 0);
        }
    }
    hf_ctx *c = s->ctx;
    delete s;
    hf_ctx_release(c);
}

extern "C" hf_status hf_server_set_chunk_bytes(hf_server *s, size_t bytes) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_set_chunk_bytes: NULL server");
    std::lock_guard<std::mutex> g(s->mu);
    s->chunk_bytes = bytes;
    return HF_OK;
}

extern "C" hf_status hf_server_session_open(hf_server *s, const hf_part *s1, const hf_part *s2, int *session) {
    if (!s || !s1 || !s2 || !session) return srv_fail(HF_EINVAL, "hf_server_session_open: NULL argument");
    // the pair is validated by the first build (roles, sizes)
    const int n = hf_part_n(s1);
    if (n <= 0 || n != hf_part_n(s2)) return srv_fail(HF_EINVAL, "hf_server_session_open: part sizes differ");
    std::lock_guard<std::mutex> g(s->mu);
    const int i = s->nsessions.load();
    if (i >= kMaxSessions) return srv_fail(HF_EINVAL, "hf_server_session_open: more than %d sessions", kMaxSessions);
    Session &ss = s->sessions[i];
    hf_part_retain(s1);
    hf_part_retain(s2);
    ss.s1 = s1;
    ss.s2 = s2;
    ss.n = n;
    ss.open.store(true);
    s->nsessions.store(i + 1, std::memory_order_release);  // visible to readers from here on
    *session = i;
    s->stats.sessions++;
    return HF_OK;
}

extern "C" hf_status hf_server_session_close(hf_server *s, int session) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_session_close: NULL server");
    const hf_part *p1, *p2;
    {
        std::lock_guard<std::mutex> g(s->mu);
        Session *ss = session_at(s, session);
        if (!ss) return srv_fail(HF_EINVAL, "hf_server_session_close: session %d", session);
        ss->open.store(false);
        ss->set_current(nullptr);
        s->stats.sessions--;
        // its unfinished requests fail; queued chunks are dropped, running
        // ones complete and are discarded
        for (auto &j : s->queue)
            if (j->req->session == session) j->superseded = true;
        for (auto &kv : s->requests) {
            Request &r = *kv.second;
            if (r.session != session || (r.state != RQ_QUEUED && r.state != RQ_RUNNING)) continue;
            r.state = RQ_FAILED;
            r.error = "session closed";
            s->stats.failed++;
        }
        p1 = ss->s1;
        p2 = ss->s2;
    }
    // the session's references; a build of it in flight holds its own
    hf_part_drop(p1);
    hf_part_drop(p2);
    return HF_OK;
}

// largest build set (rotations) whose field set fits `limit` bytes
static int max_build_rotations(int n, unsigned flags, size_t limit) {
    int lo = 0, hi = 1;
    while (hi < (1 << 20) && hf_fieldset_bytes(n, hi, flags) <= limit) hi *= 2;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        (hf_fieldset_bytes(n, mid, flags) <= limit ? lo : hi) = mid;
    }
    return lo;
}

extern "C" hf_status hf_server_submit(hf_server *s, int session, const float *h_quat, int R, unsigned flags,
                                      int64_t *request) {
    if (!s || !h_quat || !request) return srv_fail(HF_EINVAL, "hf_server_submit: NULL argument");
    if (R <= 0) return srv_fail(HF_EINVAL, "hf_server_submit: R=%d", R);
    Session *ss = session_at(s, session);
    if (!ss) return srv_fail(HF_EINVAL, "hf_server_submit: session %d", session);
    const int n = ss->n;
    size_t chunk_bytes;
    {
        std::lock_guard<std::mutex> g(s->mu);
        chunk_bytes = s->chunk_bytes;
    }
    auto r = std::make_shared<Request>();
    r->session = session;
    r->n = n;
    r->R = R;
    r->flags = flags;
    r->quats.assign(h_quat, h_quat + 4 * (size_t)R);
    r->q.resize(4 * (size_t)R);
    for (int i = 0; i < R; ++i) {
        const float *v = h_quat + 4 * (size_t)i;
        const double w = v[0], x = v[1], y = v[2], z = v[3], nq = sqrt(w * w + x * x + y * y + z * z);
        if (!(nq > 0) || !isfinite(nq)) return srv_fail(HF_EINVAL, "hf_server_submit: quaternion %d", i);
        double *o = &r->q[4 * (size_t)i];
        o[0] = w / nq; o[1] = x / nq; o[2] = y / nq; o[3] = z / nq;
    }
    // split the request when its set exceeds the chunk limit (host work,
    // outside the server mutex)
    std::vector<std::shared_ptr<Job>> jobs;
    const size_t need = hf_fieldset_bytes(n, R, flags);
    const size_t budget = hf_ctx_budget_bytes(s->ctx);
    if (chunk_bytes && need > chunk_bytes) {
        const bool halo = (flags & HF_T) != 0;  // the least-squares torque needs its 6 neighbours
        const int mb = max_build_rotations(n, flags, chunk_bytes);
        if (mb < (halo ? 7 : 1)) {
            std::lock_guard<std::mutex> g(s->mu);
            s->stats.rejected++;
            return srv_fail(HF_EBUDGET, "hf_server_submit: a chunk of N=%d does not fit %zu bytes", n, chunk_bytes);
        }
        std::vector<int> offs((size_t)R + 1), build((size_t)R * 7);
        r->owner.resize(R);
        const int C = hf_rotation_chunks(h_quat, R, mb, halo ? 1 : 0, r->owner.data(), offs.data(), build.data(),
                                         (int)build.size());
        if (C < 1) return srv_fail(HF_EINVAL, "hf_server_submit: rotation chunking failed");
        r->nchunks = C;
        r->local.assign(R, -1);
        for (int c = 0; c < C; ++c) {
            auto j = std::make_shared<Job>();
            j->req = r;
            j->chunk = c;
            j->R = offs[c + 1] - offs[c];
            j->quats.resize(4 * (size_t)j->R);
            for (int m = 0; m < j->R; ++m) {
                const int g = build[offs[c] + m];
                memcpy(&j->quats[4 * (size_t)m], h_quat + 4 * (size_t)g, 4 * sizeof(float));
                if (r->owner[g] == c) r->local[g] = m;
            }
            jobs.push_back(j);
        }
    } else {
        if (budget && need > budget) {
            std::lock_guard<std::mutex> g(s->mu);
            s->stats.rejected++;
            return srv_fail(HF_EBUDGET, "hf_server_submit: %zu bytes exceed the budget of %zu", need, budget);
        }
        r->owner.assign(R, 0);
        r->local.resize(R);
        for (int i = 0; i < R; ++i) r->local[i] = i;
        auto j = std::make_shared<Job>();
        j->req = r;
        j->R = R;
        j->quats.assign(h_quat, h_quat + 4 * (size_t)R);
        jobs.push_back(j);
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (!ss->open.load()) return srv_fail(HF_EINVAL, "hf_server_submit: session %d", session);
    // a newer request supersedes this session's still-queued jobs
    for (auto &j : s->queue)
        if (j->req->session == session && !j->superseded) {
            j->superseded = true;
            if (j->req->state != RQ_SUPERSEDED) {
                j->req->state = RQ_SUPERSEDED;
                s->stats.superseded++;
            }
        }
    r->id = s->next_id++;
    r->t_submit = now_ms();
    for (auto &j : jobs) s->queue.push_back(j);
    s->requests[r->id] = r;
    s->stats.submitted++;
    s->stats.chunks_submitted += (int64_t)jobs.size();
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

extern "C" hf_status hf_server_request_chunks(hf_server *s, int64_t request, int *chunks, int *owner) {
    if (!s || !chunks) return srv_fail(HF_EINVAL, "hf_server_request_chunks: NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->requests.find(request);
    if (it == s->requests.end()) return srv_fail(HF_EINVAL, "hf_server_request_chunks: request %lld", (long long)request);
    *chunks = it->second->nchunks;
    if (owner) std::copy(it->second->owner.begin(), it->second->owner.end(), owner);
    return HF_OK;
}

// nearest rotation of the published request to q (|q . q_r| largest, ties to
// the lower index)
static int route(const Request &r, const float *q) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    int best = 0;
    double bd = -1.0;
    for (int i = 0; i < r.R; ++i) {
        const double *v = &r.q[4 * (size_t)i];
        const double d = fabs(w * v[0] + x * v[1] + y * v[2] + z * v[3]);
        if (d > bd) { bd = d; best = i; }
    }
    return best;
}

// The set that answers for the session (no server lock): the chunk owning
// rotation `rot` (rot >= 0) or the one owning the nearest rotation to q;
// *local receives rot's index in that set.
static std::shared_ptr<SetHolder> session_set(hf_server *s, int session, int rot, const float *q, int *local,
                                              hf_status *st) {
    Session *ss = session_at(s, session);
    if (!ss) {
        *st = srv_fail(HF_EINVAL, "hf_server: session %d", session);
        return nullptr;
    }
    std::shared_ptr<Published> cur = ss->current();
    if (!cur) {
        *st = srv_fail(HF_ENOTREADY, "hf_server: session %d has no field set yet", session);
        return nullptr;
    }
    const Request &r = *cur->req;
    int c = 0;
    if (rot >= 0) {
        if (rot >= r.R) {
            *st = srv_fail(HF_EINVAL, "hf_server: rotation %d of %d", rot, r.R);
            return nullptr;
        }
        c = r.owner[rot];
        if (local) *local = r.local[rot];
    } else if (r.nchunks > 1) {
        c = r.owner[route(r, q)];
    }
    std::shared_ptr<SetHolder> h = cur->get(c);
    if (!h) {
        *st = srv_fail(HF_ENOTREADY, "hf_server: session %d: chunk %d of its field set is not resident", session, c);
        return nullptr;
    }
    cur->last_use[c].store(now_ms());
    *st = HF_OK;
    return h;
}

extern "C" hf_status hf_server_query(hf_server *s, int session, const float t[3], const float q[4], int k,
                                     float out7[7]) {
    if (!s || !t || !q || !out7) return srv_fail(HF_EINVAL, "hf_server_query: NULL argument");
    const double t0 = now_ms();
    struct rusage ru0;
    getrusage(RUSAGE_THREAD, &ru0);
    hf_status st = HF_OK;
    std::shared_ptr<SetHolder> set = session_set(s, session, -1, q, nullptr, &st);
    Session *ss = session_at(s, session);
    if (!set) {
        if (ss && st == HF_ENOTREADY) ss->not_ready++;
        return st;
    }
    const double t1 = now_ms();
    int li;
    {
        // take the lowest free lane without a lock; with every lane busy
        // (more querying threads than lanes) yield until one frees
        uint64_t m = s->free_lanes.load(std::memory_order_acquire);
        for (;;) {
            if (m == 0) {
                std::this_thread::yield();
                m = s->free_lanes.load(std::memory_order_acquire);
                continue;
            }
            li = __builtin_ctzll(m);
            if (s->free_lanes.compare_exchange_weak(m, m & ~(uint64_t(1) << li), std::memory_order_acquire))
                break;
        }
    }
    const double t2 = now_ms();
    Lane &L = s->lanes[li];
    double tl = t2;
    if (L.outstanding && s->res.answered(li, L.seq)) {
        L.outstanding = false;  // the timed-out request has been answered: the mailbox is free
        L.hold.reset();
    }
    if (s->res.live() && !L.outstanding)
        st = resident_query(s, li, L, set, t, q, k, out7, &tl);
    else
        st = hf_query_on_lane(set->fs, t, q, k, out7, L.st, L.h_out, L.d_out, &tl);
    const double t3 = now_ms();
    s->free_lanes.fetch_or(uint64_t(1) << li, std::memory_order_release);
    if (st == HF_OK) {
        if (ss) ss->answered++;
        const double us = (t3 - t0) * 1000.0;
        s->query_hist.add(us);
        {
            std::lock_guard<std::mutex> g(s->lat_mu);
            s->lat_us[s->lat_head] = (float)us;
            s->lat_head = (s->lat_head + 1) % kLatRing;
            s->lat_count = std::min(s->lat_count + 1, kLatRing);
        }
        if (us >= kSlowQueryUs) {
            // context switches of this thread during the query: involuntary
            // ones (the OS took the core) apart from voluntary ones (a wait)
            struct rusage ru1;
            getrusage(RUSAGE_THREAD, &ru1);
            const double row[TraceRing::kCols] = {t0 - s->t0, us, (t1 - t0) * 1e3, (t2 - t1) * 1e3, (tl - t2) * 1e3,
                                                  (t3 - tl) * 1e3, (double)session, (double)(ru1.ru_nivcsw - ru0.ru_nivcsw),
                                                  (double)(ru1.ru_nvcsw - ru0.ru_nvcsw)};
            s->slow_queries.put(row);
        }
    }
    s->queries++;
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

extern "C" int hf_server_trace(hf_server *s, int which, double *out, int max) {
    if (!s || !out || max <= 0 || (which != 0 && which != 1)) return 0;
    TraceRing &t = which == 0 ? s->slow_queries : s->slow_calls;
    std::lock_guard<std::mutex> g(t.mu);
    const int n = std::min(t.count, max);
    const int start = (t.head + TraceRing::kRows - t.count + (t.count - n)) % TraceRing::kRows;
    for (int i = 0; i < n; ++i)
        memcpy(out + (size_t)i * TraceRing::kCols, &t.rows[(size_t)((start + i) % TraceRing::kRows) * TraceRing::kCols],
               sizeof(double) * TraceRing::kCols);
    t.count = 0;
    return n;
}

extern "C" hf_status hf_server_session_counts(hf_server *s, int session, int64_t *answered, int64_t *not_ready) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_session_counts: NULL server");
    if (session < 0 || session >= s->nsessions.load())
        return srv_fail(HF_EINVAL, "hf_server_session_counts: session %d", session);
    const Session &ss = s->sessions[session];
    if (answered) *answered = ss.answered.load();
    if (not_ready) *not_ready = ss.not_ready.load();
    return HF_OK;
}

extern "C" hf_status hf_server_field_ptr(hf_server *s, int session, int rot, int field, const float **d_ptr) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_field_ptr: NULL server");
    if (rot < 0) return srv_fail(HF_EINVAL, "hf_server_field_ptr: rotation %d", rot);
    hf_status st = HF_OK;
    int local = 0;
    std::shared_ptr<SetHolder> set = session_set(s, session, rot, nullptr, &local, &st);
    if (!set) return st;
    return hf_fieldset_field_ptr(set->fs, local, field, d_ptr);
}

extern "C" hf_status hf_server_field_get(hf_server *s, int session, int rot, int field, float *d_dst,
                                         hf_stream stream) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_field_get: NULL server");
    if (rot < 0) return srv_fail(HF_EINVAL, "hf_server_field_get: rotation %d", rot);
    hf_status st = HF_OK;
    int local = 0;
    std::shared_ptr<SetHolder> set = session_set(s, session, rot, nullptr, &local, &st);
    if (!set) return st;
    st = hf_fieldset_get(set->fs, local, field, d_dst, stream);
    // keep the set alive until the copy has run
    if (st == HF_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return srv_fail(HF_ECUDA, "hf_server_field_get: synchronise failed");
    return st;
}

extern "C" hf_status hf_server_stats_get(hf_server *s, hf_server_stats *out) {
    if (!s || !out) return srv_fail(HF_EINVAL, "hf_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    out->queries = s->queries.load();
    out->reserved_bytes = hf_ctx_reserved_bytes(s->ctx);
    out->budget_bytes = hf_ctx_budget_bytes(s->ctx);
    out->chunk_bytes = s->chunk_bytes;
    int resident = 0;
    for (int i = 0; i < s->nsessions.load(); ++i) {
        std::shared_ptr<Published> cur = s->sessions[i].current();
        if (cur)
            for (int c = 0; c < cur->req->nchunks; ++c) resident += cur->get(c) ? 1 : 0;
    }
    out->chunks_resident = resident;
    cudaMemPool_t pool = nullptr;
    out->pool_reserved_bytes = out->pool_reserved_high = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        unsigned long long v = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) == cudaSuccess)
            out->pool_reserved_bytes = (size_t)v;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &v) == cudaSuccess)
            out->pool_reserved_high = (size_t)v;
    }
    (void)cudaGetLastError();
    out->arena_bytes = s->arena.capacity();
    out->arena_free_bytes = s->arena.free_bytes();
    out->arena_largest_free = s->arena.largest_free();
    out->arena_refusals = s->arena.failures();
    out->resident_queries = s->res_answered.load();
    out->resident_timeouts = s->res_timeouts.load();
    out->resident_live = s->res.live() ? 1 : 0;
    return HF_OK;
}

// --------------------------------------------------------- metrics log
namespace {

// the period's sample count and quantiles (bin upper edges) from the bins'
// growth since `prev`, which is advanced
void hist_period(const LogHist &h, uint32_t *prev, uint64_t *n, const double *qs, double *out, int nq) {
    uint32_t d[LogHist::kBins];
    uint64_t tot = 0;
    for (int i = 0; i < LogHist::kBins; ++i) {
        const uint32_t c = h.bin[i].load(std::memory_order_relaxed);
        d[i] = c - prev[i];
        prev[i] = c;
        tot += d[i];
    }
    *n = tot;
    for (int k = 0; k < nq; ++k) {
        const uint64_t want = std::max<uint64_t>(1, (uint64_t)ceil(qs[k] * (double)tot));
        uint64_t cum = 0;
        out[k] = 0;
        for (int i = 0; i < LogHist::kBins && tot; ++i) {
            cum += d[i];
            if (cum >= want) {
                out[k] = LogHist::upper(i);
                break;
            }
        }
    }
}

void log_num(FILE *f, const char *key, double v, bool present) {
    if (present) fprintf(f, "\"%s\": %.6g", key, v);
    else fprintf(f, "\"%s\": null", key);
}

void log_line(hf_server *s, MetricsLog &L) {
    hf_server_stats st;
    if (hf_server_stats_get(s, &st) != HF_OK) return;
    const double t = now_ms();
    FILE *f = L.f;
    fprintf(f, "{\"t_s\": %.6f, \"period_s\": %.6f", (t - s->t0) * 1e-3, (t - L.t_last) * 1e-3);
    L.t_last = t;
    fprintf(f,
            ", \"submitted\": %lld, \"completed\": %lld, \"failed\": %lld, \"rejected\": %lld, "
            "\"superseded\": %lld, \"evicted\": %lld, \"queries\": %lld, \"rotations_completed\": %lld, "
            "\"queued\": %d, \"running\": %d, \"sessions\": %d, \"reserved_bytes\": %zu, \"budget_bytes\": %zu, "
            "\"chunks_submitted\": %lld, \"chunks_completed\": %lld, \"chunks_resident\": %d, "
            "\"pool_reserved_bytes\": %zu",
            (long long)st.submitted, (long long)st.completed, (long long)st.failed, (long long)st.rejected,
            (long long)st.superseded, (long long)st.evicted, (long long)st.queries, (long long)st.rotations_completed,
            st.queued, st.running, st.sessions, st.reserved_bytes, st.budget_bytes, (long long)st.chunks_submitted,
            (long long)st.chunks_completed, st.chunks_resident, st.pool_reserved_bytes);
    const double qs[3] = {0.5, 0.99, 0.999};
    double v[3];
    uint64_t n;
    hist_period(s->query_hist, L.prev_q, &n, qs, v, 3);
    const double qmax = s->query_hist.take_max();
    fprintf(f, ", \"query\": {\"n\": %llu, ", (unsigned long long)n);
    log_num(f, "p50_us", v[0], n > 0);
    fprintf(f, ", ");
    log_num(f, "p99_us", v[1], n > 0);
    fprintf(f, ", ");
    log_num(f, "p999_us", v[2], n > 0);
    fprintf(f, ", ");
    log_num(f, "max_us", qmax, n > 0);
    hist_period(s->build_hist, L.prev_b, &n, qs, v, 2);
    const double bmax = s->build_hist.take_max();
    fprintf(f, "}, \"build\": {\"n\": %llu, ", (unsigned long long)n);
    log_num(f, "p50_ms", v[0] * 1e-3, n > 0);
    fprintf(f, ", ");
    log_num(f, "p99_ms", v[1] * 1e-3, n > 0);
    fprintf(f, ", ");
    log_num(f, "max_ms", bmax * 1e-3, n > 0);
    fprintf(f, "}, \"session_queries\": [");
    bool first = true;
    for (int i = 0; i < s->nsessions.load(std::memory_order_acquire); ++i) {
        const Session &ss = s->sessions[i];
        if (!ss.open.load()) continue;
        fprintf(f, "%s[%d, %lld, %lld]", first ? "" : ", ", i, (long long)ss.answered.load(),
                (long long)ss.not_ready.load());
        first = false;
    }
    fprintf(f, "]}\n");
    fflush(f);
}

void log_run(hf_server *s, MetricsLog *L) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(L->mu);
    auto next = std::chrono::steady_clock::now();
    for (;;) {
        next += std::chrono::milliseconds(L->period_ms);
        if (L->cv.wait_until(lk, next, [&] { return L->stop; })) break;
        lk.unlock();
        log_line(s, *L);
        lk.lock();
    }
    lk.unlock();
    log_line(s, *L);  // the closing line covers the rest of the last period
}

// log_mu held
void log_stop(hf_server *s) {
    if (!s->log) return;
    MetricsLog &L = *s->log;
    {
        std::lock_guard<std::mutex> g(L.mu);
        L.stop = true;
    }
    L.cv.notify_all();
    if (L.th.joinable()) L.th.join();
    fclose(L.f);
    s->log.reset();
}

}  // namespace

extern "C" hf_status hf_server_log_open(hf_server *s, const char *path, int period_ms) {
    if (!s || !path) return srv_fail(HF_EINVAL, "hf_server_log_open: NULL argument");
    if (period_ms < 10) return srv_fail(HF_EINVAL, "hf_server_log_open: period %d ms (at least 10)", period_ms);
    std::lock_guard<std::mutex> g(s->log_mu);
    log_stop(s);
    FILE *f = fopen(path, "a");
    if (!f) return srv_fail(HF_EINVAL, "hf_server_log_open: cannot open %s", path);
    std::unique_ptr<MetricsLog> L(new MetricsLog());
    L->f = f;
    L->period_ms = period_ms;
    L->t_last = now_ms();
    for (int i = 0; i < LogHist::kBins; ++i) {  // the first period starts now
        L->prev_q[i] = s->query_hist.bin[i].load();
        L->prev_b[i] = s->build_hist.bin[i].load();
    }
    s->query_hist.take_max();
    s->build_hist.take_max();
    L->th = std::thread(log_run, s, L.get());
    s->log = std::move(L);
    return HF_OK;
}

extern "C" hf_status hf_server_log_close(hf_server *s) {
    if (!s) return srv_fail(HF_EINVAL, "hf_server_log_close: NULL server");
    std::lock_guard<std::mutex> g(s->log_mu);
    log_stop(s);
    return HF_OK;
}

// ------------------------------------------------- session checkpoints
// A session's published data (the request's rotations, its chunk routing and
// every resident chunk's field set) as NPY arrays, so that a restarted
// server serves it again without rebuilding.
extern "C" hf_status hf_server_session_save(hf_server *s, int session, const char *path) {
    if (!s || !path) return srv_fail(HF_EINVAL, "hf_server_session_save: NULL argument");
    Session *ss = session_at(s, session);
    if (!ss) return srv_fail(HF_EINVAL, "hf_server_session_save: session %d", session);
    std::shared_ptr<Published> cur = ss->current();
    if (!cur) return srv_fail(HF_ENOTREADY, "hf_server_session_save: session %d has no field data", session);
    const Request &r = *cur->req;
    std::vector<std::shared_ptr<SetHolder>> held(r.nchunks);  // kept alive while they are written
    std::vector<int64_t> present(r.nchunks), owner(r.owner.begin(), r.owner.end()), local(r.local.begin(), r.local.end());
    for (int c = 0; c < r.nchunks; ++c) {
        held[c] = cur->get(c);
        present[c] = held[c] ? 1 : 0;
    }
    cudaSetDevice(s->device);
    FILE *f = fopen(path, "wb");
    if (!f) return srv_fail(HF_EINVAL, "hf_server_session_save: cannot create %s", path);
    const std::vector<int64_t> meta = {hf_ckpt_magic(), hf_ckpt_version(), HF_CKPT_SESSION, r.n, r.R, r.flags,
                                       r.nchunks, 0};
    bool ok = hf_ckpt_write_i64(f, meta) && hf_ckpt_write_f32(f, {r.R, 4}, r.quats.data()) &&
              hf_ckpt_write_i64(f, owner) && hf_ckpt_write_i64(f, local) && hf_ckpt_write_i64(f, present);
    hf_status st = ok ? HF_OK : srv_fail(HF_EINVAL, "hf_server_session_save: write failed");
    cudaStream_t io = nullptr;
    if (st == HF_OK && cudaStreamCreateWithFlags(&io, cudaStreamNonBlocking) != cudaSuccess)
        st = srv_fail(HF_ECUDA, "hf_server_session_save: stream");
    for (int c = 0; c < r.nchunks && st == HF_OK; ++c)
        if (held[c]) st = hf_fieldset_write(held[c]->fs, f, io);
    if (io) cudaStreamDestroy(io);
    fclose(f);
    return st;
}

extern "C" hf_status hf_server_session_restore(hf_server *s, int session, const char *path) {
    if (!s || !path) return srv_fail(HF_EINVAL, "hf_server_session_restore: NULL argument");
    Session *ss = session_at(s, session);
    if (!ss) return srv_fail(HF_EINVAL, "hf_server_session_restore: session %d", session);
    cudaSetDevice(s->device);
    FILE *f = fopen(path, "rb");
    if (!f) return srv_fail(HF_EINVAL, "hf_server_session_restore: cannot open %s", path);
    std::vector<int64_t> meta, owner, local, present, shape;
    std::vector<float> quats;
    const bool ok = hf_ckpt_read_i64(f, meta) && meta.size() >= 8 && meta[0] == hf_ckpt_magic() &&
                    meta[1] == hf_ckpt_version() && meta[2] == HF_CKPT_SESSION;
    const int n = ok ? (int)meta[3] : 0, R = ok ? (int)meta[4] : 0, C = ok ? (int)meta[6] : 0;
    if (!ok || n != ss->n || R < 1 || C < 1 || !hf_ckpt_read_f32(f, shape, quats) ||
        shape != std::vector<int64_t>{R, 4} || !hf_ckpt_read_i64(f, owner) || (int)owner.size() != R ||
        !hf_ckpt_read_i64(f, local) || (int)local.size() != R || !hf_ckpt_read_i64(f, present) ||
        (int)present.size() != C) {
        fclose(f);
        return srv_fail(HF_EINVAL, "hf_server_session_restore: %s is not a session checkpoint for N=%d", path, ss->n);
    }
    auto r = std::make_shared<Request>();
    r->session = session;
    r->n = n;
    r->R = R;
    r->flags = (unsigned)meta[5];
    r->nchunks = C;
    r->quats = quats;
    r->owner.assign(owner.begin(), owner.end());
    r->local.assign(local.begin(), local.end());
    r->q.resize(4 * (size_t)R);
    for (int i = 0; i < R; ++i) {
        const float *v = &quats[4 * (size_t)i];
        const double w = v[0], x = v[1], y = v[2], z = v[3], nq = sqrt(w * w + x * x + y * y + z * z);
        double *o = &r->q[4 * (size_t)i];
        o[0] = w / nq; o[1] = x / nq; o[2] = y / nq; o[3] = z / nq;
    }
    for (int i = 0; i < R; ++i)
        if (r->owner[i] < 0 || r->owner[i] >= C) {
            fclose(f);
            return srv_fail(HF_EINVAL, "hf_server_session_restore: %s: bad chunk routing", path);
        }
    auto pub = std::make_shared<Published>(r);
    hf_status st = HF_OK;
    cudaStream_t io = nullptr;
    if (cudaStreamCreateWithFlags(&io, cudaStreamNonBlocking) != cudaSuccess)
        st = srv_fail(HF_ECUDA, "hf_server_session_restore: stream");
    for (int c = 0; c < C && st == HF_OK; ++c) {
        if (!present[c]) continue;
        hf_fieldset *fs = nullptr;
        st = hf_fieldset_read(s->ctx, f, &fs, nullptr, io);
        if (st != HF_OK) break;
        if (hf_fieldset_n(fs) != n || hf_fieldset_flags(fs) != (r->flags | HF_E | HF_F)) {
            hf_fieldset_release(fs);
            st = srv_fail(HF_EINVAL, "hf_server_session_restore: chunk %d does not match the session", c);
            break;
        }
        pub->last_use[c].store(now_ms());
        pub->set(c, std::make_shared<SetHolder>(fs, &s->graveyard, hf_fieldset_bytes(n, hf_fieldset_rotations(fs), r->flags)));
    }
    if (io) cudaStreamDestroy(io);
    fclose(f);
    if (st != HF_OK) return st;  // the sets loaded so far go to the graveyard with pub
    std::lock_guard<std::mutex> g(s->mu);
    r->id = s->next_id++;
    r->t_submit = r->t_done = now_ms();
    r->state = RQ_DONE;
    r->chunks_done = C;
    s->requests[r->id] = r;
    ss->set_current(pub);
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
