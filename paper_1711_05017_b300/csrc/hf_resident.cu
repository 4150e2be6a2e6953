// hf_resident.cu -- the host side of the resident query kernel
// (query_resident_kernel in hf_kernels.cu): mailboxes, the keeper thread that
// keeps instances queued, and the post-and-wait of one query.  Used by the
// server's query lanes and by a context's hf_query when enabled.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>

#include "hf.h"
#include "hf_internal.h"

namespace hf {

namespace {
double steady_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}
void cpu_relax() {
#if defined(__x86_64__) || defined(__i386__)
    __builtin_ia32_pause();
#endif
}
}  // namespace

bool ResidentQueries::start(int device, int lanes) {
    if (live() || lanes < 1 || lanes > 64) return false;
    device_ = device;
    lanes_ = lanes;
    cudaSetDevice(device);
    int lo = 0, hi = 0;
    const size_t bytes = 512 + sizeof(QueryMail) * (size_t)lanes;
    void *h = nullptr, *d = nullptr;
    bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess && hmalloc_mapped(&h, bytes) == cudaSuccess;
    if (ok) {
        h_ = (char *)h;
        memset(h, 0, bytes);
        ok = cudaHostGetDevicePointer(&d, h, 0) == cudaSuccess;
    }
    if (ok) {
        d_ = (char *)d;
        ok = dmalloc(&d_served_, sizeof(unsigned) * (size_t)lanes) == cudaSuccess &&
             cudaMemset(d_served_, 0, sizeof(unsigned) * (size_t)lanes) == cudaSuccess &&
             cudaStreamCreateWithPriority(&st_, cudaStreamNonBlocking, hi) == cudaSuccess &&
             cudaStreamSynchronize(st_) == cudaSuccess;
    }
    if (!ok) {
        (void)cudaGetLastError();
        stop();
        return false;
    }
    quit_.store(false);
    thread_ = std::thread(&ResidentQueries::keeper, this);
    // ready once the first instance is queued (or the keeper has given up)
    for (int i = 0; i < 2000 && !live() && !quit_.load(); ++i) std::this_thread::sleep_for(std::chrono::microseconds(500));
    if (live()) return true;
    stop();
    return false;
}

void ResidentQueries::stop() {
    quit_.store(true);
    if (thread_.joinable()) thread_.join();
    live_.store(false);
    if (st_) cudaStreamDestroy(st_);
    if (d_served_) cudaFree(d_served_);
    if (h_) cudaFreeHost(h_);
    st_ = nullptr;
    d_served_ = nullptr;
    h_ = d_ = nullptr;
}

// Keeps two instances queued on st_; on quit raises the stop flag and waits
// for them, so that none runs after it returns.
void ResidentQueries::keeper() {
    cudaSetDevice(device_);
    constexpr int kRing = 3;
    cudaEvent_t ev[kRing] = {};
    bool ok = true;
    for (auto &e : ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    auto *d_req = reinterpret_cast<unsigned *>(d_);
    auto *d_stop = reinterpret_cast<const unsigned *>(d_ + 256);
    auto *d_mail = reinterpret_cast<QueryMail *>(d_ + 512);
    int head = 0, queued = 0;
    while (ok && !quit_.load()) {
        if (queued < 2) {
            const int slot = (head + queued) % kRing;
            if (launch_query_resident(d_mail, d_req, d_served_, d_stop, lanes_, kLifeNs, st_) != cudaSuccess ||
                cudaEventRecord(ev[slot], st_) != cudaSuccess) {
                ok = false;
                break;
            }
            ++queued;
            live_.store(true, std::memory_order_release);
            continue;
        }
        const cudaError_t q = cudaEventQuery(ev[head]);
        if (q == cudaSuccess) {
            head = (head + 1) % kRing;
            --queued;
            continue;
        }
        if (q != cudaErrorNotReady) {
            ok = false;
            break;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(2));
    }
    live_.store(false, std::memory_order_release);
    quit_.store(true);
    (void)cudaGetLastError();
    __atomic_store_n(h_stop(), 1u, __ATOMIC_RELEASE);  // the running instance ends at its next poll
    cudaStreamSynchronize(st_);
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
}

bool ResidentQueries::query(int lane, const QueryReq &rq, unsigned *seq, float out7[7], double wait_ms,
                            double *posted_ms) {
    QueryMail *m = h_mail() + lane;
    m->rq = rq;
    unsigned s = *seq + 1;
    if (s == 0) s = 1;
    *seq = s;
    __atomic_store_n(h_req() + lane, s, __ATOMIC_RELEASE);
    const double posted = steady_ms();
    if (posted_ms) *posted_ms = posted;
    const double give_up = posted + wait_ms;
    for (unsigned spins = 1; __atomic_load_n(&m->done, __ATOMIC_ACQUIRE) != s; ++spins) {
        if ((spins & 255u) == 0 && steady_ms() > give_up) return false;
        cpu_relax();
    }
    for (int a = 0; a < 7; ++a) out7[a] = ((volatile float *)m->out)[a];
    return true;
}

bool ResidentQueries::answered(int lane, unsigned seq) const {
    return __atomic_load_n(&h_mail()[lane].done, __ATOMIC_ACQUIRE) == seq;
}

}  // namespace hf
