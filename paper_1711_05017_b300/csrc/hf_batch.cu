// hf_batch.cu -- many part pairs of uneven grid sizes built as one CUDA
// graph (the precompute of Section 4.2 for a whole scene at once).
//
// Every pair owns its rotation data on the device; its outputs go to a
// "slot" (a field set).  By default each pair has its own slot; when the
// outputs of all pairs exceed the device, pairs of the same grid size and
// rotation count share `slots_per_size` slots round-robin, and a slot then
// holds the last of its pairs after a launch (a streaming sink).  Capture
// records each slot's pairs in order on one of `lanes` branches forked from
// and joined into one capture stream; a launch of the graph runs the whole
// batch with one host call, slots on different branches overlapping on the
// device.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <utility>
#include <vector>

#include "hf.h"
#include "hf_internal.h"

namespace {
hf_status bfail(hf_status s, const char *msg) {
    hf::set_last_error(msg);
    return s;
}
}  // namespace

struct hf_batch {
    hf_ctx *ctx = nullptr;
    int npairs = 0;
    unsigned flags = 0;
    std::vector<const hf_part *> s1, s2;
    std::vector<int> R, n, slot_of;
    std::vector<hf_fieldset *> slots;
    std::vector<std::vector<int>> slot_pairs;  // pairs in launch order per slot
    std::vector<float *> d_rot9, d_P;
    std::vector<double *> d_P64;
    std::vector<int *> d_nbr;
    std::vector<char> have_rot;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> last_pair;  // per slot: the pair whose fields it holds after a launch
};

extern "C" void hf_batch_release(hf_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto p : b->d_rot9) cudaFree(p);
    for (auto p : b->d_P) cudaFree(p);
    for (auto p : b->d_P64) cudaFree(p);
    for (auto p : b->d_nbr) cudaFree(p);
    for (auto f : b->slots) hf_fieldset_release(f);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

extern "C" hf_status hf_batch_create(hf_ctx *ctx, int npairs, const hf_part *const *s1, const hf_part *const *s2,
                                     const int *R, unsigned flags, int slots_per_size, hf_batch **out) {
    if (!ctx || !out || npairs <= 0 || !s1 || !s2 || !R) return bfail(HF_EINVAL, "hf_batch_create: bad arguments");
    *out = nullptr;
    hf_batch *b = new hf_batch();
    b->ctx = ctx;
    b->npairs = npairs;
    b->flags = flags | HF_E | HF_F;
    b->s1.assign(s1, s1 + npairs);
    b->s2.assign(s2, s2 + npairs);
    b->R.assign(R, R + npairs);
    b->n.resize(npairs);
    b->slot_of.resize(npairs);
    std::map<std::pair<int, int>, std::vector<int>> size_slots;  // (n, R) -> slot ids
    std::map<std::pair<int, int>, int> seen;                     // (n, R) -> pairs so far
    for (int i = 0; i < npairs; ++i) {
        const int n = hf_part_n(s1[i]);
        if (n <= 0 || n != hf_part_n(s2[i]) || R[i] <= 0 || ((flags & HF_T) && R[i] < 7)) {
            hf_batch_release(b);
            return bfail(HF_EINVAL, "hf_batch_create: pair with mismatched parts or bad rotation count");
        }
        b->n[i] = n;
        const std::pair<int, int> key(n, R[i]);
        const int k = seen[key]++;
        auto &ss = size_slots[key];
        if (slots_per_size <= 0 || (int)ss.size() < slots_per_size) {
            ss.push_back((int)b->slot_pairs.size());
            b->slot_pairs.emplace_back();
        }
        const int slot = ss[slots_per_size <= 0 ? ss.size() - 1 : k % slots_per_size];
        b->slot_of[i] = slot;
        b->slot_pairs[slot].push_back(i);
    }
    if (cudaSetDevice(hf_ctx_device(ctx)) != cudaSuccess) {
        hf_batch_release(b);
        return bfail(HF_ECUDA, "hf_batch_create: cannot select the context's device");
    }
    const size_t ns = b->slot_pairs.size();
    b->slots.assign(ns, nullptr);
    b->last_pair.assign(ns, -1);
    hf_status st = HF_OK;
    for (size_t s = 0; s < ns && st == HF_OK; ++s) {
        const int p0 = b->slot_pairs[s][0];
        st = hf_fieldset_create(ctx, b->n[p0], b->R[p0], b->flags, &b->slots[s]);
    }
    cudaError_t e = cudaSuccess;
    b->d_rot9.assign(npairs, nullptr);
    b->d_P.assign(npairs, nullptr);
    b->d_P64.assign(npairs, nullptr);
    b->d_nbr.assign(npairs, nullptr);
    b->have_rot.assign(npairs, 0);
    for (int i = 0; i < npairs && st == HF_OK && e == cudaSuccess; ++i) {
        e = cudaMalloc(&b->d_rot9[i], (size_t)R[i] * 9 * sizeof(float));
        if (e == cudaSuccess && (flags & HF_T)) {
            e = cudaMalloc(&b->d_nbr[i], (size_t)R[i] * 6 * sizeof(int));
            if (e == cudaSuccess) e = cudaMalloc(&b->d_P[i], (size_t)R[i] * 18 * sizeof(float));
            if (e == cudaSuccess) e = cudaMalloc(&b->d_P64[i], (size_t)R[i] * 18 * sizeof(double));
        }
    }
    if (st == HF_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (st == HF_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    b->branch.assign(ns, nullptr);
    b->join.assign(ns, nullptr);
    for (size_t s = 0; s < ns && st == HF_OK && e == cudaSuccess; ++s) {
        e = cudaStreamCreateWithFlags(&b->branch[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming);
    }
    if (st != HF_OK || e != cudaSuccess) {
        hf_batch_release(b);
        if (st != HF_OK) return st;
        return bfail(e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "hf_batch_create: allocation failed");
    }
    *out = b;
    return HF_OK;
}

extern "C" hf_status hf_batch_set_rotations(hf_batch *b, int pair, const float *h_quat) {
    if (!b || !h_quat || pair < 0 || pair >= b->npairs) return bfail(HF_EINVAL, "hf_batch_set_rotations: bad arguments");
    if (cudaSetDevice(hf_ctx_device(b->ctx)) != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_set_rotations: device");
    std::vector<float> rot9, P32;
    std::vector<double> q64, P64;
    std::vector<int> nbr;
    const int R = b->R[pair];
    const int bad = hf_prepare_rotations(h_quat, R, (b->flags & HF_T) != 0, rot9, q64, nbr, P32, P64);
    if (bad < 0) return bfail(HF_EINVAL, "hf_batch_set_rotations: a quaternion is zero or not finite");
    // synchronous uploads: no graph launch may be in flight while rotations change
    cudaError_t e = cudaMemcpy(b->d_rot9[pair], rot9.data(), rot9.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && (b->flags & HF_T)) {
        e = cudaMemcpy(b->d_nbr[pair], nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_P[pair], P32.data(), P32.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_P64[pair], P64.data(), P64.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    // queries against a slot go to the pair it holds after a launch (its
    // last pair): that pair's quaternions are the slot's
    const int slot = b->slot_of[pair];
    if (e == cudaSuccess && b->slot_pairs[slot].back() == pair)
        e = cudaMemcpy(hf_fieldset_device_quats(b->slots[slot]), q64.data(), q64.size() * sizeof(double),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_set_rotations: upload failed");
    b->have_rot[pair] = 1;
    if (bad) return bfail(HF_EINVAL, "hf_batch_set_rotations: rank-deficient torque neighbourhood (NaN torque)");
    return HF_OK;
}

extern "C" hf_status hf_batch_capture(hf_batch *b, int lanes) {
    if (!b) return bfail(HF_EINVAL, "hf_batch_capture: NULL batch");
    for (int i = 0; i < b->npairs; ++i)
        if (!b->have_rot[i]) return bfail(HF_ENOTREADY, "hf_batch_capture: a pair has no rotations");
    if (cudaSetDevice(hf_ctx_device(b->ctx)) != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_capture: device");
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return bfail(HF_ECUDA, "hf_batch_capture: begin capture failed");
    // slot s runs on branch s % L; a branch's slots run one after another
    const int ns = (int)b->slots.size();
    const int L = lanes <= 0 ? ns : std::min(lanes, ns);
    hf_status st = HF_OK;
    if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) st = HF_ECUDA;
    for (int l = 0; l < L && st == HF_OK; ++l)
        if (cudaStreamWaitEvent(b->branch[l], b->fork, 0) != cudaSuccess) st = HF_ECUDA;
    for (int s = 0; s < ns && st == HF_OK; ++s) {
        for (int p : b->slot_pairs[s]) {
            st = hf_set_launch(b->ctx, b->s1[p], b->s2[p], b->slots[s], b->R[p], b->d_rot9[p], b->d_nbr[p],
                               b->d_P[p], b->d_P64[p], b->branch[s % L]);
            if (st != HF_OK) break;
        }
    }
    for (int l = 0; l < L && st == HF_OK; ++l)
        if (cudaEventRecord(b->join[l], b->branch[l]) != cudaSuccess ||
            cudaStreamWaitEvent(b->cap, b->join[l], 0) != cudaSuccess)
            st = HF_ECUDA;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != HF_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != HF_OK ? st : bfail(HF_ECUDA, "hf_batch_capture: end capture failed");
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_capture: instantiate failed");
    return HF_OK;
}

extern "C" hf_status hf_batch_launch(hf_batch *b, hf_stream stream) {
    if (!b || !b->exec) return bfail(HF_ENOTREADY, "hf_batch_launch: capture first");
    if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_launch: launch failed");
    for (size_t s = 0; s < b->slots.size(); ++s) {
        b->last_pair[s] = b->slot_pairs[s].back();
        hf_fieldset_mark_ready(b->slots[s]);
    }
    return HF_OK;
}

extern "C" hf_status hf_batch_fieldset(const hf_batch *b, int pair, const hf_fieldset **out) {
    if (!b || !out || pair < 0 || pair >= b->npairs) return bfail(HF_EINVAL, "hf_batch_fieldset: bad arguments");
    const int slot = b->slot_of[pair];
    if (b->last_pair[slot] != pair) return bfail(HF_ENOTREADY, "hf_batch_fieldset: the pair's slot holds another pair");
    *out = b->slots[slot];
    return HF_OK;
}

extern "C" int hf_batch_slots(const hf_batch *b) { return b ? (int)b->slots.size() : 0; }
