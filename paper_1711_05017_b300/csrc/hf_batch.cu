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
#include <deque>
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
    // the one-launch mode: the work-item table, its queue head, counters and
    // status word, and the per-size intermediates
    hf::PersistSeg *d_segs = nullptr;
    int *d_lut = nullptr;         // run holding item 256 i
    unsigned *d_queue = nullptr;  // [0] queue head, then the counters
    int *d_status = nullptr;
    std::vector<float2 *> scratch;
    int queue_items = 0, queue_runs = 0;
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
    if (b->d_segs) cudaFree(b->d_segs);
    if (b->d_lut) cudaFree(b->d_lut);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->d_status) cudaFree(b->d_status);
    for (auto p : b->scratch) cudaFree(p);
    for (auto s : b->branch) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto p : b->s1) hf_part_drop(p);
    for (auto p : b->s2) hf_part_drop(p);
    hf_ctx *c = b->ctx;
    delete b;
    hf_ctx_release(c);
}

extern "C" hf_status hf_batch_create(hf_ctx *ctx, int npairs, const hf_part *const *s1, const hf_part *const *s2,
                                     const int *R, unsigned flags, int slots_per_size, hf_batch **out) {
    if (!ctx || !out || npairs <= 0 || !s1 || !s2 || !R) return bfail(HF_EINVAL, "hf_batch_create: bad arguments");
    *out = nullptr;
    hf_batch *b = new hf_batch();
    b->ctx = ctx;
    hf_ctx_retain(ctx);
    b->npairs = npairs;
    b->flags = flags | HF_E | HF_F;
    b->s1.assign(s1, s1 + npairs);
    b->s2.assign(s2, s2 + npairs);
    for (int i = 0; i < npairs; ++i) {
        hf_part_retain(s1[i]);
        hf_part_retain(s2[i]);
    }
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
        e = hf::dmalloc(&b->d_rot9[i], (size_t)R[i] * 9 * sizeof(float));
        if (e == cudaSuccess && (flags & HF_T)) {
            e = hf::dmalloc(&b->d_nbr[i], (size_t)R[i] * 6 * sizeof(int));
            if (e == cudaSuccess) e = hf::dmalloc(&b->d_P[i], (size_t)R[i] * 18 * sizeof(float));
            if (e == cudaSuccess) e = hf::dmalloc(&b->d_P64[i], (size_t)R[i] * 18 * sizeof(double));
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
    hf::Range range_("hf_batch_capture");
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

// ------------------------------------------------------ one-launch mode
// The whole batch as one launch of the work-queue kernel (E + F, grids
// 64/96/128): every pair's rotations are cut into chunks; a chunk's pass A,
// B and C items form three runs, emitted with a lag (A of chunk k beside B of
// chunk k - 2 and C of chunk k - 4, in runs of kRun items taken in turn) so
// that different passes of different chunks share the device and a pass
// rarely waits for its producer.  Each grid size has kSlots intermediate
// slots; a chunk's pass A waits until the slot's previous chunk has finished
// pass C, and, when pairs share an output set, until the previous pair's
// same chunk has.
namespace {
constexpr int kSlots = 6, kLag = 2, kRun = 2048;
constexpr long long kDefaultSpin = 1LL << 21;  // polls of at least 256 ns each: about two seconds
}  // namespace

extern "C" hf_status hf_batch_capture_queue(hf_batch *b, int chunk, long long spin_limit, int self_test) {
    hf::Range range_("hf_batch_capture_queue");
    if (!b) return bfail(HF_EINVAL, "hf_batch_capture_queue: NULL batch");
    if (b->flags & ~(unsigned)(HF_E | HF_F))
        return bfail(HF_EUNSUPPORTED, "hf_batch_capture_queue: the one-launch build holds E and F only");
    for (int i = 0; i < b->npairs; ++i) {
        if (!b->have_rot[i]) return bfail(HF_ENOTREADY, "hf_batch_capture_queue: a pair has no rotations");
        if (b->n[i] != 64 && b->n[i] != 96 && b->n[i] != 128)
            return bfail(HF_EUNSUPPORTED, "hf_batch_capture_queue: grids of 64, 96 or 128 only");
        if (!hf_part_texture(b->s2[i]) || hf_part_role(b->s1[i]) != HF_STATIONARY ||
            hf_part_role(b->s2[i]) != HF_MOVING)
            return bfail(HF_EINVAL, "hf_batch_capture_queue: a pair's roles are wrong or its moving part has no texture");
    }
    if (chunk <= 0) chunk = 32;
    if (spin_limit <= 0) spin_limit = kDefaultSpin;
    if (cudaSetDevice(hf_ctx_device(b->ctx)) != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_capture_queue: device");
    cudaError_t e = hf::persist_init();
    if (e != cudaSuccess) return bfail(HF_ECUDA, "hf_batch_capture_queue: kernel set-up failed");
    // the previous graph reads the tables and intermediates freed below: it
    // goes first, so that a failure from here on leaves nothing to launch
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    // the pair-chunks, in pair order
    struct PC {
        int pair, n, r0, cnt, slot, cA, cB, cC;
    };
    std::vector<PC> pcs;
    std::map<int, int> per_size;  // n -> chunks so far
    for (int p = 0; p < b->npairs; ++p)
        for (int r0 = 0; r0 < b->R[p]; r0 += chunk) {
            PC c;
            c.pair = p;
            c.n = b->n[p];
            c.r0 = r0;
            c.cnt = std::min(chunk, b->R[p] - r0);
            c.slot = per_size[c.n]++ % kSlots;
            c.cA = 3 * (int)pcs.size();
            c.cB = c.cA + 1;
            c.cC = c.cA + 2;
            pcs.push_back(c);
        }
    // intermediates: per size, kSlots slots of X1, Y1, Y2 for `chunk` rotations
    for (auto p : b->scratch) cudaFree(p);
    b->scratch.clear();
    std::map<int, float2 *> base;
    for (auto &kv : per_size) {
        const int n = kv.first;
        const size_t he = (size_t)n * n * (n / 2 + 1);
        float2 *p = nullptr;
        e = hf::dmalloc(&p, (size_t)kSlots * 3 * chunk * he * sizeof(float2));
        if (e != cudaSuccess) return bfail(HF_ENOMEM, "hf_batch_capture_queue: intermediates");
        b->scratch.push_back(p);
        base[n] = p;
    }
    auto bt = [](int n) { return n * (n / 2 + 1) / 32; };  // pass B column tiles per rotation
    auto items = [&](const PC &c, int pass) { return (pass == 1 ? bt(c.n) : c.n) * c.cnt; };
    // dependencies of a chunk's pass A: the slot's previous chunk and the
    // previous pair in the same output set
    std::map<std::pair<int, int>, int> slot_last;     // (n, slot) -> pc index
    std::map<std::pair<int, int>, int> out_last;      // (output set, r0) -> pc index
    std::vector<int> depA0(pcs.size(), -1), depA1(pcs.size(), -1);
    for (size_t i = 0; i < pcs.size(); ++i) {
        const PC &c = pcs[i];
        auto k1 = std::make_pair(c.n, c.slot);
        if (slot_last.count(k1)) depA0[i] = slot_last[k1];
        slot_last[k1] = (int)i;
        auto k2 = std::make_pair(b->slot_of[c.pair], c.r0);
        if (out_last.count(k2) && pcs[out_last[k2]].pair != c.pair) depA1[i] = out_last[k2];
        out_last[k2] = (int)i;
    }
    // runs, emitted with the lag between passes
    std::vector<hf::PersistSeg> segs;
    int total = 0;
    auto make_runs = [&](int i, int pass, std::deque<hf::PersistSeg> &q) {
        const PC &c = pcs[i];
        const size_t he = (size_t)c.n * c.n * (c.n / 2 + 1);
        float2 *sb = base[c.n] + (size_t)c.slot * 3 * chunk * he;
        hf::PersistSeg g = {};
        g.pass = pass;
        g.n = c.n;
        g.dep[0] = g.dep[1] = -1;
        if (pass == 0) {
            if (depA0[i] >= 0) { g.dep[0] = pcs[depA0[i]].cC; g.dep_target[0] = items(pcs[depA0[i]], 2); }
            if (depA1[i] >= 0) { g.dep[1] = pcs[depA1[i]].cC; g.dep_target[1] = items(pcs[depA1[i]], 2); }
            g.done = c.cA;
        } else if (pass == 1) {
            g.dep[0] = c.cA;
            g.dep_target[0] = items(c, 0);
            g.done = c.cB;
        } else {
            g.dep[0] = c.cB;
            g.dep_target[0] = items(c, 1);
            g.done = c.cC;
        }
        g.rot9 = b->d_rot9[c.pair] + (size_t)9 * c.r0;
        g.tex = hf_part_texture(b->s2[c.pair]);
        g.box = hf_part_support(b->s2[c.pair]);
        g.R1hat = hf_part_spectrum(b->s1[c.pair]);
        g.X1 = sb;
        g.Y1 = sb + (size_t)chunk * he;
        g.Y2 = sb + 2 * (size_t)chunk * he;
        g.out = hf_fieldset_fields(b->slots[b->slot_of[c.pair]], c.r0);
        const int tot = items(c, pass);
        for (int f = 0; f < tot; f += kRun) {
            g.first = f;
            g.count = std::min(kRun, tot - f);
            q.push_back(g);
        }
    };
    // Emission by steps: in each step at most one chunk's pass A, one's pass B
    // and one's pass C, their runs taken in turn.  A pass is emitted only in
    // a step after every step holding a run it waits for, so each item's
    // producers hold smaller tickets: pass B of a chunk comes kLag steps after
    // its pass A, pass C kLag steps after its pass B (1 step when nothing else
    // can go), and pass A waits for the passes C its slot or output set
    // depend on.
    const int M = (int)pcs.size();
    std::vector<int> stepA(M, -1), stepB(M, -1), stepC(M, -1);
    int na = 0, nb = 0, nc = 0;
    for (int step = 0; nc < M; ++step) {
        auto a_ok = [&](int k) {
            for (int d : {depA0[k], depA1[k]})
                if (d >= 0 && (stepC[d] < 0 || stepC[d] >= step)) return false;
            return true;
        };
        const bool doA = na < M && a_ok(na);
        bool doB = nb < na && step - stepA[nb] >= kLag;
        bool doC = nc < nb && step - stepB[nc] >= kLag;
        if (!doA && !doB && !doC) {  // nothing under the lag: the next pass that can go at all
            doB = nb < na && step - stepA[nb] >= 1;
            doC = nc < nb && step - stepB[nc] >= 1;
        }
        std::deque<hf::PersistSeg> qa, qb, qc;
        if (doA) { make_runs(na, 0, qa); stepA[na++] = step; }
        if (doB) { make_runs(nb, 1, qb); stepB[nb++] = step; }
        if (doC) { make_runs(nc, 2, qc); stepC[nc++] = step; }
        if (!doA && !doB && !doC) return bfail(HF_EINVAL, "hf_batch_capture_queue: no schedulable pass (internal)");
        while (!qa.empty() || !qb.empty() || !qc.empty()) {
            for (auto *q : {&qa, &qb, &qc}) {
                if (q->empty()) continue;
                hf::PersistSeg g = q->front();
                q->pop_front();
                g.base = total;
                total += g.count;
                segs.push_back(g);
            }
        }
    }
    if (self_test & 1) {
        // a wait that nothing satisfies: the first pass B run needs one item
        // more than its producer has, so it runs out its bounded wait
        for (auto &g : segs)
            if (g.pass == 1) {
                g.dep_target[0] += 1;
                break;
            }
    }
    // device tables
    std::vector<int> lut(((size_t)total + 255) / 256);
    for (size_t i = 0, r = 0; i < lut.size(); ++i) {
        while (r + 1 < segs.size() && segs[r + 1].base <= (int)(256 * i)) ++r;
        lut[i] = (int)r;
    }
    if (b->d_segs) cudaFree(b->d_segs);
    if (b->d_lut) cudaFree(b->d_lut);
    if (b->d_queue) cudaFree(b->d_queue);
    b->d_segs = nullptr;
    b->d_lut = nullptr;
    b->d_queue = nullptr;
    if (!b->d_status && hf::dmalloc(&b->d_status, sizeof(int)) != cudaSuccess)
        return bfail(HF_ENOMEM, "hf_batch_capture_queue: status word");
    const size_t ncount = 1 + 3 * pcs.size();
    if (hf::dmalloc(&b->d_segs, segs.size() * sizeof(hf::PersistSeg)) != cudaSuccess ||
        hf::dmalloc(&b->d_lut, lut.size() * sizeof(int)) != cudaSuccess ||
        hf::dmalloc(&b->d_queue, ncount * sizeof(unsigned)) != cudaSuccess)
        return bfail(HF_ENOMEM, "hf_batch_capture_queue: work tables");
    if (cudaMemcpy(b->d_segs, segs.data(), segs.size() * sizeof(hf::PersistSeg), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_lut, lut.data(), lut.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess)
        return bfail(HF_ECUDA, "hf_batch_capture_queue: upload failed");
    b->queue_items = total;
    b->queue_runs = (int)segs.size();
    // the graph: reset the queue head and counters, then the one launch
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return bfail(HF_ECUDA, "hf_batch_capture_queue: begin capture failed");
    e = cudaMemsetAsync(b->d_queue, 0, ncount * sizeof(unsigned), b->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->cap);
    if (e == cudaSuccess)
        e = hf::run_persistent(b->d_segs, b->d_lut, (int)segs.size(), total, b->d_queue, b->d_queue + 1, b->d_status,
                               spin_limit, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(HF_ECUDA, "hf_batch_capture_queue: capture failed");
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess)
        return bfail(HF_ECUDA, "hf_batch_capture_queue: instantiate failed");
    return HF_OK;
}

extern "C" hf_status hf_batch_status(hf_batch *b, hf_stream stream, int *items, int *runs) {
    if (!b) return bfail(HF_EINVAL, "hf_batch_status: NULL batch");
    if (items) *items = b->queue_items;
    if (runs) *runs = b->queue_runs;
    if (!b->d_status) return HF_OK;
    int st = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return bfail(HF_ECUDA, "hf_batch_status: read failed");
    if (st != hf::PERSIST_OK)
        return bfail(HF_ETIMEOUT, "hf_batch_status: a work item's wait ran out; the launch stopped early");
    return HF_OK;
}

extern "C" hf_status hf_batch_launch(hf_batch *b, hf_stream stream) {
    hf::Range range_("hf_batch_launch");
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
