// hf_api.cu -- the C ABI declared in include/hf.h: contexts, parts, field
// sets, budget accounting, the float64 host set-up of the rotation
// neighbourhoods for the torque, and the pose-query entry points.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "hf.h"
#include "hf_internal.h"

using hf::FieldPtrs;

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

static hf_status fail(hf_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

namespace hf {
void set_last_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }
bool pencil_n(int n) {
    static int forced = -1;
    if (forced < 0) {
        const char *e = getenv("HF_PIPELINE");
        forced = (e && e[0] == 'p') ? 1 : 0;
    }
    return n >= 256 || forced == 1;
}
}  // namespace hf

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
    } while (0)

// ------------------------------------------------------------------ handles
// (the stationary spectrum's x/y transforms are a kind of their own, so that
// the rotation passes' averages are the rotation passes' alone)
enum ProfKind { kSplat, kPassA, kPassB, kPassBFwd, kPassC, kTorque, kQuery, kResample, kYtc, kStatA, kProfKinds };
static const char *kProfNames[kProfKinds] = {"splat",  "passA", "passB",    "passB_fwd", "passC",
                                             "torque", "query", "resample", "y_tc",      "passA_stationary"};

struct Tune {  // the autotuner's choice for one grid size
    bool set = false;
    int chunk = 0;
    int pencil = 0;
    int tile_b = 0, tile_c = 0;  // launch-shape candidates of passes B and C (hf::run_passB/C)
    int lanes = 1;               // 2: alternate chunks over two streams, so passes of neighbouring chunks overlap
    double rot_per_s = 0;
};
static int tune_slot(int n) { return n == 32 ? 0 : n == 64 ? 1 : n == 96 ? 2 : n == 128 ? 3 : 4; }

struct hf_ctx {
    int device = 0;
    // The context lives while the caller's handle or any part, field set,
    // batch or server made from it does: each holds a reference, so the
    // objects can be released in any order (a garbage collector finalises
    // the members of a reference cycle in no particular order).
    std::atomic<int> refs{1};
    Tune tune[5];
    size_t budget = 0, reserved = 0;
    std::mutex mu;
    cudaStream_t qstream = nullptr;             // high-priority stream for hf_query
    float *h_qout = nullptr;  // mapped pinned 7-float answer mailbox
    float *d_qout = nullptr;  // its device alias
    std::mutex qmu;
    // hf_query through the resident query kernel when enabled (one lane), under qmu
    hf::ResidentQueries *res = nullptr;
    unsigned res_seq = 0;
    // single-pose low-pass scratch (partial sums and the pose counter), under qmu
    double *lp_part = nullptr;
    unsigned *lp_count = nullptr;
    // per-kernel timing
    bool prof = false;
    std::mutex pmu;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    long long launches[kProfKinds] = {};
    double ms[kProfKinds] = {};
};

struct hf_part {
    hf_ctx *ctx;  // must outlive the part
    int n, role;
    float *grid;   // HF_MOVING: N^3
    float2 *spec;  // HF_STATIONARY: (h^3/N^3) rho1^ in [kz*][ky*][kx*] slot order
    size_t bytes;
    // HF_MOVING: the grid as stacked padded z-slices in a gather-capable 2D
    // array, (N+1) wide and N(N+1) high, sampled by 2x2 texture gathers
    float *slab = nullptr;
    size_t slab_pitch = 0;  // bytes
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    // with the texture: the grid's support as cell intervals per axis (6 ints
    // after kSupportMaskWords words of mask scratch); the texture resample
    // issues no gathers for samples in cells outside it
    unsigned *supmask = nullptr;
    int *box = nullptr;
    // HF_MOVING after hf_part_spectral: the centred spectrum of rho2 padded to
    // table_os * N nodes per axis, full cube, natural order (spectral mode)
    float2 *table = nullptr;
    int table_os = 0;
    size_t table_bytes = 0;  // the table and its gather array
    // the table as a float2 gather texture of stacked, wrap-padded slices
    // (read by the spectral field build; the queries read the table itself)
    cudaArray_t tarr = nullptr;
    cudaTextureObject_t ttex = 0;
    // HF_STATIONARY after hf_part_moments: the spectra of the moment fields
    // G_a = -(u x grad rho1)_a, 3 half spectra (slot order, scaled like spec)
    float2 *mspec = nullptr;
    // the caller's handle, each server session over the part, each build in
    // flight and each batch holding it; freed with the last
    std::atomic<int> refs{1};
};

struct hf_fieldset {
    hf_ctx *ctx = nullptr;
    int n = 0, R = 0;
    unsigned flags = 0;
    int nf = 0;                  // fields held per rotation
    int slot[7];                 // field index -> slot within a rotation block, -1 if not held
    float *data = nullptr;       // R x nf x N^3
    // two pipelines, each with its own intermediates, run alternate chunks on
    // two internal streams so that one chunk's texture-bound resample can
    // overlap the other's shared-memory-bound passes
    float2 *scratch[2] = {};     // 3 x chunk x N*N*(N/2+1): X1, Y1, Y2
    cudaStream_t lane[2] = {};
    cudaEvent_t fork = nullptr, join[2] = {};
    float *d_rot9 = nullptr;     // R x 9
    double *d_quat = nullptr;    // R x 4 (normalised)
    int *d_nbr = nullptr;        // R x 6
    float *d_P = nullptr;        // R x 18
    double *d_P64 = nullptr;     // R x 18
    int chunk = 1;
    int tile_b = 0, tile_c = 0;  // launch shapes of passes B and C (autotuner)
    int lanes = 1;  // pipelines used by compute (HF_LANES=2 alternates chunks over two)
    bool pencil = false;  // pencil pipeline (x/y stages as separate kernels) instead of slab passes
    int prec = hf::PREC_FP32;  // y stages on the tensor cores (pencil pipeline at N = 256)
    bool spectral = false;     // rotated spectrum interpolated from the moving part's table
    bool torque_analytic = false;  // HF_TA: torque from the stationary moment spectra
    bool ready = false;
    size_t bytes = 0;
    cudaStream_t mem_stream = nullptr;  // non-null: stream-ordered device memory, pageable staging
    hf::Arena *arena = nullptr;  // non-null: the device memory is one range of this arena
    void *arena_block = nullptr;  // that range
    std::vector<char> pageable_stage;
    void *h_stage = nullptr;     // staging for the per-call uploads (pinned unless mem_stream)
    bool stage_owned_pinned = false;  // h_stage is the set's own pinned allocation
    size_t stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;  // the last uploads from h_stage have been consumed
    // the host preparation of the last rotation set (matrices, neighbours,
    // least-squares operators), reused while the quaternions are the same
    // bytes: a field set is typically recomputed over one rotation set as
    // the parts change
    std::vector<float> prep_quat, prep_rot9, prep_P32;
    std::vector<double> prep_q64, prep_P64;
    std::vector<int> prep_nbr;
    int prep_bad = -1;
};

static bool charge(hf_ctx *c, size_t b) {
    std::lock_guard<std::mutex> g(c->mu);
    if (c->budget && c->reserved + b > c->budget) return false;
    c->reserved += b;
    return true;
}
static void uncharge(hf_ctx *c, size_t b) {
    std::lock_guard<std::mutex> g(c->mu);
    c->reserved -= std::min(b, c->reserved);
}

static cudaEvent_t prof_event(hf_ctx *c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch `fn` on `st`, bracketed by timing events when the context profiles.
// A launch is checked with cudaGetLastError, so a stale non-sticky error left
// in this thread by an earlier unrelated call is cleared first.
template <class F>
static cudaError_t timed(hf_ctx *c, int kind, cudaStream_t st, F &&fn) {
    (void)cudaGetLastError();
    if (!c || !c->prof) return fn();
    // launches recorded into a graph are not timed: their events never run
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return fn();
    std::lock_guard<std::mutex> g(c->pmu);
    cudaEvent_t a = prof_event(c), b = prof_event(c);
    if (!a || !b) return fn();
    cudaEventRecord(a, st);
    cudaError_t e = fn();
    cudaEventRecord(b, st);
    c->pending.push_back({kind, a, b});
    return e;
}

extern "C" hf_status hf_profile_enable(hf_ctx *c, int on) {
    if (!c) return fail(HF_EINVAL, "hf_profile_enable: ctx is NULL");
    c->prof = on != 0;
    return HF_OK;
}

extern "C" int hf_profile_read(hf_ctx *c) {
    if (!c) return 0;
    std::lock_guard<std::mutex> g(c->pmu);
    cudaSetDevice(c->device);
    for (auto &r : c->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->launches[r.kind] += 1;
            c->ms[r.kind] += ms;
        }
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->pending.clear();
    return kProfKinds;
}

extern "C" hf_status hf_profile_entry(const hf_ctx *c, int i, const char **name, long long *launches,
                                      double *total_ms) {
    if (!c || i < 0 || i >= kProfKinds) return fail(HF_EINVAL, "hf_profile_entry: index %d", i);
    if (name) *name = kProfNames[i];
    if (launches) *launches = c->launches[i];
    if (total_ms) *total_ms = c->ms[i];
    return HF_OK;
}

extern "C" void hf_profile_reset(hf_ctx *c) {
    if (!c) return;
    hf_profile_read(c);
    std::lock_guard<std::mutex> g(c->pmu);
    for (int k = 0; k < kProfKinds; ++k) {
        c->launches[k] = 0;
        c->ms[k] = 0.0;
    }
}

// kernel shared-memory limits for entry points that take no context: once per device
static cudaError_t ensure_kernel_attrs() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    if (done[dev]) return cudaSuccess;
    for (int n : {32, 64, 96, 128, 256})
        if ((e = hf::fft_init_attrs(n)) != cudaSuccess) return e;
    if ((e = hf::set_tc_attrs()) != cudaSuccess) return e;
    done[dev] = true;
    return cudaSuccess;
}

extern "C" const char *hf_version(void) { return "hf 1.0 sm_103a"; }
extern "C" const char *hf_last_error(void) { return g_err; }

std::atomic<long long> hf::g_alloc_count{0}, hf::g_alloc_fail_at{0};

extern "C" void hf_inject_alloc_failure(long long nth, long long *count) {
    const long long c = hf::g_alloc_count.load();
    hf::g_alloc_fail_at.store(nth > 0 ? c + nth : 0);
    if (count) *count = c;
}

extern "C" hf_status hf_ctx_create(int device, size_t budget, hf_ctx **out) {
    if (!out) return fail(HF_EINVAL, "hf_ctx_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    CU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(HF_EINVAL, "hf_ctx_create: device %d of %d", device, ndev);
    CU(cudaSetDevice(device));
    hf_ctx *c = new (std::nothrow) hf_ctx();
    if (!c) return fail(HF_ENOMEM, "hf_ctx_create: host allocation");
    c->device = device;
    c->budget = budget;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->qstream, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaHostAlloc(&c->h_qout, 8 * sizeof(float), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c->d_qout, c->h_qout, 0);
    for (int n : {32, 64, 96, 128, 256})
        if (e == cudaSuccess) e = hf::fft_init_attrs(n);
    if (e == cudaSuccess) e = hf::set_tc_attrs();
    if (e != cudaSuccess) {
        hf_ctx_destroy(c);
        return fail(HF_ECUDA, "hf_ctx_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return HF_OK;
}

static void ctx_free(hf_ctx *c);
void hf_ctx_retain(hf_ctx *c) {
    if (c) c->refs.fetch_add(1);
}
void hf_ctx_release(hf_ctx *c) {
    if (c && c->refs.fetch_sub(1) == 1) ctx_free(c);
}

// the caller's handle goes; the context itself once its last object has
extern "C" void hf_ctx_destroy(hf_ctx *c) { hf_ctx_release(c); }

static void ctx_free(hf_ctx *c) {
    cudaSetDevice(c->device);
    delete c->res;  // stops its kernel
    if (c->qstream) cudaStreamDestroy(c->qstream);
    if (c->h_qout) cudaFreeHost(c->h_qout);
    if (c->lp_part) cudaFree(c->lp_part);
    if (c->lp_count) cudaFree(c->lp_count);
    hf_profile_read(c);
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    delete c;
}

extern "C" size_t hf_ctx_budget_bytes(const hf_ctx *c) { return c ? c->budget : 0; }

// Driver entry points for loading whole modules: resolved through the runtime
// (the library does not link the driver library itself).
namespace {
struct ModuleLoader {
    CUresult (*func_get_module)(CUmodule *, CUfunction) = nullptr;
    CUresult (*module_function_count)(unsigned int *, CUmodule) = nullptr;
    CUresult (*module_enumerate)(CUfunction *, unsigned int, CUmodule) = nullptr;
    CUresult (*func_load)(CUfunction) = nullptr;
    bool ok = false;
    ModuleLoader() {
        auto get = [](const char *name, void **fp) {
            cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
            return cudaGetDriverEntryPointByVersion(name, fp, 12040, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess && *fp;
        };
        ok = get("cuFuncGetModule", (void **)&func_get_module) &&
             get("cuModuleGetFunctionCount", (void **)&module_function_count) &&
             get("cuModuleEnumerateFunctions", (void **)&module_enumerate) && get("cuFuncLoad", (void **)&func_load);
        (void)cudaGetLastError();
    }
};
}  // namespace

extern "C" hf_status hf_ctx_preload(hf_ctx *ctx, int *loaded) {
    if (!ctx) return fail(HF_EINVAL, "hf_ctx_preload: NULL context");
    if (loaded) *loaded = 0;
    static ModuleLoader L;
    if (!L.ok) return fail(HF_EUNSUPPORTED, "hf_ctx_preload: the driver has no per-function loading");
    CU(cudaSetDevice(ctx->device));
    int total = 0;
    for (const void *anchor : {hf::module_anchor_fft(), hf::module_anchor_kernels(), hf::module_anchor_tc()}) {
        cudaFunction_t f = nullptr;
        CU(cudaGetFuncBySymbol(&f, anchor));
        CUmodule mod = nullptr;
        unsigned int count = 0;
        if (L.func_get_module(&mod, (CUfunction)f) != CUDA_SUCCESS || L.module_function_count(&count, mod) != CUDA_SUCCESS)
            return fail(HF_ECUDA, "hf_ctx_preload: the module of a kernel file");
        std::vector<CUfunction> fns(count);
        if (count && L.module_enumerate(fns.data(), count, mod) != CUDA_SUCCESS)
            return fail(HF_ECUDA, "hf_ctx_preload: enumerating a module's kernels");
        for (CUfunction fn : fns)
            if (L.func_load(fn) != CUDA_SUCCESS) return fail(HF_ECUDA, "hf_ctx_preload: loading a kernel");
        total += (int)count;
    }
    if (loaded) *loaded = total;
    return HF_OK;
}

extern "C" int hf_tc_timeouts(int reset) { return hf::tc_timeouts(reset != 0); }
extern "C" int hf_bulk_timeouts(int reset) { return hf::bulk_timeouts(reset != 0); }

extern "C" hf_status hf_bulk_selftest(int device, int plant, int *timeouts) {
    if (!timeouts) return fail(HF_EINVAL, "hf_bulk_selftest: timeouts is NULL");
    CU(cudaSetDevice(device));
    const int before = hf::bulk_timeouts(false);
    if (before < 0) return fail(HF_ECUDA, "hf_bulk_selftest: cannot read the counter");
    const int nb = hf::bulk_selftest_bytes();
    std::vector<unsigned char> h(nb), back(nb);
    for (int i = 0; i < nb; ++i) h[i] = (unsigned char)(i * 37 + 11);
    void *d = nullptr;
    CU(hf::dmalloc(&d, 2 * (size_t)nb));
    cudaError_t e = cudaMemcpy(d, h.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset((char *)d + nb, 0, nb);
    if (e == cudaSuccess) e = hf::run_bulk_selftest(d, (char *)d + nb, plant, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(back.data(), (char *)d + nb, nb, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(HF_ECUDA, "hf_bulk_selftest: %s", cudaGetErrorString(e));
    *timeouts = hf::bulk_timeouts(false) - before;
    if (!plant && (*timeouts != 0 || back != h)) return fail(HF_ECUDA, "hf_bulk_selftest: the copy did not arrive");
    return plant ? (*timeouts > 0 ? HF_ETIMEOUT : fail(HF_ECUDA, "hf_bulk_selftest: the planted wait completed"))
                 : HF_OK;
}

extern "C" size_t hf_ctx_reserved_bytes(const hf_ctx *c) {
    if (!c) return 0;
    std::lock_guard<std::mutex> g(const_cast<hf_ctx *>(c)->mu);
    return c->reserved;
}

// ------------------------------------------------------------------ density
extern "C" hf_status hf_density_build(hf_ctx *ctx, int n, const float *d_pts, const float *d_sigma,
                                      const float *d_amp, int P, float *d_grid_out, hf_stream stream) {
    hf::Range range_("hf_density_build");
    if (!ctx) return fail(HF_EINVAL, "hf_density_build: ctx is NULL");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_density_build: N=%d not supported", n);
    if (P < 0 || !d_grid_out || (P > 0 && (!d_pts || !d_sigma)))
        return fail(HF_EINVAL, "hf_density_build: bad arguments (P=%d)", P);
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    CU(timed(ctx, kSplat, st, [&] { return hf::run_splat(n, d_pts, d_sigma, d_amp, P, d_grid_out, st); }));
    return HF_OK;
}

extern "C" hf_status hf_density_mesh(hf_ctx *ctx, int n, const double *d_V, int nv, const int *d_T, int nt,
                                     double sigma, double gamma_max, int max_depth, float *d_grid_out,
                                     float *d_aux_out, hf_stream stream) {
    hf::Range range_("hf_density_mesh");
    if (!ctx || !d_V || !d_T || !d_grid_out) return fail(HF_EINVAL, "hf_density_mesh: NULL argument");
    if (n < 2 || n > 512) return fail(HF_EUNSUPPORTED, "hf_density_mesh: N=%d outside 2..512", n);
    if (nv < 3 || nt < 1) return fail(HF_EINVAL, "hf_density_mesh: %d vertices, %d triangles", nv, nt);
    if (!(sigma > 0) || !(gamma_max > 0) || max_depth < 0 || max_depth > 12)
        return fail(HF_EINVAL, "hf_density_mesh: sigma, gamma_max > 0 and 0 <= max_depth <= 12 required");
    CU(cudaSetDevice(ctx->device));
    // every index must name a vertex: checked on the host before any kernel reads them
    std::vector<int> tri((size_t)3 * nt);
    CU(cudaMemcpy(tri.data(), d_T, tri.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int v : tri)
        if (v < 0 || v >= nv) return fail(HF_EINVAL, "hf_density_mesh: triangle index %d outside 0..%d", v, nv - 1);
    (void)cudaGetLastError();
    CU(hf::run_mesh_sdf(n, d_V, d_T, nt, sigma, gamma_max, max_depth, d_grid_out, d_aux_out, (cudaStream_t)stream));
    return HF_OK;
}

// --------------------------------------------------------------------- parts
static hf_status stationary_spectrum(hf_ctx *c, int n, const float *d_grid, float2 *spec, float scale,
                                     cudaStream_t st) {
    // pass A with the identity: a plain copy of each plane into the transform
    const size_t he = hf::half_spec_elems(n);
    float2 *X1 = nullptr;
    CU(hf::dmalloc_async(&X1, 2 * he * sizeof(float2), st));
    cudaError_t e;
    if (hf::pencil_n(n)) {
        e = timed(c, kStatA, st, [&] { return hf::run_xfwd(n, d_grid, X1 + he, 1, st); });
        if (e == cudaSuccess) e = timed(c, kStatA, st, [&] { return hf::run_yfwd(n, X1 + he, X1, 1, st); });
    } else {
        e = timed(c, kStatA, st, [&] { return hf::run_passA_planes(n, d_grid, X1, 1, st); });
    }
    if (e == cudaSuccess) e = timed(c, kPassBFwd, st, [&] { return hf::run_passB_forward(n, X1, spec, scale, st); });
    const cudaError_t f = cudaFreeAsync(X1, st);
    if (e == cudaSuccess) e = f;
    if (e != cudaSuccess) return fail(HF_ECUDA, "stationary spectrum: %s", cudaGetErrorString(e));
    return HF_OK;
}

// (h^3 / N^3) in float64: the Riemann-sum volume element of Eq. 1 and the
// inverse transform's normalisation, rounded once
static float spectrum_scale(int n) {
    const double h = 2.0 / n;
    return (float)(h * h * h / ((double)n * n * n));
}

static hf_status spectral_table_fill(hf_part *p, const float *d_grid, cudaStream_t st);
static hf_status moment_spectra_fill(hf_part *p, cudaStream_t st);

static hf_status part_fill(hf_part *p, const float *d_grid, cudaStream_t st) {
    if (p->role == HF_MOVING && p->table) {
        const hf_status s = spectral_table_fill(p, d_grid, st);
        if (s != HF_OK) return s;
    }
    if (p->role == HF_MOVING) {
        const int n = p->n;
        CU(cudaMemcpyAsync(p->grid, d_grid, (size_t)n * n * n * sizeof(float), cudaMemcpyDeviceToDevice, st));
        if (p->arr) {
            int tw = 0, th = 0;
            hf::tex_layout(n, &tw, &th);
            CU(hf::run_pad_slices(n, d_grid, p->slab, p->slab_pitch / sizeof(float), st));
            CU(cudaMemcpy2DToArrayAsync(p->arr, 0, 0, p->slab, p->slab_pitch, (size_t)tw * sizeof(float), (size_t)th,
                                        cudaMemcpyDeviceToDevice, st));
            if (p->box) CU(hf::run_support(n, d_grid, p->supmask, p->box, st));
        }
        return HF_OK;
    }
    hf_status s = stationary_spectrum(p->ctx, p->n, d_grid, p->spec, spectrum_scale(p->n), st);
    if (s == HF_OK && p->mspec) s = moment_spectra_fill(p, st);
    return s;
}

static void moving_texture_free(hf_part *p) {
    if (p->tex) cudaDestroyTextureObject(p->tex);
    if (p->arr) cudaFreeArray(p->arr);
    if (p->slab) cudaFree(p->slab);
    if (p->supmask) cudaFree(p->supmask);
    p->tex = 0;
    p->arr = nullptr;
    p->slab = nullptr;
    p->supmask = nullptr;
    p->box = nullptr;
}

// the gather-capable array + texture object of a moving part; when the device
// cannot hold the stacked slices in one gather array, the part keeps only the
// plain grid and the resample reads it with ordinary loads
static hf_status moving_texture_alloc(hf_part *p) {
    const int n = p->n;
    int maxw = 0, maxh = 0, tw = 0, th = 0;
    hf::tex_layout(n, &tw, &th);
    if (cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DGatherWidth, p->ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DGatherHeight, p->ctx->device) != cudaSuccess ||
        tw > maxw || th > maxh)
        return HF_OK;
    const size_t w = (size_t)tw, h = (size_t)th;
    cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
    CU(hf::dmalloc_pitch(&p->slab, &p->slab_pitch, w * sizeof(float), h));
    cudaError_t e = hf::dmalloc_array(&p->arr, &fd, w, h, cudaArrayTextureGather);
    if (e == cudaSuccess) {
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = p->arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = cudaAddressModeClamp;
        td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        e = cudaCreateTextureObject(&p->tex, &rd, &td, nullptr);
    }
    const char *sup = getenv("HF_SUPPORT");
    if (e == cudaSuccess && !(sup && sup[0] == '0')) {
        e = hf::dmalloc(&p->supmask, (hf::kSupportMaskWords + 6) * sizeof(unsigned));
        if (e == cudaSuccess) p->box = reinterpret_cast<int *>(p->supmask + hf::kSupportMaskWords);
    }
    if (e != cudaSuccess) {
        moving_texture_free(p);
        return fail(e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "hf_part_create: texture: %s",
                    cudaGetErrorString(e));
    }
    return HF_OK;
}

extern "C" hf_status hf_part_create(hf_ctx *ctx, int n, const float *d_grid, int role, hf_part **out,
                                    hf_stream stream) {
    hf::Range range_("hf_part_create");
    if (!ctx || !out || !d_grid) return fail(HF_EINVAL, "hf_part_create: NULL argument");
    *out = nullptr;
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_part_create: N=%d not supported", n);
    if (role != HF_STATIONARY && role != HF_MOVING) return fail(HF_EINVAL, "hf_part_create: role %d", role);
    if ((uintptr_t)d_grid % 8) return fail(HF_EINVAL, "hf_part_create: d_grid must be 8-byte aligned");
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n3 = (size_t)n * n * n;
    // moving: the grid plus the padded slices (pitched buffer and array) and
    // the support words
    int tw = 0, th = 0;
    hf::tex_layout(n, &tw, &th);
    const size_t bytes = role == HF_MOVING ? n3 * sizeof(float) + 2 * ((size_t)tw + 32) * th * sizeof(float) +
                                                 (hf::kSupportMaskWords + 6) * sizeof(unsigned)
                                           : hf::half_spec_elems(n) * sizeof(float2);
    if (!charge(ctx, bytes)) return fail(HF_EBUDGET, "hf_part_create: %zu bytes exceed the budget", bytes);
    hf_part *p = new (std::nothrow) hf_part{ctx, n, role, nullptr, nullptr, bytes};
    if (!p) {
        uncharge(ctx, bytes);
        return fail(HF_ENOMEM, "hf_part_create: host allocation");
    }
    void *mem = nullptr;
    cudaError_t e = hf::dmalloc(&mem, role == HF_MOVING ? n3 * sizeof(float) : bytes);
    if (e != cudaSuccess) {
        delete p;
        uncharge(ctx, bytes);
        return fail(HF_ENOMEM, "hf_part_create: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    if (role == HF_MOVING) p->grid = (float *)mem;
    else p->spec = (float2 *)mem;
    hf_status s = HF_OK;
    if (role == HF_MOVING) s = moving_texture_alloc(p);
    if (s == HF_OK) s = part_fill(p, d_grid, st);
    if (s != HF_OK) {
        moving_texture_free(p);
        cudaFree(mem);
        delete p;
        uncharge(ctx, bytes);
        return s;
    }
    hf_ctx_retain(ctx);
    *out = p;
    return HF_OK;
}

extern "C" int hf_part_n(const hf_part *p) { return p ? p->n : 0; }

extern "C" hf_status hf_part_update(hf_part *p, const float *d_grid, hf_stream stream) {
    if (!p || !d_grid) return fail(HF_EINVAL, "hf_part_update: NULL argument");
    if ((uintptr_t)d_grid % 8) return fail(HF_EINVAL, "hf_part_update: d_grid must be 8-byte aligned");
    CU(cudaSetDevice(p->ctx->device));
    return part_fill(p, d_grid, (cudaStream_t)stream);
}

// the centred, zero-padded spectrum of a moving part (Section 3.2: the
// moving spectrum is precomputed, then read at rotated frequencies)
static void table_free(hf_part *p) {
    if (p->ttex) cudaDestroyTextureObject(p->ttex);
    if (p->tarr) cudaFreeArray(p->tarr);
    if (p->table) cudaFree(p->table);
    if (p->table_bytes) uncharge(p->ctx, p->table_bytes);
    p->ttex = 0;
    p->tarr = nullptr;
    p->table = nullptr;
    p->table_bytes = 0;
}

static hf_status spectral_table_fill(hf_part *p, const float *d_grid, cudaStream_t st) {
    const int n = p->n, np = p->table_os * n;
    const size_t np3 = (size_t)np * np * np;
    float *pad = nullptr;
    float2 *half = nullptr;
    CU(hf::dmalloc_async(&pad, np3 * sizeof(float), st));
    cudaError_t e = hf::dmalloc_async(&half, hf::half_spec_elems(np) * sizeof(float2), st);
    hf_status s = HF_OK;
    if (e == cudaSuccess) e = hf::run_pad_center(n, d_grid, pad, np, st);
    if (e == cudaSuccess) s = stationary_spectrum(p->ctx, np, pad, half, 1.0f, st);
    if (e == cudaSuccess && s == HF_OK) e = hf::run_spectral_complete(np, half, p->table, st);
    if (pad) cudaFreeAsync(pad, st);
    if (half) cudaFreeAsync(half, st);
    if (e == cudaSuccess && s == HF_OK) {  // the gather texture, through a padded staging slab
        int w = 0, h = 0;
        hf::table_tex_layout(np, &w, &h);
        float2 *slab = nullptr;
        e = hf::dmalloc_async(&slab, (size_t)w * h * sizeof(float2), st);
        if (e == cudaSuccess) e = hf::run_pad_table(p->table, np, slab, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DToArrayAsync(p->tarr, 0, 0, slab, (size_t)w * sizeof(float2), (size_t)w * sizeof(float2),
                                         (size_t)h, cudaMemcpyDeviceToDevice, st);
        if (slab) cudaFreeAsync(slab, st);
    }
    if (s != HF_OK) return s;
    if (e != cudaSuccess) return fail(HF_ECUDA, "hf_part_spectral: %s", cudaGetErrorString(e));
    return HF_OK;
}

extern "C" hf_status hf_part_spectral(hf_part *p, int os, hf_stream stream) {
    hf::Range range_("hf_part_spectral");
    if (!p) return fail(HF_EINVAL, "hf_part_spectral: NULL part");
    if (p->role != HF_MOVING) return fail(HF_EINVAL, "hf_part_spectral: the part must be HF_MOVING");
    if (os != 1 && os != 2) return fail(HF_EINVAL, "hf_part_spectral: os must be 1 or 2 (%d)", os);
    if (!hf::supported_n(os * p->n))
        return fail(HF_EUNSUPPORTED, "hf_part_spectral: padded size %d not supported", os * p->n);
    CU(cudaSetDevice(p->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t np = (size_t)os * p->n, tbytes = np * np * np * sizeof(float2);
    int tw = 0, th = 0, maxw = 0, maxh = 0;
    hf::table_tex_layout((int)np, &tw, &th);
    if (cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DGatherWidth, p->ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DGatherHeight, p->ctx->device) != cudaSuccess ||
        tw > maxw || th > maxh)
        return fail(HF_EUNSUPPORTED, "hf_part_spectral: a %d x %d gather texture exceeds the device's limits", tw, th);
    const size_t bytes = tbytes + (size_t)tw * th * sizeof(float2);
    if (p->table && p->table_os != os) {
        CU(cudaStreamSynchronize(st));
        table_free(p);
    }
    if (!p->table) {
        if (!charge(p->ctx, bytes)) return fail(HF_EBUDGET, "hf_part_spectral: %zu bytes exceed the budget", bytes);
        p->table_bytes = bytes;
        cudaError_t e = hf::dmalloc(&p->table, tbytes);
        if (e != cudaSuccess) p->table = nullptr;
        if (e == cudaSuccess) {
            cudaChannelFormatDesc fd = cudaCreateChannelDesc<float2>();
            e = hf::dmalloc_array(&p->tarr, &fd, (size_t)tw, (size_t)th, cudaArrayTextureGather);
            if (e != cudaSuccess) p->tarr = nullptr;
        }
        if (e == cudaSuccess) {
            cudaResourceDesc rd = {};
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = p->tarr;
            cudaTextureDesc td = {};
            td.addressMode[0] = cudaAddressModeClamp;
            td.addressMode[1] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModePoint;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            e = cudaCreateTextureObject(&p->ttex, &rd, &td, nullptr);
            if (e != cudaSuccess) p->ttex = 0;
        }
        if (e != cudaSuccess) {
            table_free(p);
            return fail(e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "hf_part_spectral: %zu bytes: %s", bytes,
                        cudaGetErrorString(e));
        }
    }
    p->table_os = os;
    const hf_status s = spectral_table_fill(p, p->grid, st);
    if (s != HF_OK) {  // no half-filled table stays behind
        cudaStreamSynchronize(st);
        table_free(p);
    }
    return s;
}

extern "C" int hf_part_spectral_os(const hf_part *p) { return p && p->table ? p->table_os : 0; }

// The moment spectra of a stationary part (analytic torque): grad rho1 from
// the part's spectrum by the force passes against a unit delta at node 0
// (E = h^3 rho1, F = -h^3 grad rho1), the moment fields G = -(u x grad rho1),
// and their forward transforms scaled like the spectrum.  Pass B takes the
// moving density transformed along x and y only: for the delta that is 1 on
// the z = 0 plane and 0 elsewhere.
static hf_status moment_spectra_fill(hf_part *p, cudaStream_t st) {
    const int n = p->n;
    const size_t he = hf::half_spec_elems(n), n3 = (size_t)n * n * n;
    std::vector<float2> ones((size_t)n * (n / 2 + 1), make_float2(1.f, 0.f));  // the z = 0 plane
    float2 *sc = nullptr;  // delta spectrum, Y1, Y2
    float *fl = nullptr;   // E, Fx, Fy, Fz, then G (3 fields)
    CU(hf::dmalloc_async(&sc, 3 * he * sizeof(float2), st));
    cudaError_t e = hf::dmalloc_async(&fl, 7 * n3 * sizeof(float), st);
    hf_status s = HF_OK;
    if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, he * sizeof(float2), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sc, ones.data(), ones.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = hf::run_passB(n, sc, p->spec, sc + he, sc + 2 * he, 1, st);
    if (e == cudaSuccess) {
        FieldPtrs out{fl, fl + n3, fl + 2 * n3, fl + 3 * n3, 4 * n3};
        e = hf::run_passC(n, sc + he, sc + 2 * he, out, 1, st);
    }
    if (e == cudaSuccess) e = hf::run_moment_fields(n, fl + n3, fl + 2 * n3, fl + 3 * n3, fl + 4 * n3, st);
    for (int a = 0; a < 3 && e == cudaSuccess && s == HF_OK; ++a)
        s = stationary_spectrum(p->ctx, n, fl + (4 + a) * n3, p->mspec + a * he, spectrum_scale(n), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `ones` is pageable and lives here
    if (sc) cudaFreeAsync(sc, st);
    if (fl) cudaFreeAsync(fl, st);
    if (s != HF_OK) return s;
    if (e != cudaSuccess) return fail(HF_ECUDA, "hf_part_moments: %s", cudaGetErrorString(e));
    return HF_OK;
}

extern "C" hf_status hf_part_moments(hf_part *p, hf_stream stream) {
    hf::Range range_("hf_part_moments");
    if (!p) return fail(HF_EINVAL, "hf_part_moments: NULL part");
    if (p->role != HF_STATIONARY) return fail(HF_EINVAL, "hf_part_moments: the part must be HF_STATIONARY");
    if (p->n > 128) return fail(HF_EUNSUPPORTED, "hf_part_moments: N=%d (the analytic torque runs at N <= 128)", p->n);
    CU(cudaSetDevice(p->ctx->device));
    if (!p->mspec) {
        const size_t bytes = 3 * hf::half_spec_elems(p->n) * sizeof(float2);
        if (!charge(p->ctx, bytes)) return fail(HF_EBUDGET, "hf_part_moments: %zu bytes exceed the budget", bytes);
        const cudaError_t e = hf::dmalloc(&p->mspec, bytes);
        if (e != cudaSuccess) {
            p->mspec = nullptr;
            uncharge(p->ctx, bytes);
            return fail(HF_ENOMEM, "hf_part_moments: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
    }
    const hf_status s = moment_spectra_fill(p, (cudaStream_t)stream);
    if (s != HF_OK) {  // no half-filled moment spectra stay behind
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaFree(p->mspec);
        p->mspec = nullptr;
        uncharge(p->ctx, 3 * hf::half_spec_elems(p->n) * sizeof(float2));
    }
    return s;
}

void hf_part_retain(const hf_part *p) {
    if (p) const_cast<hf_part *>(p)->refs.fetch_add(1);
}

void hf_part_drop(const hf_part *p) { hf_part_release(const_cast<hf_part *>(p)); }

extern "C" void hf_part_release(hf_part *p) {
    if (!p || p->refs.fetch_sub(1) != 1) return;
    cudaSetDevice(p->ctx->device);
    table_free(p);
    if (p->mspec) {
        cudaFree(p->mspec);
        uncharge(p->ctx, 3 * hf::half_spec_elems(p->n) * sizeof(float2));
    }
    moving_texture_free(p);
    cudaFree(p->grid ? (void *)p->grid : (void *)p->spec);
    uncharge(p->ctx, p->bytes);
    hf_ctx *c = p->ctx;
    delete p;
    hf_ctx_release(c);
}

// ---------------------------------------------- rotation set-up (float64)
namespace {

struct Quat {
    double w, x, y, z;
};

Quat qnorm(const float *q) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double n = sqrt(w * w + x * x + y * y + z * z);
    return {w / n, x / n, y / n, z / n};
}

bool qfinite(const Quat &q) { return isfinite(q.w) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z); }

void rot_from_quat(const Quat &q, double R[9]) {
    const double w = q.w, x = q.x, y = q.y, z = q.z;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// axis-angle vector of R_j R_i^T, from the relative quaternion q_j * conj(q_i)
void rel_log(const Quat &qi, const Quat &qj, double v[3]) {
    const double w = qj.w * qi.w + qj.x * qi.x + qj.y * qi.y + qj.z * qi.z;
    double x = -qj.w * qi.x + qj.x * qi.w - qj.y * qi.z + qj.z * qi.y;
    double y = -qj.w * qi.y + qj.x * qi.z + qj.y * qi.w - qj.z * qi.x;
    double z = -qj.w * qi.z - qj.x * qi.y + qj.y * qi.x + qj.z * qi.w;
    double ww = w;
    if (ww < 0) { ww = -ww; x = -x; y = -y; z = -z; }
    const double s = sqrt(x * x + y * y + z * z);
    if (s < 1e-300) { v[0] = v[1] = v[2] = 0; return; }
    const double th = 2.0 * atan2(s, ww);
    v[0] = th * x / s;
    v[1] = th * y / s;
    v[2] = th * z / s;
}

// 6 nearest rotations by |q_i . q_j| (i.e. geodesic angle), ties to the lower index
void nearest6(const std::vector<Quat> &Q, int i, int nb[6]) {
    double bd[6];
    for (int s = 0; s < 6; ++s) { bd[s] = -1.0; nb[s] = -1; }
    const Quat &a = Q[i];
    for (int j = 0; j < (int)Q.size(); ++j) {
        if (j == i) continue;
        double d = fabs(a.w * Q[j].w + a.x * Q[j].x + a.y * Q[j].y + a.z * Q[j].z);
        if (d > 1.0) d = 1.0;
        if (d <= bd[5]) continue;
        int pos = 5;
        while (pos > 0 && d > bd[pos - 1]) --pos;
        for (int s = 5; s > pos; --s) { bd[s] = bd[s - 1]; nb[s] = nb[s - 1]; }
        bd[pos] = d;
        nb[pos] = j;
    }
}

// P = (A^T A)^{-1} A^T for the 6 x 3 A; false when A^T A is numerically singular
bool ls_pinv(const double A[6][3], double P[3][6]) {
    double N[3][3] = {};
    for (int s = 0; s < 6; ++s)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) N[r][c] += A[s][r] * A[s][c];
    double inv[3][3];
    inv[0][0] = N[1][1] * N[2][2] - N[1][2] * N[2][1];
    inv[0][1] = N[0][2] * N[2][1] - N[0][1] * N[2][2];
    inv[0][2] = N[0][1] * N[1][2] - N[0][2] * N[1][1];
    inv[1][0] = N[1][2] * N[2][0] - N[1][0] * N[2][2];
    inv[1][1] = N[0][0] * N[2][2] - N[0][2] * N[2][0];
    inv[1][2] = N[0][2] * N[1][0] - N[0][0] * N[1][2];
    inv[2][0] = N[1][0] * N[2][1] - N[1][1] * N[2][0];
    inv[2][1] = N[0][1] * N[2][0] - N[0][0] * N[2][1];
    inv[2][2] = N[0][0] * N[1][1] - N[0][1] * N[1][0];
    const double det = N[0][0] * inv[0][0] + N[0][1] * inv[1][0] + N[0][2] * inv[2][0];
    if (!(det != 0.0) || !isfinite(det)) return false;
    double fn = 0, fi = 0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            inv[r][c] /= det;
            fn += N[r][c] * N[r][c];
            fi += inv[r][c] * inv[r][c];
        }
    if (!isfinite(fi) || sqrt(fn) * sqrt(fi) > 1e16) return false;  // Frobenius condition of A^T A
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 6; ++s) P[r][s] = inv[r][0] * A[s][0] + inv[r][1] * A[s][1] + inv[r][2] * A[s][2];
    return true;
}

// neighbour indices and least-squares operators for every rotation; returns
// the number of rank-deficient rotations (their operator entries are NaN)
int torque_setup(const std::vector<Quat> &Q, std::vector<int> &nbr, std::vector<float> &P32,
                 std::vector<double> &P64, int *h_status) {
    const int R = (int)Q.size();
    nbr.assign((size_t)R * 6, 0);
    P32.assign((size_t)R * 18, 0.f);
    P64.assign((size_t)R * 18, 0.0);
    std::vector<char> deficient((size_t)R, 0);
    // rotation i's neighbours and operator depend on Q alone, so the O(R^2)
    // search splits over host threads by rotation with unchanged results
    auto rows = [&](int i0, int i1) {
        for (int i = i0; i < i1; ++i) {
            int nb[6];
            nearest6(Q, i, nb);
            double A[6][3], P[3][6];
            bool ok = true;
            for (int s = 0; s < 6; ++s) {
                if (nb[s] < 0) { ok = false; break; }
                rel_log(Q[i], Q[nb[s]], A[s]);
            }
            ok = ok && ls_pinv(A, P);
            for (int s = 0; s < 6; ++s) nbr[(size_t)6 * i + s] = nb[s] < 0 ? i : nb[s];
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 6; ++s) {
                    const double v = ok ? P[r][s] : NAN;
                    P64[(size_t)18 * i + 6 * r + s] = v;
                    P32[(size_t)18 * i + 6 * r + s] = (float)v;
                }
            deficient[i] = ok ? 0 : 1;
        }
    };
    const int hw = (int)std::thread::hardware_concurrency();
    const int nth = std::max(1, std::min({hw > 0 ? hw : 1, 16, R / 128}));
    if (nth == 1) {
        rows(0, R);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nth; ++t) pool.emplace_back(rows, (int)((long)R * t / nth), (int)((long)R * (t + 1) / nth));
        for (auto &th : pool) th.join();
    }
    int bad = 0;
    for (int i = 0; i < R; ++i) {
        if (h_status) h_status[i] = deficient[i];
        bad += deficient[i];
    }
    return bad;
}

int default_chunk(int n) {
    const char *env = getenv("HF_ROT_CHUNK");
    if (env && atoi(env) > 0) return atoi(env);
    switch (n) {  // rotations per launch: enough CTAs for several waves on 148 SMs
        case 32: return 256;
        case 64: return 128;
        case 96: return 48;
        case 256: return 4;
        default: return 32;
    }
}

// pass C's launch shape when the autotuner has not chosen one: at 64^3,
// 96^3 and 128^3 the bulk-staged form (tile 5; 256 threads per CTA at 128^3),
// else the built-in one
int default_tile_c(int n) { return n >= 64 && n <= 128 ? 5 : 0; }

}  // namespace

// -------------------------------------------------- rotation-set chunking
// A rotation set too large for one build is split into chunks that are built
// (and kept) separately.  Each chunk owns a compact group of rotations: the
// lowest-index unassigned rotation and its nearest unassigned ones by
// geodesic angle, added while the chunk's build set still fits max_build.
// With halo, the build set is the owned rotations plus their 6 nearest in
// the whole set, in global index order: the least-squares torque of an owned
// rotation then sees exactly the neighbours (and tie order) it has in the
// whole set, so its fields equal those of a build of the whole set.
extern "C" int hf_rotation_chunks(const float *h_quat, int R, int max_build, int halo, int *h_owner, int *h_offsets,
                                  int *h_build, int build_cap) {
    if (!h_quat || !h_owner || !h_offsets || !h_build || R < 1 || max_build < (halo ? 7 : 1) || build_cap < R)
        return -1;
    std::vector<Quat> Q((size_t)R);
    for (int r = 0; r < R; ++r) {
        Q[r] = qnorm(h_quat + 4 * (size_t)r);
        if (!qfinite(Q[r])) return -1;
    }
    std::vector<int> nb;
    if (halo) {
        if (R < 7) return -1;  // the torque needs 6 neighbours
        nb.assign((size_t)R * 6, 0);
        for (int i = 0; i < R; ++i) nearest6(Q, i, &nb[(size_t)6 * i]);
    }
    std::vector<char> assigned((size_t)R, 0), inb((size_t)R, 0);
    std::vector<std::pair<double, int>> order;
    int nchunks = 0, used = 0, left = R;
    h_offsets[0] = 0;
    while (left > 0) {
        int seed = 0;
        while (assigned[seed]) ++seed;
        order.clear();
        const Quat &a = Q[seed];
        for (int j = 0; j < R; ++j)
            if (!assigned[j]) order.push_back({-fabs(a.w * Q[j].w + a.x * Q[j].x + a.y * Q[j].y + a.z * Q[j].z), j});
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<double, int> &u, const std::pair<double, int> &v) { return u.first < v.first; });
        std::vector<int> members;
        int owned = 0;
        for (const auto &o : order) {
            const int j = o.second;
            int add[7], na = 0;
            if (!inb[j]) add[na++] = j;
            if (halo)
                for (int s = 0; s < 6; ++s) {
                    const int k = nb[(size_t)6 * j + s];
                    if (!inb[k]) add[na++] = k;
                }
            if (owned > 0 && (int)members.size() + na > max_build) break;
            for (int t = 0; t < na; ++t) {
                inb[add[t]] = 1;
                members.push_back(add[t]);
            }
            assigned[j] = 1;
            h_owner[j] = nchunks;
            ++owned;
            --left;
        }
        std::sort(members.begin(), members.end());
        if (used + (int)members.size() > build_cap) return -1;
        for (int m : members) {
            h_build[used++] = m;
            inb[m] = 0;
        }
        h_offsets[++nchunks] = used;
    }
    return nchunks;
}

// ---------------------------------------------------------------- fieldsets
static size_t fieldset_bytes(int n, int R, unsigned flags, int chunk, int lanes);
// intermediates per rotation: 3 half spectra for the slab passes, 5 for the pencil pipeline
static size_t fields_spectra(bool pencil) { return pencil ? 5 : 3; }

// h_stage_ext: caller-owned pinned staging for the per-compute uploads (used
// if at least the set's staging bytes; else the set makes its own); lanes:
// 1 or 2 pipelines, 0 for the context's choice; arena: where the device
// memory comes from when not null (EBUDGET when no free range fits)
static hf_status fieldset_create_impl(hf_ctx *ctx, int n, int R, unsigned flags, cudaStream_t mem_stream,
                                      hf_fieldset **out, void *h_stage_ext = nullptr, size_t h_stage_ext_bytes = 0,
                                      int lanes = 0, hf::Arena *arena = nullptr);

extern "C" hf_status hf_fieldset_create(hf_ctx *ctx, int n, int R, unsigned flags, hf_fieldset **out) {
    return fieldset_create_impl(ctx, n, R, flags, nullptr, out);
}

hf_status hf_fieldset_create_stream_ordered(hf_ctx *ctx, int n, int R, unsigned flags, cudaStream_t st,
                                            hf_fieldset **out, void *h_stage, size_t h_stage_bytes, int lanes,
                                            hf::Arena *arena) {
    return fieldset_create_impl(ctx, n, R, flags, st, out, h_stage, h_stage_bytes, lanes, arena);
}

static hf_status fieldset_create_impl(hf_ctx *ctx, int n, int R, unsigned flags, cudaStream_t mem_stream,
                                      hf_fieldset **out, void *h_stage_ext, size_t h_stage_ext_bytes, int lanes,
                                      hf::Arena *arena) {
    if (!ctx || !out) return fail(HF_EINVAL, "hf_fieldset_create: NULL argument");
    *out = nullptr;
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_fieldset_create: N=%d not supported", n);
    if (R <= 0) return fail(HF_EINVAL, "hf_fieldset_create: R=%d", R);
    flags |= HF_E | HF_F;  // energy and force are always held
    if ((flags & HF_T) && R < 7) return fail(HF_EINVAL, "hf_fieldset_create: torque needs R >= 7 (R=%d)", R);
    if ((flags & HF_T) && (flags & HF_TA))
        return fail(HF_EINVAL, "hf_fieldset_create: HF_T and HF_TA are alternatives");
    if ((flags & HF_TORQUE_F64) && (flags & HF_TORQUE_C))
        return fail(HF_EINVAL, "hf_fieldset_create: HF_TORQUE_F64 and HF_TORQUE_C are alternatives");
    if ((flags & HF_TA) && (n > 128 || (flags & HF_SPECTRAL)))
        return fail(HF_EUNSUPPORTED, "hf_fieldset_create: HF_TA needs N <= 128 and the spatial route");
    const unsigned precf = flags & (HF_PREC_SPLIT_BF16 | HF_PREC_SPLIT_F16);
    if (precf == (HF_PREC_SPLIT_BF16 | HF_PREC_SPLIT_F16))
        return fail(HF_EINVAL, "hf_fieldset_create: at most one precision flag");
    if (precf && n != 256) return fail(HF_EUNSUPPORTED, "hf_fieldset_create: split precision needs N=256 (N=%d)", n);
    CU(cudaSetDevice(ctx->device));
    hf_fieldset *fs = new (std::nothrow) hf_fieldset();
    if (!fs) return fail(HF_ENOMEM, "hf_fieldset_create: host allocation");
    fs->ctx = ctx;
    hf_ctx_retain(ctx);
    fs->n = n;
    fs->R = R;
    fs->flags = flags;
    int nf = 0;
    for (int f = 0; f < 7; ++f) fs->slot[f] = -1;
    fs->slot[0] = nf++;
    if (flags & HF_F)
        for (int f = 1; f <= 3; ++f) fs->slot[f] = nf++;
    if (flags & (HF_T | HF_TA))
        for (int f = 4; f <= 6; ++f) fs->slot[f] = nf++;
    fs->nf = nf;
    fs->torque_analytic = (flags & HF_TA) != 0;
    fs->pencil = hf::pencil_n(n);
    fs->prec = (flags & HF_PREC_SPLIT_F16) ? hf::PREC_SPLIT_F16 : (flags & HF_PREC_SPLIT_BF16) ? hf::PREC_SPLIT_BF16
                                                                                             : hf::PREC_FP32;
    fs->spectral = (flags & HF_SPECTRAL) != 0;
    fs->chunk = default_chunk(n);
    fs->tile_c = default_tile_c(n);
    {
        const Tune &t = ctx->tune[tune_slot(n)];
        const char *ev = getenv("HF_ROT_CHUNK");
        if (t.set && !(ev && atoi(ev) > 0)) {
            fs->chunk = t.chunk;
            fs->pencil = t.pencil || n >= 256;
            fs->tile_b = t.tile_b;
            fs->tile_c = t.tile_c;
        }
    }
    fs->chunk = std::min(fs->chunk, R);
    {
        const char *ev = getenv("HF_LANES");
        const Tune &t = ctx->tune[tune_slot(n)];
        fs->lanes = ev ? ((atoi(ev) == 2) ? 2 : 1) : (t.set && t.lanes == 2 ? 2 : 1);
        // the tuner times the spatial route; on the spectral route pass B reads
        // the table through the texture units, and two pipelines' gathers
        // contend (at os = 2 the build ran at half the rate)
        if (!ev && (flags & HF_SPECTRAL)) fs->lanes = 1;
        if (lanes == 1 || lanes == 2) fs->lanes = lanes;
    }
    const size_t n3 = (size_t)n * n * n;
    const size_t data_b = (size_t)R * nf * n3 * sizeof(float);
    const size_t scr_b = (fields_spectra(fs->pencil) + ((flags & HF_TA) ? 3 : 0)) * (size_t)fs->chunk *
                         hf::half_spec_elems(n) * sizeof(float2);
    fs->stage_bytes = (size_t)R * (9 * sizeof(float) + 4 * sizeof(double) + 6 * sizeof(int) + 18 * sizeof(float) +
                                   18 * sizeof(double));
    fs->bytes = data_b + fs->lanes * scr_b + fs->stage_bytes;
    if (!charge(ctx, fs->bytes)) {
        const size_t b = fs->bytes;
        delete fs;
        hf_ctx_release(ctx);
        return fail(HF_EBUDGET, "hf_fieldset_create: %zu bytes exceed the budget", b);
    }
    fs->mem_stream = mem_stream;
    fs->arena = arena;
    // from an arena: one range for all the set's device arrays, carved in the
    // order they are allocated below (each on 256 bytes), so that a set frees
    // one contiguous range
    bool arena_short = false;
    size_t carve = 0, carve_end = 0;
    if (arena) {
        const size_t a = hf::Arena::kAlign;
        auto up = [&](size_t b) { return (b + a - 1) / a * a; };
        size_t total = up(data_b) + fs->lanes * up(scr_b) + up((size_t)R * 9 * sizeof(float)) +
                       up((size_t)R * 4 * sizeof(double)) + up((size_t)R * 6 * sizeof(int)) +
                       up((size_t)R * 18 * sizeof(float)) + up((size_t)R * 18 * sizeof(double));
        if (!hf::alloc_fails()) {  // (an injected failure is an allocation error, not a short arena)
            fs->arena_block = arena->alloc(total);
            arena_short = !fs->arena_block;
        }
        carve = (size_t)fs->arena_block;
        carve_end = carve + total;
    }
    auto dalloc = [&](void **p, size_t b) {
        if (arena) {
            if (!fs->arena_block) return cudaErrorMemoryAllocation;
            const size_t len = (b + hf::Arena::kAlign - 1) / hf::Arena::kAlign * hf::Arena::kAlign;
            if (carve + len > carve_end) return cudaErrorMemoryAllocation;
            *p = (void *)carve;
            carve += len;
            return cudaSuccess;
        }
        return mem_stream ? hf::dmalloc_async(p, b, mem_stream) : hf::dmalloc(p, b);
    };
    cudaError_t e = dalloc((void **)&fs->data, data_b);
    for (int l = 0; l < fs->lanes; ++l) {
        if (e == cudaSuccess) e = dalloc((void **)&fs->scratch[l], scr_b);
        // the pipelines' own streams and events only with two of them
        if (e == cudaSuccess && fs->lanes == 2) e = cudaStreamCreateWithFlags(&fs->lane[l], cudaStreamNonBlocking);
        if (e == cudaSuccess && fs->lanes == 2) e = cudaEventCreateWithFlags(&fs->join[l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && fs->lanes == 2) e = cudaEventCreateWithFlags(&fs->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dalloc((void **)&fs->d_rot9, (size_t)R * 9 * sizeof(float));
    if (e == cudaSuccess) e = dalloc((void **)&fs->d_quat, (size_t)R * 4 * sizeof(double));
    if (e == cudaSuccess) e = dalloc((void **)&fs->d_nbr, (size_t)R * 6 * sizeof(int));
    if (e == cudaSuccess) e = dalloc((void **)&fs->d_P, (size_t)R * 18 * sizeof(float));
    if (e == cudaSuccess) e = dalloc((void **)&fs->d_P64, (size_t)R * 18 * sizeof(double));
    if (e == cudaSuccess) {
        if (h_stage_ext && h_stage_ext_bytes >= fs->stage_bytes) {
            fs->h_stage = h_stage_ext;  // the caller's pinned buffer
        } else if (mem_stream) {
            fs->pageable_stage.resize(fs->stage_bytes + 64);
            fs->h_stage = fs->pageable_stage.data();
        } else {
            e = hf::hmalloc(&fs->h_stage, fs->stage_bytes);
            fs->stage_owned_pinned = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fs->stage_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        hf_fieldset_release(fs);
        if (arena_short)  // within the budget, but no free range of the arena is large enough
            return fail(HF_EBUDGET, "hf_fieldset_create: no free arena range of the size needed");
        return fail(e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "hf_fieldset_create: %s",
                    cudaGetErrorString(e));
    }
    *out = fs;
    return HF_OK;
}

static size_t fieldset_bytes(int n, int R, unsigned flags, int chunk, int lanes) {
    const int nf = 4 + ((flags & (HF_T | HF_TA)) ? 3 : 0);
    const size_t n3 = (size_t)n * n * n;
    const size_t scr_b = (fields_spectra(hf::pencil_n(n)) + ((flags & HF_TA) ? 3 : 0)) * (size_t)chunk *
                         hf::half_spec_elems(n) * sizeof(float2);
    const size_t stage = (size_t)R * (9 * sizeof(float) + 4 * sizeof(double) + 6 * sizeof(int) + 18 * sizeof(float) +
                                      18 * sizeof(double));
    return (size_t)R * nf * n3 * sizeof(float) + lanes * scr_b + stage;
}

extern "C" size_t hf_fieldset_bytes(int n, int R, unsigned flags) {
    if (!hf::supported_n(n) || R <= 0) return 0;
    return fieldset_bytes(n, R, flags, std::min(default_chunk(n), R), 1);
}

// For stream-ordered sets the caller guarantees no work still uses the set;
// the frees are then ordered on the set's memory stream without a device-wide
// synchronisation.
extern "C" void hf_fieldset_release(hf_fieldset *fs) {
    if (!fs) return;
    cudaSetDevice(fs->ctx->device);
    auto dfree = [&](void *p) {
        if (!p || fs->arena) return;  // an arena set frees its one range below
        if (fs->mem_stream) cudaFreeAsync(p, fs->mem_stream);
        else cudaFree(p);
    };
    dfree(fs->data);
    for (int l = 0; l < 2; ++l) {
        dfree(fs->scratch[l]);
        if (fs->lane[l]) cudaStreamDestroy(fs->lane[l]);
        if (fs->join[l]) cudaEventDestroy(fs->join[l]);
    }
    if (fs->fork) cudaEventDestroy(fs->fork);
    dfree(fs->d_rot9);
    dfree(fs->d_quat);
    dfree(fs->d_nbr);
    dfree(fs->d_P);
    dfree(fs->d_P64);
    if (fs->arena_block) fs->arena->release(fs->arena_block);
    if (fs->stage_owned_pinned) cudaFreeHost(fs->h_stage);
    if (fs->stage_done) cudaEventDestroy(fs->stage_done);
    uncharge(fs->ctx, fs->bytes);
    hf_ctx *c = fs->ctx;
    delete fs;
    hf_ctx_release(c);
}

int hf_ctx_device(const hf_ctx *c) { return c ? c->device : 0; }
bool hf_fieldset_is_ready(const hf_fieldset *fs) { return fs && fs->ready; }
const void *hf_fieldset_arena_block(const hf_fieldset *fs) { return fs ? fs->arena_block : nullptr; }
void hf_fieldset_mark_ready(hf_fieldset *fs) { fs->ready = true; }
double *hf_fieldset_device_quats(hf_fieldset *fs) { return fs->d_quat; }
hf::FieldPtrs hf_fieldset_fields(hf_fieldset *fs, int rot) {
    const size_t n3 = (size_t)fs->n * fs->n * fs->n, rs = (size_t)fs->nf * n3;
    float *base = fs->data + (size_t)rot * rs;
    return hf::FieldPtrs{base, base + n3, base + 2 * n3, base + 3 * n3, rs};
}
cudaTextureObject_t hf_part_texture(const hf_part *p) { return p->tex; }
const int *hf_part_support(const hf_part *p) { return p->box; }
const float2 *hf_part_spectrum(const hf_part *p) { return p->spec; }
int hf_part_role(const hf_part *p) { return p->role; }

extern "C" int hf_fieldset_n(const hf_fieldset *fs) { return fs ? fs->n : 0; }
extern "C" int hf_fieldset_rotations(const hf_fieldset *fs) { return fs ? fs->R : 0; }
extern "C" unsigned hf_fieldset_flags(const hf_fieldset *fs) { return fs ? fs->flags : 0u; }

// the energy/force passes for `cnt` rotations whose float matrices are at
// rot9 (cnt x 9, device); outputs through `out` (first rotation at out.E)
static hf_status run_fields(hf_ctx *c, int n, bool pencil, int prec, const hf_part *s1, const hf_part *s2,
                            const float *rot9, int cnt, float2 *scratch, size_t scratch_rot, float *planes,
                            FieldPtrs out, cudaStream_t st, bool spectral = false, int tile_b = 0, int tile_c = 0) {
    float2 *X1 = scratch, *Y1 = scratch + scratch_rot, *Y2 = scratch + 2 * scratch_rot;
    if (spectral) {
        CU(timed(c, kPassB, st, [&] {
            return hf::run_passB_spectral(n, s2->table, s2->ttex, s2->table_os, rot9, s1->spec, Y1, Y2, cnt, st);
        }));
        if (pencil) {
            float2 *A = scratch + 3 * scratch_rot, *B = scratch + 4 * scratch_rot;
            if (prec != hf::PREC_FP32)
                CU(timed(c, kYtc, st, [&] { return hf::run_yinv_tc(n, prec, Y1, Y2, A, X1, B, cnt, st); }));
            else
                CU(timed(c, kPassC, st, [&] { return hf::run_yinv(n, Y1, Y2, A, X1, B, cnt, st); }));
            CU(timed(c, kPassC, st, [&] { return hf::run_xinv(n, A, X1, B, out, cnt, st); }));
        } else {
            CU(timed(c, kPassC, st, [&] { return hf::run_passC(n, Y1, Y2, out, cnt, st); }));
        }
        return HF_OK;
    }
    if (pencil) {
        float2 *A = scratch + 3 * scratch_rot, *B = scratch + 4 * scratch_rot;
        if (s2->tex) {  // resample fused into the x forward through the texture units
            CU(timed(c, kPassA, st, [&] { return hf::run_xfwd_tex(n, s2->tex, s2->box, rot9, A, cnt, st); }));
        } else {
            if (!planes) return fail(HF_EUNSUPPORTED, "field-set build: the moving part has no texture");
            CU(timed(c, kResample, st, [&] { return hf::run_resample_chunk(n, s2->grid, rot9, planes, cnt, st); }));
            CU(timed(c, kPassA, st, [&] { return hf::run_xfwd(n, planes, A, cnt, st); }));
        }
        if (prec != hf::PREC_FP32)
            CU(timed(c, kYtc, st, [&] { return hf::run_yfwd_tc(n, prec, A, X1, cnt, st); }));
        else
            CU(timed(c, kPassA, st, [&] { return hf::run_yfwd(n, A, X1, cnt, st); }));
        CU(timed(c, kPassB, st, [&] { return hf::run_passB(n, X1, s1->spec, Y1, Y2, cnt, st); }));
        if (prec != hf::PREC_FP32)
            CU(timed(c, kYtc, st, [&] { return hf::run_yinv_tc(n, prec, Y1, Y2, A, X1, B, cnt, st); }));
        else
            CU(timed(c, kPassC, st, [&] { return hf::run_yinv(n, Y1, Y2, A, X1, B, cnt, st); }));
        CU(timed(c, kPassC, st, [&] { return hf::run_xinv(n, A, X1, B, out, cnt, st); }));
        return HF_OK;
    }
    // the rotated resample runs inside pass A through the texture units;
    // without a texture (its size outside the gather limits) it runs on its own
    if (s2->tex) {
        CU(timed(c, kPassA, st, [&] { return hf::run_passA_tex(n, s2->tex, s2->box, rot9, X1, cnt, st); }));
    } else {
        if (!planes) return fail(HF_EUNSUPPORTED, "field-set build: the moving part has no texture");
        CU(timed(c, kResample, st, [&] { return hf::run_resample_chunk(n, s2->grid, rot9, planes, cnt, st); }));
        CU(timed(c, kPassA, st, [&] { return hf::run_passA_planes(n, planes, X1, cnt, st); }));
    }
    CU(timed(c, kPassB, st, [&] { return hf::run_passB(n, X1, s1->spec, Y1, Y2, cnt, st, tile_b); }));
    if (out.Tx) {  // analytic torque: three more spectra after Y2 in the scratch
        float2 *YT = scratch + 3 * scratch_rot;
        CU(timed(c, kPassB, st, [&] { return hf::run_passB_torque(n, X1, s1->mspec, YT, scratch_rot, cnt, st); }));
        CU(timed(c, kPassC, st, [&] { return hf::run_passC_torque(n, Y1, Y2, YT, scratch_rot, out, cnt, st); }));
        return HF_OK;
    }
    CU(timed(c, kPassC, st, [&] { return hf::run_passC(n, Y1, Y2, out, cnt, st, tile_c); }));
    return HF_OK;
}

static hf_status check_pair(const hf_part *s1, const hf_part *s2, int n, const char *who) {
    if (!s1 || !s2) return fail(HF_EINVAL, "%s: NULL part", who);
    if (s1->role != HF_STATIONARY || s2->role != HF_MOVING)
        return fail(HF_EINVAL, "%s: s1 must be HF_STATIONARY and s2 HF_MOVING", who);
    if (s1->n != n || s2->n != n) return fail(HF_EINVAL, "%s: grid sizes differ (%d, %d, %d)", who, s1->n, s2->n, n);
    return HF_OK;
}

// the torque product's precision from the flags (hf_internal.h run_torque)
static int torque_mode(unsigned flags) {
    return (flags & HF_TORQUE_F64) ? 1 : ((flags & HF_TORQUE_C) ? 2 : 0);
}

// Host preparation of a rotation set: normalised quaternions, float32
// matrices and (with torque) the neighbours and float64 least-squares
// operators.  Returns the number of rank-deficient rotations, or -1 when a
// quaternion is zero or not finite.
int hf_prepare_rotations(const float *h_quat, int R, bool torque, std::vector<float> &rot9, std::vector<double> &q64,
                         std::vector<int> &nbr, std::vector<float> &P32, std::vector<double> &P64) {
    std::vector<Quat> Q(R);
    for (int r = 0; r < R; ++r) {
        Q[r] = qnorm(h_quat + 4 * (size_t)r);
        if (!qfinite(Q[r])) return -1;
    }
    rot9.resize((size_t)R * 9);
    q64.resize((size_t)R * 4);
    for (int r = 0; r < R; ++r) {
        double M[9];
        rot_from_quat(Q[r], M);
        for (int k = 0; k < 9; ++k) rot9[(size_t)9 * r + k] = (float)M[k];
        q64[4 * (size_t)r + 0] = Q[r].w;
        q64[4 * (size_t)r + 1] = Q[r].x;
        q64[4 * (size_t)r + 2] = Q[r].y;
        q64[4 * (size_t)r + 3] = Q[r].z;
    }
    return torque ? torque_setup(Q, nbr, P32, P64, nullptr) : 0;
}

// Device part of a field-set build: every launch, nothing else (so that it
// can be captured in a CUDA graph).  Rotation data comes from the given
// device arrays; outputs go to fs.
hf_status hf_set_launch(hf_ctx *ctx, const hf_part *s1, const hf_part *s2, hf_fieldset *fs, int R,
                        const float *d_rot9, const int *d_nbr, const float *d_P, const double *d_P64,
                        cudaStream_t st) {
    const int n = fs->n;
    if (R <= 0 || R > fs->R) return fail(HF_EINVAL, "field set holds %d rotations, %d asked", fs->R, R);
    hf_status cs = check_pair(s1, s2, n, "field-set build");
    if (cs != HF_OK) return cs;
    if (fs->spectral && !s2->table)
        return fail(HF_ENOTREADY, "field-set build: HF_SPECTRAL needs hf_part_spectral on the moving part");
    if (fs->torque_analytic && !s1->mspec)
        return fail(HF_ENOTREADY, "field-set build: HF_TA needs hf_part_moments on the stationary part");
    const size_t n3 = (size_t)n * n * n;
    const size_t rs = (size_t)fs->nf * n3;
    const size_t scr_rot = (size_t)fs->chunk * hf::half_spec_elems(n);
    hf_status s;
    // with two pipelines: fork them off the caller's stream, alternate
    // chunks, join; with one: run on the caller's stream
    if (fs->lanes == 2) {
        CU(cudaEventRecord(fs->fork, st));
        CU(cudaStreamWaitEvent(fs->lane[0], fs->fork, 0));
        CU(cudaStreamWaitEvent(fs->lane[1], fs->fork, 0));
    }
    for (int r0 = 0, c = 0; r0 < R; r0 += fs->chunk, ++c) {
        const int cnt = std::min(fs->chunk, R - r0);
        const int l = fs->lanes == 2 ? (c & 1) : 0;
        FieldPtrs out;
        float *base = fs->data + (size_t)r0 * rs;
        out.E = base;
        out.rot_stride = rs;
        out.Fx = base + n3;
        out.Fy = base + 2 * n3;
        out.Fz = base + 3 * n3;
        if (fs->torque_analytic) {
            out.Tx = base + (size_t)fs->slot[4] * n3;
            out.Ty = base + (size_t)fs->slot[5] * n3;
            out.Tz = base + (size_t)fs->slot[6] * n3;
        }
        s = run_fields(ctx, n, fs->pencil, fs->prec, s1, s2, d_rot9 + (size_t)9 * r0, cnt, fs->scratch[l], scr_rot,
                       nullptr, out, fs->lanes == 2 ? fs->lane[l] : st, fs->spectral, fs->tile_b, fs->tile_c);
        if (s != HF_OK) return s;
    }
    for (int l = 0; l < 2 && fs->lanes == 2; ++l) {
        CU(cudaEventRecord(fs->join[l], fs->lane[l]));
        CU(cudaStreamWaitEvent(st, fs->join[l], 0));
    }
    if (fs->flags & HF_T) {
        CU(timed(ctx, kTorque, st, [&] {
            return hf::run_torque(n, R, fs->data, rs, fs->data + (size_t)fs->slot[4] * n3, rs, d_nbr, d_P, d_P64,
                                  torque_mode(fs->flags), st);
        }));
    }
    return HF_OK;
}

extern "C" hf_status hf_fieldset_compute(hf_ctx *ctx, const hf_part *s1, const hf_part *s2, const float *h_quat,
                                         int R, hf_fieldset *fs, hf_stream stream) {
    hf::Range range_("hf_fieldset_compute");
    if (!ctx || !fs || !h_quat) return fail(HF_EINVAL, "hf_fieldset_compute: NULL argument");
    if (R != fs->R) return fail(HF_EINVAL, "hf_fieldset_compute: R=%d but the set holds %d", R, fs->R);
    hf_status s = check_pair(s1, s2, fs->n, "hf_fieldset_compute");
    if (s != HF_OK) return s;
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t qbytes = (size_t)R * 4 * sizeof(float);
    if (fs->prep_bad < 0 || fs->prep_quat.size() != (size_t)R * 4 || memcmp(fs->prep_quat.data(), h_quat, qbytes)) {
        fs->prep_bad = -1;
        const int b = hf_prepare_rotations(h_quat, R, (fs->flags & HF_T) != 0, fs->prep_rot9, fs->prep_q64,
                                           fs->prep_nbr, fs->prep_P32, fs->prep_P64);
        if (b < 0) return fail(HF_EINVAL, "hf_fieldset_compute: a quaternion is zero or not finite");
        fs->prep_quat.assign(h_quat, h_quat + (size_t)R * 4);
        fs->prep_bad = b;
    }
    const int bad = fs->prep_bad;
    const std::vector<float> &rot9 = fs->prep_rot9, &P32 = fs->prep_P32;
    const std::vector<double> &q64 = fs->prep_q64, &P64 = fs->prep_P64;
    const std::vector<int> &nbr = fs->prep_nbr;
    // stage through the set's staging buffer once the previous call's uploads are done
    CU(cudaEventSynchronize(fs->stage_done));
    float *s_rot = (float *)fs->h_stage;
    double *s_q = (double *)(s_rot + (size_t)9 * R);
    int *s_nbr = (int *)(s_q + (size_t)4 * R);
    float *s_P = (float *)(s_nbr + (size_t)6 * R);
    double *s_P64 = (double *)(s_P + (size_t)18 * R);
    memcpy(s_rot, rot9.data(), rot9.size() * sizeof(float));
    memcpy(s_q, q64.data(), q64.size() * sizeof(double));
    fs->ready = false;
    CU(cudaMemcpyAsync(fs->d_rot9, s_rot, (size_t)R * 9 * sizeof(float), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(fs->d_quat, s_q, (size_t)R * 4 * sizeof(double), cudaMemcpyHostToDevice, st));
    if (fs->flags & HF_T) {
        memcpy(s_nbr, nbr.data(), nbr.size() * sizeof(int));
        memcpy(s_P, P32.data(), P32.size() * sizeof(float));
        memcpy(s_P64, P64.data(), P64.size() * sizeof(double));
        CU(cudaMemcpyAsync(fs->d_nbr, s_nbr, nbr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(fs->d_P, s_P, P32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        CU(cudaMemcpyAsync(fs->d_P64, s_P64, P64.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    CU(cudaEventRecord(fs->stage_done, st));
    s = hf_set_launch(ctx, s1, s2, fs, R, fs->d_rot9, fs->d_nbr, fs->d_P, fs->d_P64, st);
    if (s != HF_OK) return s;
    fs->ready = true;
    if (bad) return fail(HF_EINVAL, "hf_fieldset_compute: %d rotation(s) with a rank-deficient neighbourhood", bad);
    return HF_OK;
}

extern "C" hf_status hf_fieldset_build(hf_ctx *ctx, const hf_part *s1, const hf_part *s2, const float *h_quat,
                                       int R, unsigned flags, hf_fieldset **out, hf_stream stream) {
    if (!out) return fail(HF_EINVAL, "hf_fieldset_build: out is NULL");
    *out = nullptr;
    if (!s2) return fail(HF_EINVAL, "hf_fieldset_build: NULL part");
    hf_fieldset *fs = nullptr;
    hf_status s = hf_fieldset_create(ctx, s2->n, R, flags, &fs);
    if (s != HF_OK) return s;
    s = hf_fieldset_compute(ctx, s1, s2, h_quat, R, fs, stream);
    if (s != HF_OK && !fs->ready) {
        const hf_status keep = s;
        char msg[sizeof g_err];
        memcpy(msg, g_err, sizeof msg);
        hf_fieldset_release(fs);
        memcpy(g_err, msg, sizeof msg);
        return keep;
    }
    *out = fs;
    return s;
}

static hf_status field_check(const hf_fieldset *fs, int rot, int field, const char *who) {
    if (!fs) return fail(HF_EINVAL, "%s: NULL field set", who);
    if (rot < 0 || rot >= fs->R) return fail(HF_EINVAL, "%s: rotation %d of %d", who, rot, fs->R);
    if (field < 0 || field > 6 || fs->slot[field] < 0) return fail(HF_EINVAL, "%s: field %d not held", who, field);
    if (!fs->ready) return fail(HF_ENOTREADY, "%s: field set not computed", who);
    return HF_OK;
}

extern "C" hf_status hf_fieldset_field_ptr(const hf_fieldset *fs, int rot, int field, const float **d_ptr) {
    hf_status s = field_check(fs, rot, field, "hf_fieldset_field_ptr");
    if (s != HF_OK) return s;
    if (!d_ptr) return fail(HF_EINVAL, "hf_fieldset_field_ptr: d_ptr is NULL");
    const size_t n3 = (size_t)fs->n * fs->n * fs->n;
    *d_ptr = fs->data + ((size_t)rot * fs->nf + fs->slot[field]) * n3;
    return HF_OK;
}

extern "C" hf_status hf_fieldset_get(const hf_fieldset *fs, int rot, int field, float *d_dst, hf_stream stream) {
    const float *src = nullptr;
    hf_status s = hf_fieldset_field_ptr(fs, rot, field, &src);
    if (s != HF_OK) return s;
    if (!d_dst) return fail(HF_EINVAL, "hf_fieldset_get: d_dst is NULL");
    CU(cudaSetDevice(fs->ctx->device));
    const size_t n3 = (size_t)fs->n * fs->n * fs->n;
    CU(cudaMemcpyAsync(d_dst, src, n3 * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return HF_OK;
}

// -------------------------------------------------------------------- query
static hf::QueryGeom query_geom(const hf_fieldset *fs) {
    hf::QueryGeom g;
    g.base = fs->data;
    g.rot_stride = (size_t)fs->nf * fs->n * fs->n * fs->n;
    for (int f = 0; f < 7; ++f) g.field_slot[f] = fs->slot[f];
    g.n = fs->n;
    g.R = fs->R;
    g.quats = fs->d_quat;
    return g;
}

extern "C" hf_status hf_query_batch(const hf_fieldset *fs, const float *d_tq, int Q, int k, float *d_out,
                                    hf_stream stream) {
    hf::Range range_("hf_query_batch");
    if (!fs) return fail(HF_EINVAL, "hf_query_batch: NULL field set");
    if (Q < 0 || (Q > 0 && (!d_tq || !d_out))) return fail(HF_EINVAL, "hf_query_batch: bad buffers");
    if (k < 1 || k > 8 || k > fs->R) return fail(HF_EINVAL, "hf_query_batch: k_blend=%d", k);
    if (!fs->ready) return fail(HF_ENOTREADY, "hf_query_batch: field set not computed");
    CU(cudaSetDevice(fs->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    CU(timed(fs->ctx, kQuery, st, [&] { return hf::run_query(query_geom(fs), d_tq, Q, k, d_out, st); }));
    return HF_OK;
}

// One pose query: the pose travels as a kernel argument and the kernel
// writes its 7 results straight into mapped pinned host memory (h_out, whose
// device alias is d_out), so a query is one launch and one synchronise.
// A single query's request for the resident query kernel: the checks of
// hf_query_on_lane, then the set's geometry and the pose.
hf_status hf_query_request(const hf_fieldset *fs, const float t[3], const float q[4], int k, hf::QueryReq *rq) {
    if (!fs || !t || !q || !rq) return fail(HF_EINVAL, "hf_query: NULL argument");
    if (k < 1 || k > 8 || k > fs->R) return fail(HF_EINVAL, "hf_query: k_blend=%d", k);
    if (!fs->ready) return fail(HF_ENOTREADY, "hf_query: field set not computed");
    rq->g = query_geom(fs);
    for (int a = 0; a < 3; ++a) rq->pose.v[a] = t[a];
    for (int a = 0; a < 4; ++a) rq->pose.v[3 + a] = q[a];
    rq->n = fs->n;
    rq->k = k;
    return HF_OK;
}

hf_status hf_query_on_lane(const hf_fieldset *fs, const float t[3], const float q[4], int k, float out7[7],
                           cudaStream_t st, float *h_out, float *d_out, double *launched_ms) {
    if (!fs || !t || !q || !out7) return fail(HF_EINVAL, "hf_query: NULL argument");
    if (k < 1 || k > 8 || k > fs->R) return fail(HF_EINVAL, "hf_query: k_blend=%d", k);
    if (!fs->ready) return fail(HF_ENOTREADY, "hf_query: field set not computed");
    (void)cudaGetLastError();  // drop a stale non-sticky error before checking the launch
    hf::Pose7 pose;
    for (int a = 0; a < 3; ++a) pose.v[a] = t[a];
    for (int a = 0; a < 4; ++a) pose.v[3 + a] = q[a];
    CU(hf::run_query_one(query_geom(fs), pose, k, d_out, st));
    if (launched_ms)
        *launched_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    CU(cudaStreamSynchronize(st));
    for (int a = 0; a < 7; ++a) out7[a] = ((volatile float *)h_out)[a];
    return HF_OK;
}

extern "C" hf_status hf_query(const hf_fieldset *fs, const float t[3], const float q[4], int k, float out7[7]) {
    if (!fs) return fail(HF_EINVAL, "hf_query: NULL field set");
    hf_ctx *c = fs->ctx;
    std::lock_guard<std::mutex> g(c->qmu);
    CU(cudaSetDevice(c->device));
    if (c->res && c->res->live()) {
        hf::QueryReq rq;
        const hf_status s = hf_query_request(fs, t, q, k, &rq);
        if (s != HF_OK) return s;
        if (c->res->query(0, rq, &c->res_seq, out7, 20.0, nullptr)) return HF_OK;
        // not answered in time: stop the kernel (after which nothing reads the
        // set) and answer by launch; the context's queries launch from now on
        delete c->res;
        c->res = nullptr;
    }
    return hf_query_on_lane(fs, t, q, k, out7, c->qstream, c->h_qout, c->d_qout);
}

extern "C" hf_status hf_ctx_resident_queries(hf_ctx *c, int on) {
    if (!c) return fail(HF_EINVAL, "hf_ctx_resident_queries: NULL context");
    std::lock_guard<std::mutex> g(c->qmu);
    CU(cudaSetDevice(c->device));
    if (on && !c->res) {
        c->res = new (std::nothrow) hf::ResidentQueries();
        if (!c->res || !c->res->start(c->device, 1)) {
            delete c->res;
            c->res = nullptr;
            (void)cudaGetLastError();
            return fail(HF_ECUDA, "hf_ctx_resident_queries: the resident query kernel did not start");
        }
        c->res_seq = 0;
    } else if (!on && c->res) {
        delete c->res;
        c->res = nullptr;
    }
    return HF_OK;
}

// ----------------------------------------------------- single-step entries
// ------------------------------------------------- truncated single poses
static hf_status lowpass_check(const hf_part *s1, const hf_part *s2, int K, const char *who) {
    if (!s1 || !s2) return fail(HF_EINVAL, "%s: NULL part", who);
    if (s1->role != HF_STATIONARY || s2->role != HF_MOVING)
        return fail(HF_EINVAL, "%s: s1 must be HF_STATIONARY and s2 HF_MOVING", who);
    if (s1->n != s2->n) return fail(HF_EINVAL, "%s: grid sizes differ (%d, %d)", who, s1->n, s2->n);
    if (K < 1 || 2 * K >= s1->n) return fail(HF_EINVAL, "%s: K=%d outside 1..N/2-1", who, K);
    if (!s2->table) return fail(HF_ENOTREADY, "%s: the moving part has no spectral table (hf_part_spectral)", who);
    return HF_OK;
}

extern "C" hf_status hf_lowpass_query(const hf_part *s1, const hf_part *s2, int K, const float t[3], const float q[4],
                                      float out7[7]) {
    if (!t || !q || !out7) return fail(HF_EINVAL, "hf_lowpass_query: NULL argument");
    hf_status s = lowpass_check(s1, s2, K, "hf_lowpass_query");
    if (s != HF_OK) return s;
    const Quat Q = qnorm(q);
    if (!qfinite(Q)) return fail(HF_EINVAL, "hf_lowpass_query: the quaternion is zero or not finite");
    double M[9];
    rot_from_quat(Q, M);
    hf::LowpassPose pose;
    for (int k = 0; k < 9; ++k) pose.R[k] = (float)M[k];
    for (int a = 0; a < 3; ++a) pose.t[a] = t[a];
    hf_ctx *c = s1->ctx;
    std::lock_guard<std::mutex> g(c->qmu);
    CU(cudaSetDevice(c->device));
    if (!c->lp_part || !c->lp_count) {  // both or neither
        double *part = nullptr;
        unsigned *count = nullptr;
        cudaError_t e = hf::dmalloc(&part, sizeof(double) * 7 * hf::kLowpassMaxSplit);
        if (e == cudaSuccess) e = hf::dmalloc(&count, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(count, 0, sizeof(unsigned));
        if (e != cudaSuccess) {
            if (part) cudaFree(part);
            if (count) cudaFree(count);
            return fail(e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "hf_lowpass_query: scratch: %s",
                        cudaGetErrorString(e));
        }
        if (c->lp_part) cudaFree(c->lp_part);
        if (c->lp_count) cudaFree(c->lp_count);
        c->lp_part = part;
        c->lp_count = count;
    }
    (void)cudaGetLastError();
    CU(hf::run_lowpass(s1->n, s1->spec, s2->table, s2->table_os, K, nullptr, 1, &pose, c->lp_part, c->lp_count,
                       c->d_qout, c->qstream));
    CU(cudaStreamSynchronize(c->qstream));
    for (int a = 0; a < 7; ++a) out7[a] = ((volatile float *)c->h_qout)[a];
    return HF_OK;
}

extern "C" hf_status hf_lowpass_query_batch(const hf_part *s1, const hf_part *s2, int K, const float *d_tq, int Q,
                                            float *d_out, hf_stream stream) {
    if ((!d_tq || !d_out) && Q > 0) return fail(HF_EINVAL, "hf_lowpass_query_batch: NULL buffer");
    if (Q < 0) return fail(HF_EINVAL, "hf_lowpass_query_batch: Q=%d", Q);
    hf_status s = lowpass_check(s1, s2, K, "hf_lowpass_query_batch");
    if (s != HF_OK) return s;
    if (Q == 0) return HF_OK;
    CU(cudaSetDevice(s1->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t pb = sizeof(double) * 7 * (size_t)hf::lowpass_split(K) * Q;
    double *part = nullptr;
    unsigned *count = nullptr;
    CU(hf::dmalloc_async(&part, pb, st));
    cudaError_t e = hf::dmalloc_async(&count, sizeof(unsigned) * (size_t)Q, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned) * (size_t)Q, st);
    if (e == cudaSuccess) {
        (void)cudaGetLastError();
        e = hf::run_lowpass(s1->n, s1->spec, s2->table, s2->table_os, K, d_tq, Q, nullptr, part, count, d_out, st);
    }
    cudaFreeAsync(part, st);
    if (count) cudaFreeAsync(count, st);
    if (e != cudaSuccess) return fail(HF_ECUDA, "hf_lowpass_query_batch: %s", cudaGetErrorString(e));
    return HF_OK;
}

extern "C" hf_status hf_resample(int n, const float *d_rho, const float h_R[9], float *d_out, hf_stream stream) {
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_resample: N=%d not supported", n);
    if (!d_rho || !h_R || !d_out) return fail(HF_EINVAL, "hf_resample: NULL argument");
    (void)cudaGetLastError();
    hf::Rot9 r;
    for (int k = 0; k < 9; ++k) r.r[k] = h_R[k];
    CU(hf::run_resample(n, d_rho, r, d_out, (cudaStream_t)stream));
    return HF_OK;
}

extern "C" size_t hf_rfft3d_scratch_bytes(int n) {
    if (!hf::supported_n(n)) return 0;
    return 3 * hf::half_spec_elems(n) * sizeof(float2) + 256;
}

extern "C" hf_status hf_rfft3d(int n, const float *d_in, float *d_out, void *d_scratch, hf_stream stream) {
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_rfft3d: N=%d not supported", n);
    if (!d_in || !d_out || !d_scratch) return fail(HF_EINVAL, "hf_rfft3d: NULL argument");
    if ((uintptr_t)d_scratch % 16) return fail(HF_EINVAL, "hf_rfft3d: scratch must be 16-byte aligned");
    if ((uintptr_t)d_in % 8) return fail(HF_EINVAL, "hf_rfft3d: d_in must be 8-byte aligned");
    CU(ensure_kernel_attrs());
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    const size_t he = hf::half_spec_elems(n);
    float2 *X1 = (float2 *)d_scratch, *spec = X1 + he;
    if (hf::pencil_n(n)) {
        CU(hf::run_xfwd(n, d_in, spec + he, 1, st));
        CU(hf::run_yfwd(n, spec + he, X1, 1, st));
    } else {
        CU(hf::run_passA_planes(n, d_in, X1, 1, st));
    }
    CU(hf::run_passB_forward(n, X1, spec, 1.0f, st));
    CU(hf::run_unpermute(n, spec, (float2 *)d_out, st));
    return HF_OK;
}

extern "C" size_t hf_fields_scratch_bytes(int n) {
    if (!hf::supported_n(n)) return 0;
    const size_t n3 = (size_t)n * n * n;
    return fields_spectra(hf::pencil_n(n)) * hf::half_spec_elems(n) * sizeof(float2) + 4 * n3 * sizeof(float) + 256;
}

extern "C" hf_status hf_fields(hf_ctx *ctx, const hf_part *s1, const hf_part *s2, const float h_quat[4], float *d_E,
                               float *d_Fx, float *d_Fy, float *d_Fz, void *d_scratch, hf_stream stream) {
    hf::Range range_("hf_fields");
    if (!ctx || !h_quat || !d_E || !d_scratch) return fail(HF_EINVAL, "hf_fields: NULL argument");
    if ((uintptr_t)d_scratch % 16) return fail(HF_EINVAL, "hf_fields: scratch must be 16-byte aligned");
    hf_status s = check_pair(s1, s2, s1 ? s1->n : 0, "hf_fields");
    if (s != HF_OK) return s;
    const int n = s1->n;
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t he = hf::half_spec_elems(n), n3 = (size_t)n * n * n;
    float2 *scr = (float2 *)d_scratch;
    float *dummy = (float *)(scr + fields_spectra(hf::pencil_n(n)) * he);
    float *planes = dummy + 3 * n3;
    float *rot = planes + n3;
    const Quat q = qnorm(h_quat);
    if (!qfinite(q)) return fail(HF_EINVAL, "hf_fields: quaternion is zero or not finite");
    double M[9];
    rot_from_quat(q, M);
    float m9[9];
    for (int k = 0; k < 9; ++k) m9[k] = (float)M[k];
    CU(cudaMemcpyAsync(rot, m9, sizeof m9, cudaMemcpyHostToDevice, st));
    FieldPtrs out{d_E, d_Fx ? d_Fx : dummy, d_Fy ? d_Fy : dummy + n3, d_Fz ? d_Fz : dummy + 2 * n3, 0};
    s = run_fields(ctx, n, hf::pencil_n(n), hf::PREC_FP32, s1, s2, rot, 1, scr, he, planes, out, st);
    if (s != HF_OK) return s;
    CU(cudaStreamSynchronize(st));  // m9 lives on this stack frame
    return HF_OK;
}

extern "C" hf_status hf_torque(hf_ctx *ctx, int n, int R, const float *h_quat, const float *d_E, float *d_T,
                               unsigned flags, int *h_status, hf_stream stream) {
    hf::Range range_("hf_torque");
    if (!ctx || !h_quat || !d_E || !d_T) return fail(HF_EINVAL, "hf_torque: NULL argument");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_torque: N=%d not supported", n);
    if (R < 7) return fail(HF_EINVAL, "hf_torque: R=%d < 7", R);
    if ((flags & HF_TORQUE_F64) && (flags & HF_TORQUE_C))
        return fail(HF_EINVAL, "hf_torque: HF_TORQUE_F64 and HF_TORQUE_C are alternatives");
    CU(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<Quat> Q(R);
    for (int r = 0; r < R; ++r) {
        Q[r] = qnorm(h_quat + 4 * (size_t)r);
        if (!qfinite(Q[r])) return fail(HF_EINVAL, "hf_torque: quaternion %d is zero or not finite", r);
    }
    std::vector<int> nbr;
    std::vector<float> P32;
    std::vector<double> P64;
    const int bad = torque_setup(Q, nbr, P32, P64, h_status);
    int *d_nbr = nullptr;
    float *d_P = nullptr;
    double *d_P64 = nullptr;
    cudaError_t e = hf::dmalloc_async(&d_nbr, nbr.size() * sizeof(int), st);
    if (e == cudaSuccess) e = hf::dmalloc_async(&d_P, P32.size() * sizeof(float), st);
    if (e == cudaSuccess) e = hf::dmalloc_async(&d_P64, P64.size() * sizeof(double), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_P, P32.data(), P32.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_P64, P64.data(), P64.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    const size_t n3 = (size_t)n * n * n;
    if (e == cudaSuccess)
        e = timed(ctx, kTorque, st, [&] {
            return hf::run_torque(n, R, d_E, n3, d_T, 3 * n3, d_nbr, d_P, d_P64, torque_mode(flags), st);
        });
    if (d_nbr) cudaFreeAsync(d_nbr, st);
    if (d_P) cudaFreeAsync(d_P, st);
    if (d_P64) cudaFreeAsync(d_P64, st);
    const cudaError_t y = cudaStreamSynchronize(st);  // the host vectors are freed on return
    if (e == cudaSuccess) e = y;
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA, "hf_torque: %s", cudaGetErrorString(e));
    if (bad) return fail(HF_EINVAL, "hf_torque: %d rotation(s) with a rank-deficient neighbourhood", bad);
    return HF_OK;
}

// ---------------------------------------------------------------- autotuner
// Choice of rotation chunk (rotations per launch of each pass) and pipeline
// (slab passes or the pencil pipeline) for one grid size, by timing a build of
// E and F on synthetic parts.  Timing does not depend on the densities'
// values: the passes do the same work for any input.
extern "C" hf_status hf_tune_set(hf_ctx *ctx, int n, int chunk, int pencil) {
    if (!ctx) return fail(HF_EINVAL, "hf_tune_set: ctx is NULL");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_tune_set: N=%d not supported", n);
    Tune &t = ctx->tune[tune_slot(n)];
    if (chunk <= 0) {  // back to the built-in choice
        t = Tune();
        return HF_OK;
    }
    if (n >= 256 && !pencil) return fail(HF_EUNSUPPORTED, "hf_tune_set: N=256 runs the pencil pipeline only");
    t.set = true;
    t.chunk = chunk;
    t.pencil = pencil != 0;
    return HF_OK;
}

extern "C" hf_status hf_tune_get(const hf_ctx *ctx, int n, int *chunk, int *pencil, double *rot_per_s) {
    if (!ctx || !chunk || !pencil) return fail(HF_EINVAL, "hf_tune_get: NULL argument");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_tune_get: N=%d not supported", n);
    const Tune &t = ctx->tune[tune_slot(n)];
    *chunk = t.set ? t.chunk : default_chunk(n);
    *pencil = t.set ? (int)t.pencil : (int)(hf::pencil_n(n));
    if (rot_per_s) *rot_per_s = t.set ? t.rot_per_s : 0.0;
    return HF_OK;
}

extern "C" hf_status hf_tune_tiles(hf_ctx *ctx, int n, int set, int *tile_b, int *tile_c) {
    if (!ctx || !tile_b || !tile_c) return fail(HF_EINVAL, "hf_tune_tiles: NULL argument");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_tune_tiles: N=%d not supported", n);
    Tune &t = ctx->tune[tune_slot(n)];
    if (set) {
        if (*tile_b < 0 || *tile_b > 1 || *tile_c < 0 || *tile_c > 7 || (((*tile_c >= 2 && *tile_c <= 4) || *tile_c >= 6) && n != 128) ||
            ((*tile_b || *tile_c) && (n < 64 || n > 128)))
            return fail(HF_EINVAL, "hf_tune_tiles: tile_b %d, tile_c %d at N=%d", *tile_b, *tile_c, n);
        if (!t.set) {  // keep the built-in chunk and pipeline
            t.set = true;
            t.chunk = default_chunk(n);
            t.pencil = hf::pencil_n(n);
        }
        t.tile_b = *tile_b;
        t.tile_c = *tile_c;
    } else {
        *tile_b = t.set ? t.tile_b : 0;
        *tile_c = t.set ? t.tile_c : default_tile_c(n);
    }
    return HF_OK;
}

extern "C" hf_status hf_tune_lanes(hf_ctx *ctx, int n, int set, int *lanes) {
    if (!ctx || !lanes) return fail(HF_EINVAL, "hf_tune_lanes: NULL argument");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_tune_lanes: N=%d not supported", n);
    Tune &t = ctx->tune[tune_slot(n)];
    if (set) {
        if (*lanes != 1 && *lanes != 2) return fail(HF_EINVAL, "hf_tune_lanes: lanes %d", *lanes);
        if (!t.set) {
            t.set = true;
            t.chunk = default_chunk(n);
            t.pencil = hf::pencil_n(n);
        }
        t.lanes = *lanes;
    } else {
        *lanes = t.set ? t.lanes : 1;
    }
    return HF_OK;
}

namespace {
std::string tune_device_key(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "unknown";
    std::string k = p.name;
    for (auto &ch : k)
        if (ch == ' ' || ch == '\t') ch = '_';
    return k + "_sm" + std::to_string(p.major) + std::to_string(p.minor);
}

// The cache is a JSON document, one entry per line (device, N):
//   {"tune": [
//    {"device": "<name>_sm<cc>", "n": 128, "chunk": 128, "pipeline": "slab", "tile_b": 0, "tile_c": 0,
//     "radix": "16x8", "passB_columns_per_cta": 32, "passC_rows_per_x_batch": 32, "passC_threads": 512,
//     "rot_per_s": 33400},
//    ...]}
// It is read back by the key scan below, which accepts the lines it writes.
// the transforms' digit orders: the y and z transforms (fixed: they set the
// intermediates' slot order) and pass C's x inverse (tile 7 at 128^3: 16 x 8)
std::string tune_radix(int n, int tile_c) {
    const char *yz = n == 32 ? "8x4" : n == 64 ? "8x8" : n == 96 ? "12x8" : n == 128 ? "16x8" : "16x16";
    const char *x = n == 32 ? "4x8" : n == 64 ? "8x8" : n == 96 ? "8x12" : n == 128 ? (tile_c == 7 ? "16x8" : "8x16")
                                                                                      : "16x16";
    return std::string("yz ") + yz + ", x inverse " + x;
}
int tune_pass_b_columns(int n, int tile_b) { return tile_b == 1 && n <= 128 ? 16 : (n >= 256 ? 16 : 32); }
int tune_pass_c_rows(int n, int tile_c) {
    if (tile_c == 1 && n >= 64 && n <= 128) return 16;
    return n == 96 ? 48 : (n >= 64 ? 32 : 16);
}
int tune_pass_c_threads(int n, int tile_c) {
    if (tile_c >= 2 && tile_c != 6 && n == 128) return 256;
    return n >= 128 ? 512 : (n >= 64 ? 256 : 128);
}

std::string tune_json_line(const std::string &dev, int n, const Tune &t, const std::string &cands = "") {
    char buf[512];
    snprintf(buf, sizeof buf,
             "{\"device\": \"%s\", \"n\": %d, \"chunk\": %d, \"pipeline\": \"%s\", \"tile_b\": %d, \"tile_c\": %d, "
             "\"lanes\": %d, \"radix\": \"%s\", \"passB_columns_per_cta\": %d, \"passC_rows_per_x_batch\": %d, "
             "\"passC_threads\": %d, \"passC_staging\": \"%s\", \"rot_per_s\": %.6g}",
             dev.c_str(), n, t.chunk, t.pencil ? "pencil" : "slab", t.tile_b, t.tile_c, t.lanes,
             tune_radix(n, t.tile_c).c_str(),
             tune_pass_b_columns(n, t.tile_b), tune_pass_c_rows(n, t.tile_c), tune_pass_c_threads(n, t.tile_c),
             t.tile_c >= 5 ? "bulk" : "loads", t.rot_per_s);
    std::string l = buf;
    if (!cands.empty()) {  // every timed candidate: [chunk, pencil, tile_b, tile_c, lanes, rot_per_s]
        l.pop_back();
        l += ", \"candidates\": [" + cands + "]}";
    }
    return l;
}

// value of "key": in a line (string values unquoted); empty if absent
std::string json_field(const std::string &line, const char *key) {
    const std::string k = std::string("\"") + key + "\": ";
    size_t p = line.find(k);
    if (p == std::string::npos) return "";
    p += k.size();
    if (p < line.size() && line[p] == '"') {
        const size_t q = line.find('"', p + 1);
        return q == std::string::npos ? "" : line.substr(p + 1, q - p - 1);
    }
    const size_t q = line.find_first_of(",}", p);
    return line.substr(p, q == std::string::npos ? std::string::npos : q - p);
}

std::vector<std::string> tune_cache_lines(const char *path) {
    std::vector<std::string> out;
    FILE *f = fopen(path, "r");
    if (!f) return out;
    std::string l;
    for (int ch = fgetc(f);; ch = fgetc(f)) {  // whole lines, however long
        if (ch == EOF || ch == '\n') {
            if (l.find("\"device\"") != std::string::npos) out.push_back(l);
            l.clear();
            if (ch == EOF) break;
        } else {
            l += (char)ch;
        }
    }
    fclose(f);
    return out;
}

bool tune_cache_read(const char *path, const std::string &dev, int n, Tune &t) {
    bool hit = false;
    for (const std::string &l : tune_cache_lines(path)) {
        if (json_field(l, "device") != dev || atoi(json_field(l, "n").c_str()) != n) continue;
        const int c = atoi(json_field(l, "chunk").c_str());
        if (c <= 0) continue;
        t.set = true;
        t.chunk = c;
        t.pencil = json_field(l, "pipeline") == "pencil";
        t.tile_b = atoi(json_field(l, "tile_b").c_str());
        t.tile_c = atoi(json_field(l, "tile_c").c_str());
        t.lanes = json_field(l, "lanes") == "2" ? 2 : 1;
        t.rot_per_s = atof(json_field(l, "rot_per_s").c_str());
        hit = true;
    }
    return hit;
}

bool tune_cache_write(const char *path, const std::string &dev, int n, const Tune &t, const std::string &cands) {
    std::vector<std::string> keep;
    for (const std::string &l : tune_cache_lines(path))
        if (!(json_field(l, "device") == dev && atoi(json_field(l, "n").c_str()) == n)) {
            std::string x = l;
            while (!x.empty() && (x.back() == '\n' || x.back() == ',' || x.back() == ' ')) x.pop_back();
            keep.push_back(x);
        }
    keep.push_back(tune_json_line(dev, n, t, cands));
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fputs("{\"tune\": [\n", f);
    for (size_t i = 0; i < keep.size(); ++i) fprintf(f, " %s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    fputs("]}\n", f);
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

// a smooth synthetic density: a few periodic bumps
std::vector<float> tune_grid(int n, int seed) {
    std::vector<float> g((size_t)n * n * n);
    const double w = 2.0 * M_PI / n;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                const double v = cos(w * (x + seed)) * cos(2 * w * y) + 0.5 * sin(3 * w * (z - seed));
                g[((size_t)z * n + y) * n + x] = (float)(v > 0 ? v : 0);
            }
    return g;
}
}  // namespace

extern "C" hf_status hf_autotune(hf_ctx *ctx, int n, const char *cache_path, int *chunk_out, int *pencil_out,
                                 double *rot_per_s_out) {
    hf::Range range_("hf_autotune");
    if (!ctx) return fail(HF_EINVAL, "hf_autotune: ctx is NULL");
    if (!hf::supported_n(n)) return fail(HF_EUNSUPPORTED, "hf_autotune: N=%d not supported", n);
    CU(cudaSetDevice(ctx->device));
    const std::string dev = tune_device_key(ctx->device);
    Tune best;
    if (cache_path && *cache_path && tune_cache_read(cache_path, dev, n, best)) {
        ctx->tune[tune_slot(n)] = best;
    } else {
        // rotations per timed build: at least two launches of the largest candidate
        // (at 128^3, 256 rotations per launch were 0.8% faster than 128 on a
        // 1024-rotation build: fewer launch tails)
        const int R = n <= 32 ? 1024 : n <= 64 ? 512 : n <= 96 ? 192 : n <= 128 ? 512 : 16;
        const int chunks[] = {4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256};
        const size_t n3 = (size_t)n * n * n;
        float *d_g = nullptr;
        CU(hf::dmalloc(&d_g, 2 * n3 * sizeof(float)));
        std::vector<float> h1 = tune_grid(n, 1), h2 = tune_grid(n, 5);
        hf_part *s1 = nullptr, *s2 = nullptr;
        cudaError_t ce = cudaMemcpy(d_g, h1.data(), n3 * sizeof(float), cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(d_g + n3, h2.data(), n3 * sizeof(float), cudaMemcpyHostToDevice);
        hf_status s = ce == cudaSuccess ? HF_OK : HF_ECUDA;
        if (s == HF_OK) s = hf_part_create(ctx, n, d_g, HF_STATIONARY, &s1, nullptr);
        if (s == HF_OK) s = hf_part_create(ctx, n, d_g + n3, HF_MOVING, &s2, nullptr);
        if (s == HF_OK) ce = cudaDeviceSynchronize();
        cudaFree(d_g);
        if (s != HF_OK || ce != cudaSuccess) {
            hf_part_release(s1);
            hf_part_release(s2);
            return s != HF_OK ? s : fail(HF_ECUDA, "hf_autotune: %s", cudaGetErrorString(ce));
        }
        std::vector<float> quats((size_t)R * 4);
        for (int r = 0; r < R; ++r) {  // evenly spread unit quaternions (any rotations do)
            const double a = 0.61803398875 * r, b = 0.7548776662 * r, c = 0.5698402910 * r;
            quats[4 * r + 0] = (float)(1.0 + cos(2 * M_PI * a));
            quats[4 * r + 1] = (float)sin(2 * M_PI * b);
            quats[4 * r + 2] = (float)cos(2 * M_PI * c);
            quats[4 * r + 3] = (float)(0.3 + sin(2 * M_PI * (a + c)));
        }
        const Tune saved = ctx->tune[tune_slot(n)];
        std::string cands;  // every timed candidate, for the cache file
        auto note = [&](const Tune &t, double rps) {
            char b[96];
            snprintf(b, sizeof b, "%s[%d, %d, %d, %d, %d, %.6g]", cands.empty() ? "" : ", ", t.chunk,
                     t.pencil ? 1 : 0, t.tile_b, t.tile_c, t.lanes, rps);
            cands += b;
        };
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int pencil = 0; pencil <= 1; ++pencil) {
            if (n >= 256 && !pencil) continue;
            for (int chunk : chunks) {
                if (2 * chunk > R) continue;
                Tune &t = ctx->tune[tune_slot(n)];
                t.set = true;
                t.chunk = chunk;
                t.pencil = pencil != 0;
                hf_fieldset *fs = nullptr;
                if (hf_fieldset_create(ctx, n, R, HF_E | HF_F, &fs) != HF_OK) continue;  // does not fit
                // one untimed build, then the best of three
                float best_ms = 1e30f;
                hf_status bs = hf_fieldset_compute(ctx, s1, s2, quats.data(), R, fs, nullptr);
                for (int rep = 0; rep < 3 && bs == HF_OK; ++rep) {
                    cudaEventRecord(e0, nullptr);
                    bs = hf_fieldset_compute(ctx, s1, s2, quats.data(), R, fs, nullptr);
                    cudaEventRecord(e1, nullptr);
                    float ms = 0;
                    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                        best_ms = std::min(best_ms, ms);
                }
                hf_fieldset_release(fs);
                if (bs == HF_OK && best_ms < 1e29f) {
                    const double rps = R / (best_ms * 1e-3);
                    note(t, rps);
                    if (rps > best.rot_per_s) {
                        best = t;
                        best.rot_per_s = rps;
                    }
                }
            }
        }
        // the launch shapes of passes B and C at the best slab shape: every
        // compiled candidate (tile 0 is the one timed above)
        if (best.set && !best.pencil && n >= 64 && n <= 128) {
            for (int tb = 0; tb <= 1; ++tb)
                for (int tc = 0; tc <= 7; ++tc) {
                    if ((tb == 0 && tc == 0) || (n != 128 && ((tc >= 2 && tc <= 4) || tc >= 6))) continue;
                    Tune &t = ctx->tune[tune_slot(n)];
                    t = best;
                    t.tile_b = tb;
                    t.tile_c = tc;
                    hf_fieldset *fs = nullptr;
                    if (hf_fieldset_create(ctx, n, R, HF_E | HF_F, &fs) != HF_OK) continue;
                    float best_ms = 1e30f;
                    hf_status bs = hf_fieldset_compute(ctx, s1, s2, quats.data(), R, fs, nullptr);
                    for (int rep = 0; rep < 3 && bs == HF_OK; ++rep) {
                        cudaEventRecord(e0, nullptr);
                        bs = hf_fieldset_compute(ctx, s1, s2, quats.data(), R, fs, nullptr);
                        cudaEventRecord(e1, nullptr);
                        float ms = 0;
                        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                            best_ms = std::min(best_ms, ms);
                    }
                    hf_fieldset_release(fs);
                    if (bs == HF_OK && best_ms < 1e29f) note(t, R / (best_ms * 1e-3));
                    if (bs == HF_OK && best_ms < 1e29f && R / (best_ms * 1e-3) > best.rot_per_s) {
                        const double rps = R / (best_ms * 1e-3);
                        best = t;
                        best.rot_per_s = rps;
                    }
                }
        }
        // two pipelines alternating chunks on two streams, at the best shape
        if (best.set && getenv("HF_LANES") == nullptr) {
            Tune &t = ctx->tune[tune_slot(n)];
            t = best;
            t.lanes = 2;
            hf_fieldset *fs = nullptr;
            if (hf_fieldset_create(ctx, n, R, HF_E | HF_F, &fs) == HF_OK) {
                float best_ms = 1e30f;
                hf_status bs = hf_fieldset_compute(ctx, s1, s2, quats.data(), R, fs, nullptr);
                for (int rep = 0; rep < 3 && bs == HF_OK; ++rep) {
                    cudaEventRecord(e0, nullptr);
                    bs = hf_fieldset_compute(ctx, s1, s2, quats.data(), R, fs, nullptr);
                    cudaEventRecord(e1, nullptr);
                    float ms = 0;
                    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                        best_ms = std::min(best_ms, ms);
                }
                hf_fieldset_release(fs);
                if (bs == HF_OK && best_ms < 1e29f) {
                    const double rps = R / (best_ms * 1e-3);
                    note(t, rps);
                    if (rps > best.rot_per_s) {
                        best = t;
                        best.rot_per_s = rps;
                    }
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        hf_part_release(s1);
        hf_part_release(s2);
        (void)cudaGetLastError();
        if (!best.set) {
            ctx->tune[tune_slot(n)] = saved;
            return fail(HF_ENOMEM, "hf_autotune: no candidate fitted for N=%d", n);
        }
        ctx->tune[tune_slot(n)] = best;
        if (cache_path && *cache_path && !tune_cache_write(cache_path, dev, n, best, cands))
            return fail(HF_EINVAL, "hf_autotune: cannot write the cache file %s", cache_path);
    }
    if (chunk_out) *chunk_out = best.chunk;
    if (pencil_out) *pencil_out = best.pencil ? 1 : 0;
    if (rot_per_s_out) *rot_per_s_out = best.rot_per_s;
    return HF_OK;
}

// ------------------------------------------------------------- checkpoints
// Section 3.2 precomputes the parts' densities and spectra "prior to the
// virtual assembly session", and Section 4.2 precomputes the fields of the
// permitted orientations; these save that state and load it back, so that a
// service restarts without recomputing it.  A file is a concatenation of NPY
// (format version 1.0) arrays, a small int64 header array first, so numpy
// reads each array in turn with np.lib.format.read_array.
namespace {

constexpr int64_t kCkptMagic = 0x31504B4348465348LL;  // tag of this library's checkpoint files
constexpr int64_t kCkptVersion = 1;

bool npy_write_header(FILE *f, const char *descr, const std::vector<int64_t> &shape) {
    std::string d = std::string("{'descr': '") + descr + "', 'fortran_order': False, 'shape': (";
    for (int64_t s : shape) d += std::to_string(s) + ", ";
    d += "), }";
    const size_t total = 10 + d.size() + 1;  // magic, version, length, dict, newline
    d.append((64 - total % 64) % 64, ' ');
    d += '\n';
    if (d.size() > 65535) return false;
    const unsigned char pre[10] = {0x93, 'N', 'U', 'M', 'P', 'Y', 1, 0, (unsigned char)(d.size() & 0xff),
                                   (unsigned char)(d.size() >> 8)};
    return fwrite(pre, 1, 10, f) == 10 && fwrite(d.data(), 1, d.size(), f) == d.size();
}

// reads a version 1.0 / 2.0 / 3.0 header of a C-ordered array
bool npy_read_header(FILE *f, std::string &descr, std::vector<int64_t> &shape) {
    unsigned char pre[8];
    if (fread(pre, 1, 8, f) != 8 || pre[0] != 0x93 || memcmp(pre + 1, "NUMPY", 5) != 0) return false;
    size_t len = 0;
    if (pre[6] == 1) {
        unsigned char l[2];
        if (fread(l, 1, 2, f) != 2) return false;
        len = l[0] | (size_t)l[1] << 8;
    } else if (pre[6] == 2 || pre[6] == 3) {
        unsigned char l[4];
        if (fread(l, 1, 4, f) != 4) return false;
        len = l[0] | (size_t)l[1] << 8 | (size_t)l[2] << 16 | (size_t)l[3] << 24;
    } else {
        return false;
    }
    if (len > (1u << 20)) return false;
    std::string h(len, '\0');
    if (fread(&h[0], 1, len, f) != len) return false;
    const size_t dp = h.find("'descr'"), fp = h.find("'fortran_order'"), sp = h.find("'shape'");
    if (dp == std::string::npos || fp == std::string::npos || sp == std::string::npos) return false;
    const size_t q0 = h.find('\'', h.find(':', dp) + 1), q1 = h.find('\'', q0 + 1);
    if (q0 == std::string::npos || q1 == std::string::npos) return false;
    descr = h.substr(q0 + 1, q1 - q0 - 1);
    if (h.compare(h.find_first_not_of(' ', h.find(':', fp) + 1), 5, "False") != 0) return false;
    const size_t p0 = h.find('(', sp), p1 = h.find(')', sp);
    if (p0 == std::string::npos || p1 == std::string::npos) return false;
    shape.clear();
    const char *c = h.c_str() + p0 + 1, *e = h.c_str() + p1;
    while (c < e) {
        while (c < e && (*c == ' ' || *c == ',')) ++c;
        if (c >= e) break;
        char *end = nullptr;
        const long long v = strtoll(c, &end, 10);
        if (end == c || v < 0) return false;
        shape.push_back(v);
        c = end;
    }
    return true;
}

size_t npy_count(const std::vector<int64_t> &shape) {
    size_t n = 1;
    for (int64_t s : shape) n *= (size_t)s;
    return n;
}

bool write_host_array(FILE *f, const char *descr, const std::vector<int64_t> &shape, const void *p, size_t elem) {
    const size_t b = npy_count(shape) * elem;
    return npy_write_header(f, descr, shape) && fwrite(p, 1, b, f) == b;
}

// an array whose descr and element count the caller checks
bool read_host_array(FILE *f, const char *descr, std::vector<int64_t> &shape, std::vector<char> &out, size_t elem) {
    std::string d;
    if (!npy_read_header(f, d, shape) || d != descr) return false;
    out.resize(npy_count(shape) * elem);
    return fread(out.data(), 1, out.size(), f) == out.size();
}

constexpr size_t kIoChunk = 64u << 20;

// device bytes to the file through a host buffer, chunk by chunk
hf_status write_device(FILE *f, const void *d, size_t bytes, cudaStream_t st) {
    std::vector<char> buf(std::min(bytes, kIoChunk));
    for (size_t o = 0; o < bytes; o += kIoChunk) {
        const size_t b = std::min(kIoChunk, bytes - o);
        CU(cudaMemcpyAsync(buf.data(), (const char *)d + o, b, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (fwrite(buf.data(), 1, b, f) != b) return fail(HF_EINVAL, "checkpoint: write failed");
    }
    return HF_OK;
}

hf_status read_device(FILE *f, void *d, size_t bytes, cudaStream_t st) {
    std::vector<char> buf(std::min(bytes, kIoChunk));
    for (size_t o = 0; o < bytes; o += kIoChunk) {
        const size_t b = std::min(kIoChunk, bytes - o);
        if (fread(buf.data(), 1, b, f) != b) return fail(HF_EINVAL, "checkpoint: file is truncated");
        CU(cudaMemcpyAsync((char *)d + o, buf.data(), b, cudaMemcpyHostToDevice, st));
        CU(cudaStreamSynchronize(st));
    }
    return HF_OK;
}

bool read_meta(FILE *f, int64_t kind, std::vector<int64_t> &meta) {
    std::vector<int64_t> shape;
    std::vector<char> raw;
    if (!read_host_array(f, "<i8", shape, raw, 8) || shape.size() != 1 || shape[0] < 8) return false;
    meta.resize(shape[0]);
    memcpy(meta.data(), raw.data(), raw.size());
    return meta[0] == kCkptMagic && meta[1] == kCkptVersion && meta[2] == kind;
}

struct FileCloser {
    FILE *f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};

}  // namespace

extern "C" hf_status hf_checkpoint_info(const char *path, int *kind, int *n, int *R, unsigned *flags) {
    if (!path) return fail(HF_EINVAL, "hf_checkpoint_info: NULL path");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(HF_EINVAL, "hf_checkpoint_info: cannot open %s", path);
    FileCloser fc{f};
    std::vector<int64_t> shape;
    std::vector<char> raw;
    if (!read_host_array(f, "<i8", shape, raw, 8) || shape.size() != 1 || shape[0] < 8)
        return fail(HF_EINVAL, "hf_checkpoint_info: %s is not a checkpoint of this library", path);
    const int64_t *m = (const int64_t *)raw.data();
    if (m[0] != kCkptMagic || m[1] != kCkptVersion || m[2] < HF_CKPT_PART || m[2] > HF_CKPT_SESSION)
        return fail(HF_EINVAL, "hf_checkpoint_info: %s is not a checkpoint of this library", path);
    if (kind) *kind = (int)m[2];
    if (n) *n = (int)m[3];
    if (R) *R = m[2] == HF_CKPT_PART ? 0 : (int)m[4];
    if (flags) *flags = m[2] == HF_CKPT_PART ? (unsigned)m[4] : (unsigned)m[5];
    return HF_OK;
}

extern "C" hf_status hf_part_save(const hf_part *p, const char *path, hf_stream stream) {
    if (!p || !path) return fail(HF_EINVAL, "hf_part_save: NULL argument");
    CU(cudaSetDevice(p->ctx->device));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(HF_EINVAL, "hf_part_save: cannot create %s", path);
    FileCloser fc{f};
    const int n = p->n;
    const std::vector<int64_t> meta = {kCkptMagic, kCkptVersion, HF_CKPT_PART, n, p->role, 0, 0, 0};
    if (!write_host_array(f, "<i8", {8}, meta.data(), 8)) return fail(HF_EINVAL, "hf_part_save: write failed");
    if (p->role == HF_MOVING) {
        if (!npy_write_header(f, "<f4", {n, n, n})) return fail(HF_EINVAL, "hf_part_save: write failed");
        return write_device(f, p->grid, (size_t)n * n * n * sizeof(float), (cudaStream_t)stream);
    }
    if (!npy_write_header(f, "<c8", {n, n, n / 2 + 1})) return fail(HF_EINVAL, "hf_part_save: write failed");
    return write_device(f, p->spec, hf::half_spec_elems(n) * sizeof(float2), (cudaStream_t)stream);
}

extern "C" hf_status hf_part_load(hf_ctx *ctx, const char *path, hf_part **out, hf_stream stream) {
    if (!ctx || !path || !out) return fail(HF_EINVAL, "hf_part_load: NULL argument");
    *out = nullptr;
    CU(cudaSetDevice(ctx->device));
    FILE *f = fopen(path, "rb");
    if (!f) return fail(HF_EINVAL, "hf_part_load: cannot open %s", path);
    FileCloser fc{f};
    std::vector<int64_t> meta, shape;
    if (!read_meta(f, HF_CKPT_PART, meta)) return fail(HF_EINVAL, "hf_part_load: %s is not a part checkpoint", path);
    const int n = (int)meta[3], role = (int)meta[4];
    if (!hf::supported_n(n) || (role != HF_STATIONARY && role != HF_MOVING))
        return fail(HF_EINVAL, "hf_part_load: N=%d, role %d", n, role);
    std::string descr;
    if (!npy_read_header(f, descr, shape)) return fail(HF_EINVAL, "hf_part_load: %s: bad array header", path);
    cudaStream_t st = (cudaStream_t)stream;
    if (role == HF_MOVING) {
        if (descr != "<f4" || shape != std::vector<int64_t>{n, n, n})
            return fail(HF_EINVAL, "hf_part_load: %s: grid array of the wrong type or shape", path);
        const size_t b = (size_t)n * n * n * sizeof(float);
        float *tmp = nullptr;
        CU(hf::dmalloc_async(&tmp, b, st));
        hf_status s = read_device(f, tmp, b, st);
        if (s == HF_OK) s = hf_part_create(ctx, n, tmp, HF_MOVING, out, stream);
        cudaFreeAsync(tmp, st);
        return s;
    }
    if (descr != "<c8" || shape != std::vector<int64_t>{n, n, n / 2 + 1})
        return fail(HF_EINVAL, "hf_part_load: %s: spectrum array of the wrong type or shape", path);
    const size_t bytes = hf::half_spec_elems(n) * sizeof(float2);
    if (!charge(ctx, bytes)) return fail(HF_EBUDGET, "hf_part_load: %zu bytes exceed the budget", bytes);
    hf_part *p = new (std::nothrow) hf_part{ctx, n, HF_STATIONARY, nullptr, nullptr, bytes};
    cudaError_t e = p ? hf::dmalloc(&p->spec, bytes) : cudaErrorMemoryAllocation;
    hf_status s = e == cudaSuccess ? read_device(f, p->spec, bytes, st)
                                   : fail(HF_ENOMEM, "hf_part_load: %s", cudaGetErrorString(e));
    if (s != HF_OK) {
        if (p && p->spec) cudaFree(p->spec);
        delete p;
        uncharge(ctx, bytes);
        return s;
    }
    hf_ctx_retain(ctx);
    *out = p;
    return HF_OK;
}

hf_status hf_fieldset_write(const hf_fieldset *fs, FILE *f, cudaStream_t st) {
    if (!fs->ready || fs->prep_quat.size() != (size_t)fs->R * 4)
        return fail(HF_ENOTREADY, "field-set save: the set holds no computed rotation set");
    const int n = fs->n;
    std::vector<int64_t> meta = {kCkptMagic, kCkptVersion, HF_CKPT_FIELDSET, n, fs->R, fs->flags, fs->nf};
    for (int k = 0; k < 7; ++k) meta.push_back(fs->slot[k]);
    meta.resize(16, 0);
    if (!write_host_array(f, "<i8", {16}, meta.data(), 8) ||
        !write_host_array(f, "<f4", {fs->R, 4}, fs->prep_quat.data(), 4) ||
        !npy_write_header(f, "<f4", {fs->R, fs->nf, n, n, n}))
        return fail(HF_EINVAL, "field-set save: write failed");
    return write_device(f, fs->data, (size_t)fs->R * fs->nf * n * n * n * sizeof(float), st);
}

hf_status hf_fieldset_read(hf_ctx *ctx, FILE *f, hf_fieldset **out, cudaStream_t mem_stream, cudaStream_t st) {
    *out = nullptr;
    std::vector<int64_t> meta, shape;
    std::vector<char> raw;
    if (!read_meta(f, HF_CKPT_FIELDSET, meta) || meta.size() < 14)
        return fail(HF_EINVAL, "field-set load: not a field-set checkpoint");
    const int n = (int)meta[3], R = (int)meta[4], nf = (int)meta[6];
    const unsigned flags = (unsigned)meta[5];
    if (!read_host_array(f, "<f4", shape, raw, 4) || shape != std::vector<int64_t>{R, 4})
        return fail(HF_EINVAL, "field-set load: rotation array of the wrong type or shape");
    const float *q = (const float *)raw.data();
    hf_fieldset *fs = nullptr;
    hf_status s = fieldset_create_impl(ctx, n, R, flags, mem_stream, &fs);
    if (s != HF_OK) return s;
    std::string descr;
    if (fs->nf != nf || !npy_read_header(f, descr, shape) || descr != "<f4" ||
        shape != std::vector<int64_t>{R, nf, n, n, n}) {
        hf_fieldset_release(fs);
        return fail(HF_EINVAL, "field-set load: field array of the wrong type or shape");
    }
    for (int k = 0; k < 7; ++k)
        if (fs->slot[k] != (int)meta[7 + k]) {
            hf_fieldset_release(fs);
            return fail(HF_EINVAL, "field-set load: field layout differs from this library's");
        }
    // the rotation set's host preparation and uploads, as a compute would make them
    const int bad = hf_prepare_rotations(q, R, (flags & HF_T) != 0, fs->prep_rot9, fs->prep_q64, fs->prep_nbr,
                                         fs->prep_P32, fs->prep_P64);
    if (bad < 0) {
        hf_fieldset_release(fs);
        return fail(HF_EINVAL, "field-set load: a quaternion is zero or not finite");
    }
    fs->prep_quat.assign(q, q + (size_t)R * 4);
    fs->prep_bad = bad;
    cudaError_t e = cudaMemcpyAsync(fs->d_rot9, fs->prep_rot9.data(), fs->prep_rot9.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fs->d_quat, fs->prep_q64.data(), fs->prep_q64.size() * sizeof(double),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && (flags & HF_T)) {
        e = cudaMemcpyAsync(fs->d_nbr, fs->prep_nbr.data(), fs->prep_nbr.size() * sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(fs->d_P, fs->prep_P32.data(), fs->prep_P32.size() * sizeof(float),
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(fs->d_P64, fs->prep_P64.data(), fs->prep_P64.size() * sizeof(double),
                                cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors are pageable
    s = e == cudaSuccess ? read_device(f, fs->data, (size_t)R * nf * n * n * n * sizeof(float), st)
                         : fail(HF_ECUDA, "field-set load: %s", cudaGetErrorString(e));
    if (s != HF_OK) {
        hf_fieldset_release(fs);
        return s;
    }
    fs->ready = true;
    *out = fs;
    return HF_OK;
}

extern "C" hf_status hf_fieldset_save(const hf_fieldset *fs, const char *path, hf_stream stream) {
    if (!fs || !path) return fail(HF_EINVAL, "hf_fieldset_save: NULL argument");
    CU(cudaSetDevice(fs->ctx->device));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(HF_EINVAL, "hf_fieldset_save: cannot create %s", path);
    FileCloser fc{f};
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    return hf_fieldset_write(fs, f, (cudaStream_t)stream);
}

extern "C" hf_status hf_fieldset_load(hf_ctx *ctx, const char *path, hf_fieldset **out, hf_stream stream) {
    if (!ctx || !path || !out) return fail(HF_EINVAL, "hf_fieldset_load: NULL argument");
    CU(cudaSetDevice(ctx->device));
    FILE *f = fopen(path, "rb");
    if (!f) return fail(HF_EINVAL, "hf_fieldset_load: cannot open %s", path);
    FileCloser fc{f};
    return hf_fieldset_read(ctx, f, out, nullptr, (cudaStream_t)stream);
}

// the checkpoint's array helpers for the server's session files
bool hf_ckpt_write_i64(FILE *f, const std::vector<int64_t> &v) { return write_host_array(f, "<i8", {(int64_t)v.size()}, v.data(), 8); }
bool hf_ckpt_write_f32(FILE *f, const std::vector<int64_t> &shape, const float *p) { return write_host_array(f, "<f4", shape, p, 4); }
bool hf_ckpt_read_i64(FILE *f, std::vector<int64_t> &v) {
    std::vector<int64_t> shape;
    std::vector<char> raw;
    if (!read_host_array(f, "<i8", shape, raw, 8) || shape.size() != 1) return false;
    v.resize(shape[0]);
    memcpy(v.data(), raw.data(), raw.size());
    return true;
}
bool hf_ckpt_read_f32(FILE *f, std::vector<int64_t> &shape, std::vector<float> &v) {
    std::vector<char> raw;
    if (!read_host_array(f, "<f4", shape, raw, 4)) return false;
    v.resize(raw.size() / 4);
    memcpy(v.data(), raw.data(), raw.size());
    return true;
}
int64_t hf_ckpt_magic() { return kCkptMagic; }
int64_t hf_ckpt_version() { return kCkptVersion; }
