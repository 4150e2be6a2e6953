// hf_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdio.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <thread>

#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "hf.h"

namespace hf {

// Output pointers of one field-build launch; fields of rotation r start at
// ptr + r * rot_stride (floats).
struct FieldPtrs {
    float *E, *Fx, *Fy, *Fz;
    size_t rot_stride;
    float *Tx = nullptr, *Ty = nullptr, *Tz = nullptr;  // analytic torque fields (HF_TA), else unused
};

// One run of work items of the persistent field-build kernel: `count`
// items of one pass (0 A, 1 B, 2 C) at one grid size over one pair's
// rotation chunk, items first .. first + count - 1 of that pass.  A pass-A
// or pass-C item is one (plane, rotation), a pass-B item one (column tile,
// rotation).  Before an item runs, counters dep[d] must reach dep_target[d];
// each finished item adds 1 to counter `done`.
struct PersistSeg {
    int pass, n;
    int base, count, first;
    int dep[2], dep_target[2];
    int done;
    const float *rot9;           // the chunk's rotations (row-major 3 x 3 each)
    cudaTextureObject_t tex;     // the moving part's gather texture
    const int *box;              // and its support
    const float2 *R1hat;         // the stationary spectrum
    float2 *X1, *Y1, *Y2;        // the chunk's intermediates
    FieldPtrs out;               // fields of the chunk's first rotation
};
constexpr int kPersistNT = 256;
enum { PERSIST_OK = 0, PERSIST_TIMEOUT = 1 };

struct Rot9 {
    float r[9];  // row-major rotation matrix
};

inline bool supported_n(int n) { return n == 32 || n == 64 || n == 96 || n == 128 || n == 256; }

// grids too large for one CTA's shared memory per plane use the pencil
// pipeline; HF_PIPELINE=pencil selects it for every size (cross-checks)
bool pencil_n(int n);

// Texture layout of a moving grid: N padded (N+1)^2 slices tiled SC across
// so that the 2D array stays within the gather height limit (32768 texels).
template <int N>
struct TexLayout {
    static constexpr int SC = N <= 128 ? 1 : 4;
    static constexpr int W = SC * (N + 1);
    static constexpr int HGT = ((N + SC - 1) / SC) * (N + 1);
};
inline void tex_layout(int n, int *w, int *h) {
    const int sc = n <= 128 ? 1 : 4;
    *w = sc * (n + 1);
    *h = ((n + sc - 1) / sc) * (n + 1);
}

// elements of one half-spectrum intermediate (complex): N * N * (N/2 + 1)
inline size_t half_spec_elems(int n) { return (size_t)n * n * (n / 2 + 1); }

// hf_api.cu: the calling thread's message for hf_last_error()
void set_last_error(const char *msg);

// hf_fft.cu
cudaError_t fft_init_attrs(int n);
// the one-launch field build over a table of item runs (sorted by base;
// total items in all; lut[i] = the run holding item 256 i), with its queue
// head, counters and status word (all zero before a launch); the blocks per
// SM it runs at
cudaError_t persist_init();
int persist_blocks_per_sm();
size_t persist_smem();
cudaError_t run_persistent(const PersistSeg *d_segs, const int *d_lut, int nseg, int total, unsigned *d_queue,
                           unsigned *d_counters, int *d_status, long long spin_limit, cudaStream_t st);
cudaError_t run_passA(int n, const float *rho, const float *rot9, float2 *X1, int nrot, cudaStream_t st);
// pass A from planes already in memory: plane z of rotation r at planes + (r N + z) N^2
cudaError_t run_passA_planes(int n, const float *planes, float2 *X1, int nrot, cudaStream_t st);
// box: the moving density's support as cell intervals (run_support), or null
// for the whole torus
cudaError_t run_passA_tex(int n, cudaTextureObject_t tex, const int *box, const float *rot9, float2 *X1, int nrot,
                          cudaStream_t st);
// rotated resample of a chunk: out[r] = rho(R_r^T x_n), r < nrot
cudaError_t run_resample_chunk(int n, const float *rho, const float *rot9, float *out, int nrot, cudaStream_t st);
// the same through 2x2 texture gathers of the stacked padded slices (see hf_fft.cu)
cudaError_t run_pad_slices(int n, const float *g, float *slab, size_t pitch_floats, cudaStream_t st);
// the support of an N^3 grid g: per axis the circular interval of cells that
// hold a nonzero node, as box[2a] = first cell, box[2a + 1] = cell count
// (a = 0, 1, 2 for x, y, z); masks is kSupportMaskWords words of scratch
constexpr int kSupportMaskWords = 24;
cudaError_t run_support(int n, const float *g, unsigned *masks, int *box, cudaStream_t st);
// tile: the autotuner's launch-shape candidate (pass B: 0 the built-in 32
// columns per CTA, 1 16 columns; pass C: 0 built-in, 1 16 rows per x batch,
// 2 256 threads per CTA at N = 128)
cudaError_t run_passB(int n, const float2 *X1, const float2 *R1hat, float2 *Y1, float2 *Y2, int nrot,
                      cudaStream_t st, int tile = 0);
cudaError_t run_passB_forward(int n, const float2 *X1, float2 *spec, float scale, cudaStream_t st);
cudaError_t run_passC(int n, const float2 *Y1, const float2 *Y2, FieldPtrs out, int nrot, cudaStream_t st,
                      int tile = 0);
cudaError_t run_unpermute(int n, const float2 *spec, float2 *out, cudaStream_t st);
// spectral mode (rotation in the frequency domain): a moving part's centred
// table is built from rho2 padded to np = os n nodes (pad, forward transform
// at np, complete); pass B then interpolates the table instead of
// transforming resampled planes
cudaError_t run_pad_center(int n, const float *g, float *out, int np, cudaStream_t st);
cudaError_t run_spectral_complete(int np, const float2 *spec, float2 *table, cudaStream_t st);
cudaError_t run_passB_spectral(int n, const float2 *table, cudaTextureObject_t tex, int os, const float *rot9,
                               const float2 *R1hat, float2 *Y1, float2 *Y2, int nrot, cudaStream_t st);
// the spectral table's gather texture: np^3 cells as stacked, wrap-padded
// (np+1)^2 slices (table_tex_sc(np) per row) in a width x height float2 array
void table_tex_layout(int np, int *width, int *height);
cudaError_t run_pad_table(const float2 *table, int np, float2 *slab, cudaStream_t st);
// analytic torque (rotational gradient of Eq. 6b, moment on the stationary
// side): the three products Gm_a conj(rho2^R^) of the stationary moment
// spectra Gm (3 half spectra, slot order, scaled) with the rotated moving
// spectrum, inverse z -> YT (3 half spectra per rotation); pass C then turns
// them into T = C(G, rho2R) - t x F
cudaError_t run_passB_torque(int n, const float2 *X1, const float2 *Gm, float2 *YT, size_t yt_stride, int nrot,
                             cudaStream_t st);
cudaError_t run_passC_torque(int n, const float2 *Y1, const float2 *Y2, const float2 *YT, size_t yt_stride,
                             FieldPtrs out, int nrot, cudaStream_t st);
// hf_mesh.cu: the mesh descriptor of Eq. 2 on the N^3 nodes (rho; aux, if
// not null, gets W then the signed distance, N^3 each)
cudaError_t run_mesh_sdf(int n, const double *V, const int *T, int nt, double sigma, double gamma_max, int dmax,
                         float *rho, float *aux, cudaStream_t st);
// G_a = (u x F)_a / h^3 for the field set of rho1 against a unit delta (F =
// -h^3 grad rho1), u the node position: the stationary moment fields
cudaError_t run_moment_fields(int n, const float *Fx, const float *Fy, const float *Fz, float *G, cudaStream_t st);
// hf_lowpass.cu: single poses from spectra truncated to |k~_a| <= K (one
// pose by value when `one` is given, else Q poses d_tq Q x 7); out Q x 7
struct LowpassPose {
    float R[9];
    float t[3];
};
// thread blocks per pose; scratch per call: part Q x split x 7 doubles and
// count Q unsigned, zero on entry (each pose's counter is reset on exit)
constexpr int kLowpassMaxSplit = 512;
int lowpass_split(int K);
cudaError_t run_lowpass(int n, const float2 *spec1, const float2 *table, int os, int K, const float *d_tq, int Q,
                        const LowpassPose *one, double *part, unsigned *count, float *out, cudaStream_t st);
// pencil pipeline (any N; the only one for N = 256): planes -> Xa -> X1 (forward x, y),
// then pass B, then Y1/Y2 -> Z_S, Z_Gy, Z_Gz (inverse y) -> fields (inverse x)
cudaError_t run_xfwd(int n, const float *planes, float2 *Xa, int nrot, cudaStream_t st);
// the x forward of the pencil pipeline sampling the moving texture directly
cudaError_t run_xfwd_tex(int n, cudaTextureObject_t tex, const int *box, const float *rot9, float2 *Xa, int nrot,
                         cudaStream_t st);
cudaError_t run_yfwd(int n, const float2 *Xa, float2 *X1, int nrot, cudaStream_t st);
// hf_tc.cu: the pencil pipeline's y stages as split hi/lo DFT-matrix GEMMs on
// the tensor cores (N = 256 only); same inputs and outputs as run_yfwd /
// run_yinv
enum { PREC_FP32 = 0, PREC_SPLIT_BF16 = 1, PREC_SPLIT_F16 = 2 };
cudaError_t run_yfwd_tc(int n, int prec, const float2 *Xa, float2 *X1, int nrot, cudaStream_t st);
cudaError_t run_yinv_tc(int n, int prec, const float2 *Y1, const float2 *Y2, float2 *ZS, float2 *ZGy, float2 *ZGz,
                        int nrot, cudaStream_t st);
cudaError_t set_tc_attrs();
// CTAs of the tensor-core stages whose bounded wait for their MMAs gave up
// (their outputs are invalid); -1 if the counter cannot be read
int tc_timeouts(bool reset);
// hf_fft.cu: waits for bulk copies that gave up, and the one-block self test
// of that bounded wait (plant: the wait cannot complete)
int bulk_timeouts(bool reset);
cudaError_t run_bulk_selftest(const void *src, void *dst, int plant, cudaStream_t st);
int bulk_selftest_bytes();
cudaError_t run_yinv(int n, const float2 *Y1, const float2 *Y2, float2 *ZS, float2 *ZGy, float2 *ZGz, int nrot,
                     cudaStream_t st);
cudaError_t run_xinv(int n, const float2 *ZS, const float2 *ZGy, const float2 *ZGz, FieldPtrs out, int nrot,
                     cudaStream_t st);

// hf_kernels.cu
cudaError_t run_splat(int n, const float *pts, const float *sigma, const float *amp, int P, float *grid,
                      cudaStream_t st);
cudaError_t run_resample(int n, const float *rho, Rot9 rot, float *out, cudaStream_t st);
// mode: 0 float32 product, 1 float64 product, 2 compensated float32 (float64-class)
cudaError_t run_torque(int n, int R, const float *E, size_t e_rot_stride, float *T, size_t t_rot_stride,
                       const int *nbr, const float *P, const double *P64, int mode, cudaStream_t st);
// query: field f of rotation r at base + r*rot_stride + field_slot[f]*n^3 when
// field_slot[f] >= 0, else the field reads 0
struct QueryGeom {
    const float *base;
    size_t rot_stride;
    int field_slot[7];
    int n, R;
    const double *quats;  // R x 4, normalised, on device
};
cudaError_t run_query(const QueryGeom &g, const float *tq, int Q, int k, float *out, cudaStream_t st);
struct Pose7 {
    float v[7];  // tx, ty, tz, qw, qx, qy, qz
};
// one query, pose by value, 7 results to `out` (device or mapped host memory)
cudaError_t run_query_one(const QueryGeom &g, Pose7 pose, int k, float *out, cudaStream_t st);
// A lane's mailbox of the resident query kernel, in mapped pinned host memory:
// the host writes g, pose, n, k and then bumps the lane's request number in
// the mailbox header; the kernel writes out and then done = that number.
struct QueryReq {
    QueryGeom g;
    Pose7 pose;
    int n, k;
};
struct alignas(128) QueryMail {
    QueryReq rq;
    float out[8];
    unsigned done;
};
constexpr int kResidentLanesPerBlock = 15;  // + 1 polling warp: 512 threads
cudaError_t launch_query_resident(QueryMail *mail, unsigned *req, unsigned *served, const unsigned *stop, int lanes,
                                  unsigned long long life_ns, cudaStream_t st);

// The resident query kernel's host side (hf_resident.cu): the lanes'
// mailboxes in mapped pinned memory, each lane's last answered request number
// on the device, and a thread that keeps two instances of the kernel queued on
// a high-priority stream (the next starts on the device as the running one
// ends).  A lane is used by one thread at a time (its owner's lock or lane
// pool).  While it runs, a device-wide synchronisation waits for the running
// and the queued instance.
class ResidentQueries {
  public:
    static constexpr unsigned long long kLifeNs = 10ull * 1000 * 1000;  // one instance's service
    ~ResidentQueries() { stop(); }
    // allocate and start (false, and nothing left running, on any failure)
    bool start(int device, int lanes);
    // stop the keeper; on return no instance runs or is queued
    void stop();
    bool live() const { return live_.load(std::memory_order_acquire); }
    // post a request on `lane` (number *seq + 1, stored back) and spin until
    // it is answered or wait_ms pass: true with out7 on an answer, false on
    // timeout (the request may still be read: see answered)
    bool query(int lane, const QueryReq &rq, unsigned *seq, float out7[7], double wait_ms, double *posted_ms);
    // whether the request numbered seq on lane has been answered
    bool answered(int lane, unsigned seq) const;

  private:
    void keeper();
    int device_ = 0, lanes_ = 0;
    char *h_ = nullptr, *d_ = nullptr;  // request numbers (256 B), stop flag (256 B), mailboxes
    unsigned *d_served_ = nullptr;
    cudaStream_t st_ = nullptr;
    std::thread thread_;
    std::atomic<bool> live_{false}, quit_{false};
    unsigned *h_req() const { return reinterpret_cast<unsigned *>(h_); }
    unsigned *h_stop() const { return reinterpret_cast<unsigned *>(h_ + 256); }
    QueryMail *h_mail() const { return reinterpret_cast<QueryMail *>(h_ + 512); }
};

// An NVTX range over a library call (a profiler with NVTX support shows the
// call's kernels under its name; without one the push and pop do nothing).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// A device region handed out by host-side bookkeeping: best-fit over a free
// list kept sorted by offset and coalesced on every free.  Allocating and
// freeing are host operations with no CUDA call, so a server whose builds
// take their field sets from an arena never maps or unmaps device memory
// while its queries run.  Ranges start on 256 bytes, ranges of 2 MB or more
// on 2 MB (one large page each).  Thread-safe.  The caller owns the region:
// reset() adopts [base, base + bytes) with everything free, and the caller
// frees the region after the last range is released.
class Arena {
  public:
    static constexpr size_t kAlign = 256, kLargeAlign = size_t(2) << 20;
    void reset(uintptr_t base, size_t bytes);
    void *alloc(size_t bytes);  // nullptr when no free range fits
    bool release(void *p);      // false if p is not a live range's start
    bool owns(const void *p) const;
    size_t capacity() const;
    size_t free_bytes() const;
    size_t largest_free() const;
    int64_t failures() const;  // allocations refused for want of a range
    size_t merged_if_released(const void *p) const;  // the free range p's release would make (0: not live)
    size_t free_range_containing(const void *p) const;  // length of the free range holding p (0: none)
    bool check() const;        // the invariants (tests)
    size_t live_count() const;

  private:
    mutable std::mutex mu_;
    uintptr_t base_ = 0;
    size_t size_ = 0, free_ = 0;
    int64_t failures_ = 0;
    std::map<size_t, size_t> free_list_;  // offset -> length: disjoint, no two adjacent
    std::map<size_t, size_t> live_;       // offset -> length
};

// One kernel of each file whose device code the field builds, the queries and
// the precision variants use; hf_ctx_preload loads their modules whole.
const void *module_anchor_fft();
const void *module_anchor_kernels();
const void *module_anchor_tc();

// Allocation-failure injection for the error paths' tests (hf_inject_alloc_failure):
// every device, array and pinned-host allocation the library makes goes
// through these, which count it and, for the one the test picked, return the
// allocator's out-of-memory error without allocating.
extern std::atomic<long long> g_alloc_count, g_alloc_fail_at;
inline bool alloc_fails() {
    const long long k = g_alloc_count.fetch_add(1, std::memory_order_relaxed) + 1;
    return k == g_alloc_fail_at.load(std::memory_order_relaxed);
}
template <class T>
inline cudaError_t dmalloc(T **p, size_t b) {
    if (alloc_fails()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, b);
}
template <class T>
inline cudaError_t dmalloc_async(T **p, size_t b, cudaStream_t st) {
    if (alloc_fails()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync((void **)p, b, st);
}
template <class T>
inline cudaError_t dmalloc_pitch(T **p, size_t *pitch, size_t w, size_t h) {
    if (alloc_fails()) return cudaErrorMemoryAllocation;
    return cudaMallocPitch(p, pitch, w, h);
}
inline cudaError_t dmalloc_array(cudaArray_t *a, const cudaChannelFormatDesc *fd, size_t w, size_t h,
                                 unsigned flags) {
    if (alloc_fails()) return cudaErrorMemoryAllocation;
    return cudaMallocArray(a, fd, w, h, flags);
}
template <class T>
inline cudaError_t hmalloc_mapped(T **p, size_t b) {
    if (alloc_fails()) return cudaErrorMemoryAllocation;
    return cudaHostAlloc((void **)p, b, cudaHostAllocMapped);
}
template <class T>
inline cudaError_t hmalloc(T **p, size_t b) {
    if (alloc_fails()) return cudaErrorMemoryAllocation;
    return cudaMallocHost((void **)p, b);
}

}  // namespace hf

// hf_api.cu: one pose query on a caller-provided lane (a stream and a mapped
// pinned 7-float answer mailbox with its device alias); synchronous
struct hf_fieldset;
int hf_ctx_device(const hf_ctx *c);
// a reference to the context, held by every object made from it
void hf_ctx_retain(hf_ctx *c);
void hf_ctx_release(hf_ctx *c);
// a reference to a part, held by server sessions, their builds in flight and
// batches; the part is freed when the last reference (hf_part_release or
// hf_part_drop) goes
void hf_part_retain(const hf_part *p);
void hf_part_drop(const hf_part *p);
// whether the set's last compute enqueued all of its work
bool hf_fieldset_is_ready(const hf_fieldset *fs);
const void *hf_fieldset_arena_block(const hf_fieldset *fs);  // its arena range, or null
void hf_fieldset_mark_ready(hf_fieldset *fs);
double *hf_fieldset_device_quats(hf_fieldset *fs);
// the E, Fx, Fy, Fz pointers of rotation rot of a set (rot_stride per rotation)
hf::FieldPtrs hf_fieldset_fields(hf_fieldset *fs, int rot);
// a part's gather texture and support box (moving), stored spectrum
// (stationary) and role
cudaTextureObject_t hf_part_texture(const hf_part *p);
const int *hf_part_support(const hf_part *p);
const float2 *hf_part_spectrum(const hf_part *p);
int hf_part_role(const hf_part *p);
// host preparation of a rotation set (float32 matrices, normalised float64
// quaternions, torque neighbours and operators); -1 for a bad quaternion,
// else the number of rank-deficient neighbourhoods
int hf_prepare_rotations(const float *h_quat, int R, bool torque, std::vector<float> &rot9, std::vector<double> &q64,
                         std::vector<int> &nbr, std::vector<float> &P32, std::vector<double> &P64);
// launches of a build for the first R rotations of fs from device rotation data
hf_status hf_set_launch(hf_ctx *ctx, const hf_part *s1, const hf_part *s2, hf_fieldset *fs, int R,
                        const float *d_rot9, const int *d_nbr, const float *d_P, const double *d_P64,
                        cudaStream_t st);
// a field set whose device memory is allocated and freed in stream order on
// `st` (no device-wide synchronisation on create or release); h_stage: a
// caller-owned pinned buffer for its uploads (used if at least R * 308 bytes;
// the caller keeps it unused by others until the set's uploads are done),
// else pageable staging; lanes: 1 or 2 pipelines, 0 for the context's choice;
// arena: when not null the device memory is ranges of it (returned to it on
// release, with no CUDA call), HF_EBUDGET when no free range fits
hf_status hf_fieldset_create_stream_ordered(hf_ctx *ctx, int n, int R, unsigned flags, cudaStream_t st,
                                            hf_fieldset **out, void *h_stage = nullptr, size_t h_stage_bytes = 0,
                                            int lanes = 0, hf::Arena *arena = nullptr);
// checkpoints (hf_api.cu): a computed field set as NPY arrays on an open
// file, and back (device memory stream-ordered on mem_stream if non-null);
// the NPY array helpers and the file tag for the server's session files
hf_status hf_fieldset_write(const hf_fieldset *fs, FILE *f, cudaStream_t st);
hf_status hf_fieldset_read(hf_ctx *ctx, FILE *f, hf_fieldset **out, cudaStream_t mem_stream, cudaStream_t st);
bool hf_ckpt_write_i64(FILE *f, const std::vector<int64_t> &v);
bool hf_ckpt_write_f32(FILE *f, const std::vector<int64_t> &shape, const float *p);
bool hf_ckpt_read_i64(FILE *f, std::vector<int64_t> &v);
bool hf_ckpt_read_f32(FILE *f, std::vector<int64_t> &shape, std::vector<float> &v);
int64_t hf_ckpt_magic();
int64_t hf_ckpt_version();
// a single query's request for the resident query kernel (the checks of
// hf_query); HF_EINVAL / HF_ENOTREADY as hf_query
hf_status hf_query_request(const hf_fieldset *fs, const float t[3], const float q[4], int k, hf::QueryReq *rq);
// launched_ms, when not NULL, receives the steady-clock time (ms) at which
// the query kernel's launch call returned
hf_status hf_query_on_lane(const hf_fieldset *fs, const float t[3], const float q[4], int k, float out7[7],
                           cudaStream_t st, float *h_out, float *d_out, double *launched_ms = nullptr);
